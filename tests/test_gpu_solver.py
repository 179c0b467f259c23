"""GPU RAS preconditioner and BiCGStab solvers against the CPU oracle.

RAS (FP32 arithmetic) is compared element by element with the oracle's FP64
RAS.  Solves are compared through what is unique: the solution of M x = b
(M is nonsingular at these parameters), with the residual of the GPU
solution recomputed by the oracle's own M, and the oracle's BiCGStab
solution as a second reference.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gpu_apply, make_lattice, rel_err, wc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,block,delta,k", [
    ((8, 8, 8, 8), (4, 4, 4, 4), 1, 4),
    ((8, 12, 8, 16), (4, 4, 4, 4), 1, 4),
    ((6, 8, 6, 6), (2, 2, 2, 2), 1, 4),
    ((8, 8, 8, 8), (4, 4, 4, 4), 0, 6),
    ((12, 8, 8, 8), (3, 2, 2, 2), 1, 3),
    ((8, 8, 8, 6), (4, 4, 4, 3), 1, 4),   # odd extended t extent: the one-CTA kernel
    ((8, 8, 8, 8), (2, 2, 2, 2), 2, 2),   # overlap 2: one core t slice per CTA of the pair
    ((8, 8, 9, 8), (4, 4, 3, 4), 1, 4),   # odd extended z: the one-site-per-thread cluster kernel
])
@pytest.mark.parametrize("prec", [1, 2])
def test_ras_matches_oracle(dims, block, delta, k, prec):
    kappa, csw, tbc = 0.125, 1.0, -1
    U = synth.haar_links(dims, 7 + sum(dims))
    v = synth.z2_source(dims, 8)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    ref = op.ras(v, block=block, delta=delta, k=k)
    fi, fo = lat.field(prec).load(v), lat.field(prec)
    lat.ras(fo, fi, block=block, overlap=delta, mr_iters=k)
    out = fo.store(np.zeros_like(v))
    # measured: FP32 <= 1.3e-7 (L2) / 2.6e-7 (elementwise), FP16 storage <= 3.3e-4 / 5.8e-4
    tol = 1e-6 if prec == 1 else 1.2e-3
    assert rel_err(out, ref) <= tol
    assert np.max(np.abs(out - ref)) <= tol * np.max(np.abs(ref))


def test_ras_degenerate_cases():
    dims = (8, 8, 8, 8)
    U = synth.haar_links(dims, 1)
    lat = make_lattice(dims, U, 1.0, 0.12, -1)
    zero = np.zeros((synth.volume(dims), 4, 3), complex)
    fo = lat.field(1)
    lat.ras(fo, lat.field(1).load(zero))
    assert np.count_nonzero(fo.store(np.zeros_like(zero))) == 0
    v = synth.gaussian_source(dims, 2)
    fo2 = lat.field(1).load(v)
    lat.ras(fo2, lat.field(1).load(v), mr_iters=0)
    assert np.count_nonzero(fo2.store(np.zeros_like(zero))) == 0
    w = wc()
    for bad in [dict(block=(3, 4, 4, 4)), dict(block=(4, 4, 4, 4), overlap=2), dict(block=(8, 4, 4, 4)),
                dict(block=(4, 4, 4, 4), overlap=3)]:
        with pytest.raises(w.WCError) as e:
            lat.ras(lat.field(1), lat.field(1), **bad)
        assert e.value.status == 1


def test_fp64_bicgstab_point_source_8x8x8x8():
    """Plain FP64 BiCGStab at the 8^3x8 point-source workload to 1e-12."""
    w = wc()
    dims, U, src, csw, kappa, tbc = synth.config_inputs(1)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    x, b = lat.field(0), lat.field(0).load(src)
    info = lat.solve(x, b, tol=1e-12)
    assert info.status == 0 and info.true_rel_resid <= 1e-12
    sol = x.store(np.zeros_like(src))
    r = src - oracle.apply_M(dims, tbc, kappa, csw, U, sol)
    assert np.linalg.norm(r) <= 1.5e-12 * np.linalg.norm(src)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    ref = oracle.bicgstab(op.M, src, tol=1e-13)
    assert rel_err(sol, ref.x) <= 1e-9


@pytest.mark.parametrize("inner", [1, 2])
def test_mixed_ras_bicgstab(inner):
    dims, kappa, csw, tbc = (8, 8, 8, 16), 0.125, 1.0, -1
    U = synth.haar_links(dims, 21)
    src = synth.z2_source(dims, 22)
    w = wc()
    lat = make_lattice(dims, U, csw, kappa, tbc)
    x, b = lat.field(0), lat.field(0).load(src)
    info = lat.solve(x, b, tol=1e-10, precond=w.PRECOND_RAS, inner_prec=inner)
    assert info.status == 0 and info.true_rel_resid <= 1e-10
    sol = x.store(np.zeros_like(src))
    r = src - oracle.apply_M(dims, tbc, kappa, csw, U, sol)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
    # the preconditioner must help: fewer iterations than the plain solve
    x2 = lat.field(0)
    info2 = lat.solve(x2, b, tol=1e-10)
    assert info.iters < info2.iters


def test_solver_initial_guess_and_resume():
    dims, kappa, csw, tbc = (4, 4, 4, 8), 0.12, 1.0, -1
    U = synth.exp_links(dims, 0.3, 31)
    src = synth.gaussian_source(dims, 32)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    x, b = lat.field(0), lat.field(0).load(src)
    w = wc()
    info = lat.solve(x, b, tol=1e-6, check=False)
    assert info.status == 0
    info2 = lat.solve(x, b, tol=1e-12)       # resume from the previous solution
    assert info2.status == 0 and info2.true_rel_resid <= 1e-12
    info3 = lat.solve(x, b, tol=1e-12)       # already converged: no iteration
    assert info3.iters == 0 and info3.status == 0


def test_solver_error_paths():
    w = wc()
    dims = (4, 4, 4, 8)
    U = synth.exp_links(dims, 0.3, 41)
    lat = make_lattice(dims, U, 1.0, 0.12, -1)
    src = synth.gaussian_source(dims, 42)
    x, b = lat.field(0), lat.field(0).load(src)
    info = lat.solve(x, b, tol=1e-12, max_iter=1, max_restarts=0, check=False)
    assert info.status == 4 and info.iters == 1
    bad = src.copy()
    bad[3, 1, 2] = np.nan
    info = lat.solve(lat.field(0), lat.field(0).load(bad), tol=1e-10, check=False)
    assert info.status == 6
    with pytest.raises(w.WCError) as e:
        lat.solve(lat.field(0), lat.field(1), tol=1e-10)
    assert e.value.status == 1
    with pytest.raises(w.WCError) as e:
        lat.solve(x, b, tol=1e-10, precond=w.PRECOND_RAS, block=(3, 4, 4, 4))
    assert e.value.status == 1
    zero = lat.field(0)
    info = lat.solve(x, zero, tol=1e-10)
    assert info.status == 0 and np.count_nonzero(x.store(np.zeros_like(src))) == 0


@pytest.mark.parametrize("kw", [
    dict(),                                                                   # plain FP64 BiCGStab
    dict(precond=1, inner_prec=1, block=(2, 2, 2, 2)),                        # flexible + FP32 RAS
    dict(solver=1, delta=0.01),                                               # reliable update
    dict(solver=2, inner_tol=0.01, inner_iters=20),                           # nested
    dict(solver=1, delta=0.01, even_odd=True),                                # even-odd reliable
    dict(even_odd=True, krylov_prec=2, solver=1),                             # even-odd, FP16 vectors
])
def test_singular_free_field_stops_with_an_error(kw):
    """Failure injection at a constructed singular point: unit links,
    kappa = 1/8, periodic in every direction.  Then H has eigenvalue 8 on
    constant fields, so M = 1 - kappa H has an exact zero mode and M x = b
    has no solution for a source with a constant component.  Every solver
    kind must stop within max_iter with WC_ERR_NOT_CONVERGED or
    WC_ERR_BREAKDOWN (never report success, never hang)."""
    import time
    dims = (6, 6, 6, 6)
    U = synth.unit_links(dims)
    lat = make_lattice(dims, U, 1.0, 0.125, 1)
    src = synth.gaussian_source(dims, 77) + 1.0   # a constant component along the zero mode
    x, b = lat.field(0), lat.field(0).load(src)
    t0 = time.perf_counter()
    info = lat.solve(x, b, tol=1e-10, max_iter=300, max_restarts=2, check=False, **kw)
    assert time.perf_counter() - t0 < 60
    assert info.status in (4, 5), info
    assert info.iters <= 300


def test_free_field_batch_at_the_singular_point():
    """The batched solver at the same singular point: every right-hand side
    reports an error status, the batch returns."""
    w = wc()
    dims = (4, 4, 4, 4)
    lat = make_lattice(dims, synth.unit_links(dims), 1.0, 0.125, 1)
    srcs = [synth.gaussian_source(dims, 80 + i) + 1.0 for i in range(3)]
    xs = [lat.field(0) for _ in srcs]
    bs = [lat.field(0).load(s) for s in srcs]
    infos = w.solve_batch([lat] * 3, xs, bs, check=False, tol=1e-10, max_iter=200, max_restarts=1,
                          solver=w.SOLVER_RELIABLE)
    assert all(i.status in (4, 5) for i in infos), infos


def _batch_problem(w, dims_list, nrhs, csw=1.0, kappa=0.124):
    lats, xs, bs, srcs, ops = [], [], [], [], []
    for i, dims in enumerate(dims_list):
        U = synth.exp_links(dims, 0.3, 1100 + 10 * i)
        lat = make_lattice(dims, U, csw, kappa, -1)
        for k in range(nrhs):
            src = synth.point_source(dims, spin=k % 4, colour=(k // 4) % 3)
            lats.append(lat)
            xs.append(lat.field(0))
            bs.append(lat.field(0).load(src))
            srcs.append(src)
            ops.append((dims, U))
    return lats, xs, bs, srcs, ops


def test_batch_solve_uneven_lattices():
    """One graph launch over 3 uneven lattices x 3 point sources each; every
    solution checked against the oracle's M, and against the single-RHS
    solver's solution."""
    w = wc()
    lats, xs, bs, srcs, ops = _batch_problem(w, [(6, 6, 6, 8), (8, 8, 8, 8), (8, 6, 8, 12)], 3)
    infos = w.solve_batch(lats, xs, bs, tol=1e-10, precond=w.PRECOND_RAS, inner_prec=1, block=(2, 2, 2, 2))
    for info, lat, x, b, src, (dims, U) in zip(infos, lats, xs, bs, srcs, ops):
        assert info.status == 0 and info.true_rel_resid <= 1e-10
        sol = x.store(np.zeros_like(src))
        r = src - oracle.apply_M(dims, -1, 0.124, 1.0, U, sol)
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
        x1 = lat.field(0)
        lat.solve(x1, b, tol=1e-10, precond=w.PRECOND_RAS, inner_prec=1, block=(2, 2, 2, 2))
        assert rel_err(sol, x1.store(np.zeros_like(src))) <= 1e-8


def test_batch_solve_plain_fp64_and_autotuned_ras():
    w = wc()
    lats, xs, bs, srcs, ops = _batch_problem(w, [(8, 8, 8, 16), (16, 8, 8, 8)], 2)
    infos = w.solve_batch(lats, xs, bs, tol=1e-11)
    assert all(i.status == 0 and i.true_rel_resid <= 1e-11 for i in infos)
    xs2 = [lat.field(0) for lat in lats]
    infos2 = w.solve_batch(lats, xs2, bs, tol=1e-10, precond=w.PRECOND_RAS, inner_prec=2, block=(0, 0, 0, 0))
    for info, x, src, (dims, U) in zip(infos2, xs2, srcs, ops):
        assert info.status == 0
        sol = x.store(np.zeros_like(src))
        r = src - oracle.apply_M(dims, -1, 0.124, 1.0, U, sol)
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
    blk, ov, k = lats[0].ras_autotune(bs[0], inner_prec=2)
    assert np.prod(blk) >= 128 and all(d % b == 0 for d, b in zip(lats[0].dims, blk)) and ov == 1 and k == 4


def test_batch_solve_masks_and_errors():
    """A zero source, an already-solved RHS and an iteration cap in one batch."""
    w = wc()
    dims = (8, 8, 8, 8)
    U = synth.exp_links(dims, 0.3, 77)
    lat = make_lattice(dims, U, 1.0, 0.12, -1)
    src = synth.gaussian_source(dims, 78)
    zero = np.zeros_like(src)
    xs = [lat.field(0) for _ in range(3)]
    bs = [lat.field(0).load(src), lat.field(0).load(zero), lat.field(0).load(src)]
    lat.solve(xs[2], bs[2], tol=1e-12)
    infos = w.solve_batch([lat] * 3, xs, bs, tol=1e-10)
    assert [i.status for i in infos] == [0, 0, 0]
    assert infos[1].iters == 0 and infos[2].iters == 0 and infos[0].iters > 0
    assert np.count_nonzero(xs[1].store(np.zeros_like(src))) == 0
    xs = [lat.field(0) for _ in range(2)]
    infos = w.solve_batch([lat] * 2, xs, [bs[0], bs[2]], tol=1e-12, max_iter=2, check=False)
    assert [i.status for i in infos] == [4, 4] and [i.iters for i in infos] == [2, 2]
    with pytest.raises(w.WCError):
        w.solve_batch([lat, lat], [xs[0], xs[0]], [bs[0], bs[2]], tol=1e-10)


@pytest.mark.parametrize("inner", [1, 2])
def test_reliable_update_solver(inner):
    """FP32 BiCGStab + RAS with FP64 reliable updates reaches the FP64 true
    residual tolerance; checked with the oracle's M."""
    w = wc()
    dims, kappa, csw, tbc = (8, 8, 8, 16), 0.125, 1.0, -1
    U = synth.exp_links(dims, 0.3, 121)
    src = synth.gaussian_source(dims, 122)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    x, b = lat.field(0), lat.field(0).load(src)
    info = lat.solve(x, b, tol=1e-10, precond=w.PRECOND_RAS, inner_prec=inner, solver=w.SOLVER_RELIABLE,
                     delta=0.1)
    assert info.status == 0 and info.true_rel_resid <= 1e-10
    sol = x.store(np.zeros_like(src))
    r = src - oracle.apply_M(dims, tbc, kappa, csw, U, sol)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
    x2 = lat.field(0)
    info2 = lat.solve(x2, b, tol=1e-10, precond=w.PRECOND_RAS, inner_prec=inner)
    assert info.iters <= 3 * info2.iters + 5
    # M^+ through the action: reliable and flexible give the same S
    F = np.zeros((synth.volume(dims), 4, 3, 3), complex)
    phi = lat.field(0).load(src)
    S1 = lat.action_force(phi, F, tol=1e-12, precond=w.PRECOND_RAS, inner_prec=inner, solver=w.SOLVER_RELIABLE)
    S2 = lat.action_force(phi, F, tol=1e-12)
    assert abs(S1 - S2) <= 1e-9 * S2


def test_reliable_update_argument_errors():
    w = wc()
    dims = (8, 8, 8, 8)
    lat = make_lattice(dims, synth.unit_links(dims), 1.0, 0.1, -1)
    x, b = lat.field(0), lat.field(0).load(synth.gaussian_source(dims, 1))
    with pytest.raises(w.WCError) as e:
        lat.solve(x, b, solver=7)                                      # unknown kind
    assert e.value.status == 1
    with pytest.raises(w.WCError) as e:
        lat.solve(x, b, precond=w.PRECOND_RAS, solver=w.SOLVER_RELIABLE, delta=1.5)
    assert e.value.status == 1
    dims_odd = (8, 8, 8, 7)
    lat_odd = make_lattice(dims_odd, synth.unit_links(dims_odd), 1.0, 0.1, -1)
    with pytest.raises(w.WCError) as e:                                # even-odd needs even extents
        lat_odd.solve(lat_odd.field(0), lat_odd.field(0).load(synth.gaussian_source(dims_odd, 2)), even_odd=True)
    assert e.value.status == 1


@pytest.mark.parametrize("inner", [1, 2])
def test_batch_solve_reliable_update(inner):
    """The reliable-update solver inside the batch graph (FP32 steps, FP64
    refreshes as conditional graph nodes) on uneven lattices."""
    w = wc()
    lats, xs, bs, srcs, ops = _batch_problem(w, [(6, 6, 6, 8), (8, 8, 8, 12)], 3)
    infos = w.solve_batch(lats, xs, bs, tol=1e-10, precond=w.PRECOND_RAS, inner_prec=inner, block=(2, 2, 2, 2),
                          solver=w.SOLVER_RELIABLE, delta=0.1)
    for info, x, src, (dims, U) in zip(infos, xs, srcs, ops):
        assert info.status == 0 and info.true_rel_resid <= 1e-10
        sol = x.store(np.zeros_like(src))
        r = src - oracle.apply_M(dims, -1, 0.124, 1.0, U, sol)
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
    xs2 = [lat.field(0) for lat in lats]
    infos2 = w.solve_batch(lats, xs2, bs, tol=1e-12, max_iter=3, precond=w.PRECOND_RAS, inner_prec=inner,
                           block=(2, 2, 2, 2), solver=w.SOLVER_RELIABLE, check=False)
    assert all(i.status == 4 and i.iters == 3 for i in infos2)


@pytest.mark.parametrize("inner", [1, 2])
def test_nested_three_level_solver(inner):
    """FP64 flexible BiCGStab -> FP32 BiCGStab + RAS -> MR blocks, on the
    near-critical 32^3x64 parameters (kappa 0.128, csw 1.6) at 8^4; the
    solution is checked with the oracle's M."""
    w = wc()
    dims, U, src, csw, kappa, tbc = synth.config_inputs(3, dims=(8, 8, 8, 8))
    lat = make_lattice(dims, U, csw, kappa, tbc)
    x, b = lat.field(0), lat.field(0).load(src)
    info = lat.solve(x, b, tol=1e-10, precond=w.PRECOND_RAS, inner_prec=inner, solver=w.SOLVER_NESTED,
                     mr_iters=16, inner_tol=0.05, inner_iters=10)
    assert info.status == 0 and info.true_rel_resid <= 1e-10
    sol = x.store(np.zeros_like(src))
    r = src - oracle.apply_M(dims, tbc, kappa, csw, U, sol)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
    with pytest.raises(w.WCError) as e:
        w.solve_batch([lat], [lat.field(0)], [b], tol=1e-10, precond=w.PRECOND_RAS, solver=w.SOLVER_NESTED)
    assert e.value.status == 1
