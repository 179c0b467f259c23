"""GPU parity of the even-odd (Schur complement) operator and solves.

M^ = A_ee - k^2 H_eo A_oo^-1 H_oe and M^+ through wc_apply_schur in FP64,
FP32 and FP16 storage, element by element against the oracle's EvenOdd
(itself pinned to the full operator by block elimination, the solve
round trip and det M = det A_oo det M^).  Tolerances as for M: 1e-12, 1e-5,
5e-3 relative.  Even-odd solves of every solver kind are checked with the
oracle's full M.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_elementwise, make_lattice, wc
from oracle.evenodd import EvenOdd

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3}
CASES = [((4, 4, 4, 4), -1), ((6, 4, 8, 10), 1), ((2, 2, 2, 2), -1), ((8, 2, 4, 6), -1), ((10, 6, 2, 4), 1)]


def _setup(dims, tbc, seed, kappa=0.13, csw=1.4):
    U = synth.exp_links(dims, 0.5, seed)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    return U, lat, op, EvenOdd(dims, tbc, kappa, U, op.T)


def _gpu_schur(lat, psi, prec, dagger):
    fi = lat.field(prec).load(psi)
    fo = lat.field(prec)
    lat.apply_schur(fo, fi, dagger)
    return fo.store(np.zeros_like(psi))


@pytest.mark.parametrize("dims,tbc", CASES)
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("dagger", [False, True])
def test_schur_matches_oracle(dims, tbc, prec, dagger):
    U, lat, op, eo = _setup(dims, tbc, 700 + sum(dims))
    psi = synth.gaussian_source(dims, 710 + sum(dims))
    out = _gpu_schur(lat, psi, prec, dagger)
    assert np.abs(out[eo.odd]).max() == 0.0
    # the odd half of the input is ignored
    assert_elementwise(out, eo.schur(psi, dagger), TOL[prec])


@pytest.mark.parametrize("n", [1, 5, 12, 16])
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dagger", [False, True])
def test_schur_multi_matches_oracle(n, prec, dagger):
    """The multi-RHS Schur operator (one odd and one even pass for all n
    fields, links, A and A^-1 shared) on a volume whose last CTA is ragged
    (432 sites per parity, CTAs of 32), every field against the oracle and
    against the single-field operator."""
    dims, tbc = (6, 4, 6, 6), -1
    U, lat, op, eo = _setup(dims, tbc, 720 + n)
    srcs = [synth.gaussian_source(dims, 730 + r) for r in range(n)]
    ins = [lat.field(prec).load(s) for s in srcs]
    outs = [lat.field(prec) for _ in srcs]
    lat.apply_schur_multi(outs, ins, dagger)
    for s, o in zip(srcs, outs):
        got = o.store(np.zeros_like(s))
        assert np.abs(got[eo.odd]).max() == 0.0
        assert_elementwise(got, eo.schur(s, dagger), TOL[prec])
        assert_elementwise(got, _gpu_schur(lat, s, prec, dagger), 1e-6 if prec == 1 else 2e-3)


def test_schur_multi_argument_errors():
    w = wc()
    dims = (4, 4, 4, 4)
    U, lat, op, eo = _setup(dims, -1, 11)
    a, b = lat.field(1), lat.field(1)
    for outs, ins in [([a], [a]), ([a, a], [b, b]), ([lat.field(0)], [lat.field(0)]), ([a] * 17, [b] * 17)]:
        with pytest.raises(w.WCError) as e:
            lat.apply_schur_multi(outs, ins)
        assert e.value.status == 1


def test_schur_full_size_sampled():
    """24^3x32 (a half lattice of 221,184 sites per parity) in FP32: every
    odd site zero, sampled even sites against the oracle composition."""
    dims, tbc = (24, 24, 24, 32), -1
    U, lat, op, eo = _setup(dims, tbc, 901, kappa=0.125, csw=1.0)
    psi = synth.z2_source(dims, 902)
    out = _gpu_schur(lat, psi, 1, False)
    assert np.abs(out[eo.odd]).max() == 0.0
    # the reference on the full lattice is a few seconds of numpy; compare a
    # sample of even sites
    ref = eo.schur(psi)
    rng = np.random.default_rng(903)
    sites = rng.choice(np.flatnonzero(eo.even), 4096, replace=False)
    assert_elementwise(out[sites], ref[sites], TOL[1])


def test_schur_argument_errors():
    w = wc()
    dims = (4, 3, 4, 4)
    lat = make_lattice(dims, synth.unit_links(dims), 1.0, 0.12, -1)
    a, b = lat.field(0), lat.field(0)
    with pytest.raises(w.WCError) as e:
        lat.apply_schur(a, b)                       # odd y extent
    assert e.value.status == 1
    dims = (4, 4, 4, 4)
    lat = make_lattice(dims, synth.unit_links(dims), 1.0, 0.12, -1)
    a, c = lat.field(0), lat.field(1)
    with pytest.raises(w.WCError):
        lat.apply_schur(a, a)
    with pytest.raises(w.WCError):
        lat.apply_schur(a, c)


def test_schur_after_reloading_clover():
    """The clover inverse follows a new kappa / csw."""
    dims, tbc = (4, 4, 4, 8), -1
    U, lat, op, eo = _setup(dims, tbc, 55)
    psi = synth.gaussian_source(dims, 56)
    _gpu_schur(lat, psi, 0, False)
    lat.load_clover(0.7, 0.11)
    op2 = oracle.Operator(dims, U, 0.7, 0.11, tbc)
    eo2 = EvenOdd(dims, tbc, 0.11, U, op2.T)
    assert_elementwise(_gpu_schur(lat, psi, 0, False), eo2.schur(psi), TOL[0])


@pytest.mark.parametrize("solver", [0, 1, 2])
def test_even_odd_solve(solver):
    """Every solver kind on M^ (FLEXIBLE: plain FP64; RELIABLE: FP32 with FP64
    reliable updates; NESTED: FP64 outer, FP32 inner BiCGStab) reaches the
    FP64 true residual of the full system; the solution is checked with the
    oracle's M and the iteration count against the full-lattice solve."""
    w = wc()
    dims, kappa, csw, tbc = (8, 8, 8, 16), 0.125, 1.0, -1
    U = synth.exp_links(dims, 0.3, 131)
    src = synth.gaussian_source(dims, 132)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    x, b = lat.field(0), lat.field(0).load(src)
    info = lat.solve(x, b, tol=1e-10, solver=solver, even_odd=True, max_iter=2000)
    assert info.status == 0 and info.true_rel_resid <= 1e-10
    sol = x.store(np.zeros_like(src))
    r = src - oracle.apply_M(dims, tbc, kappa, csw, U, sol)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
    if solver == 0:
        full = lat.solve(lat.field(0), b, tol=1e-10, max_iter=2000)
        assert info.iters < full.iters


@pytest.mark.parametrize("solver,krylov,arith", [(0, 1, 0), (1, 1, 0), (1, 2, 0), (1, 2, 1), (2, 2, 1)])
def test_even_odd_reported_residual_is_that_of_the_solution(solver, krylov, arith):
    """The full residual an even-odd solve reports (x_o reconstructed
    together with the odd-site residual in one pass, the even sites in a
    second) is |b - M x| / |b| of the x it returns, recomputed by the
    oracle; also for a solve stopped after one step."""
    w = wc()
    dims, kappa, csw, tbc = (8, 8, 8, 16), 0.125, 1.0, -1
    U = synth.exp_links(dims, 0.3, 151)
    src = synth.gaussian_source(dims, 152)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    lat.set_fp64_arith(arith)
    b = lat.field(0).load(src)
    for max_iter, tol in [(2000, 1e-10), (1, 1e-14)]:
        x = lat.field(0)
        info = lat.solve(x, b, tol=tol, solver=solver, krylov_prec=krylov, even_odd=True, max_iter=max_iter,
                         max_restarts=0, check=False)
        sol = x.store(np.zeros_like(src))
        ref = np.linalg.norm(src - oracle.apply_M(dims, tbc, kappa, csw, U, sol)) / np.linalg.norm(src)
        assert abs(info.true_rel_resid - ref) <= 1e-3 * ref + 1e-14
        if max_iter == 2000:
            assert info.status == 0 and ref <= 1e-10
        else:
            assert info.status != 0 and ref > 1e-6


@pytest.mark.parametrize("margin", ["0", "1e3"])
def test_even_odd_reliable_confirmation_paths(margin, monkeypatch):
    """Even-odd reliable solves with the half solve's own FP64 confirmation
    (margin 0) and with a deferral margin so large that the full-residual
    check fails and the half solve resumes (reported as a restart): both end
    converged, checked with the oracle's M."""
    w = wc()
    dims, kappa, csw, tbc = (8, 8, 8, 16), 0.125, 1.0, -1
    U = synth.exp_links(dims, 0.3, 161)
    src = synth.gaussian_source(dims, 162)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    b = lat.field(0).load(src)
    kw = dict(tol=1e-10, solver=w.SOLVER_RELIABLE, krylov_prec=w.F16, even_odd=True, max_iter=2000)
    monkeypatch.setenv("WC_EO_DEFER_MARGIN", margin)
    x = lat.field(0)
    info = lat.solve(x, b, **kw)
    assert info.status == 0 and info.true_rel_resid <= 1e-10
    sol = x.store(np.zeros_like(src))
    r = src - oracle.apply_M(dims, tbc, kappa, csw, U, sol)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
    assert info.restarts == (0 if margin == "0" else 1)


@pytest.mark.parametrize("margin", ["0", "1e3"])
@pytest.mark.parametrize("krylov", [1, 2])
def test_even_odd_batch_confirmation_paths(margin, krylov, monkeypatch):
    """The batched even-odd reliable solve with its half solves confirming
    in FP64 themselves (margin 0), and with a margin so large that every
    full-residual confirmation fails and each Schur solve resumes on the
    host: every source converges, checked with the oracle's M."""
    w = wc()
    monkeypatch.setenv("WC_EO_DEFER_MARGIN", margin)
    dims = (6, 6, 6, 8)
    U = synth.exp_links(dims, 0.3, 1700)
    lat = make_lattice(dims, U, 1.0, 0.124, -1)
    srcs = [synth.point_source(dims, spin=k, colour=2 - k) for k in range(3)]
    xs = [lat.field(0) for _ in srcs]
    bs = [lat.field(0).load(src) for src in srcs]
    infos = w.solve_batch([lat] * 3, xs, bs, tol=1e-10, solver=w.SOLVER_RELIABLE, krylov_prec=krylov,
                          even_odd=True, max_iter=2000)
    for info, x, src in zip(infos, xs, srcs):
        assert info.status == 0 and info.true_rel_resid <= 1e-10
        assert info.restarts == (0 if margin == "0" else 1)
        sol = x.store(np.zeros_like(src))
        r = src - oracle.apply_M(dims, -1, 0.124, 1.0, U, sol)
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)


def test_even_odd_action_and_zero_source():
    """M^+ solves through the action (even-odd vs full lattice give the same
    S), and a zero source gives x = 0."""
    w = wc()
    dims, kappa, csw, tbc = (4, 4, 8, 8), 0.12, 1.2, -1
    U = synth.exp_links(dims, 0.4, 141)
    src = synth.gaussian_source(dims, 142)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    F1 = np.zeros((synth.volume(dims), 4, 3, 3), complex)
    F2 = np.zeros_like(F1)
    phi = lat.field(0).load(src)
    S1 = lat.action_force(phi, F1, tol=1e-12, even_odd=True)
    S2 = lat.action_force(phi, F2, tol=1e-12)
    assert abs(S1 - S2) <= 1e-9 * S2
    assert np.abs(F1 - F2).max() <= 1e-8 * np.abs(F2).max()
    x, z = lat.field(0).load(src), lat.field(0)
    info = lat.solve(x, z, tol=1e-10, even_odd=True)
    assert info.status == 0
    assert np.abs(x.store(np.zeros_like(src))).max() == 0.0


@pytest.mark.parametrize("solver", [0, 1])
def test_even_odd_batch(solver):
    """Even-odd inside the batched graph: 2 uneven lattices x 3 point sources
    (several Schur solves on one lattice run concurrently, each with its own
    odd-site intermediate); every solution checked with the oracle's full M;
    an odd extent is an argument error."""
    w = wc()
    lats, xs, bs, srcs, ops = [], [], [], [], []
    for i, dims in enumerate([(6, 6, 6, 8), (8, 4, 8, 12)]):
        U = synth.exp_links(dims, 0.3, 1300 + 10 * i)
        lat = make_lattice(dims, U, 1.0, 0.124, -1)
        for k in range(3):
            src = synth.point_source(dims, spin=k, colour=k)
            lats.append(lat)
            xs.append(lat.field(0))
            bs.append(lat.field(0).load(src))
            srcs.append(src)
            ops.append((dims, U))
    infos = w.solve_batch(lats, xs, bs, tol=1e-10, solver=solver, even_odd=True, max_iter=2000)
    for info, x, src, (dims, U) in zip(infos, xs, srcs, ops):
        assert info.status == 0 and info.true_rel_resid <= 1e-10
        sol = x.store(np.zeros_like(src))
        r = src - oracle.apply_M(dims, -1, 0.124, 1.0, U, sol)
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
    dims = (6, 5, 6, 8)
    lat = make_lattice(dims, synth.unit_links(dims), 1.0, 0.12, -1)
    with pytest.raises(w.WCError) as e:
        w.solve_batch([lat], [lat.field(0)], [lat.field(0).load(synth.z2_source(dims, 3))], tol=1e-10,
                      even_odd=True)
    assert e.value.status == 1


@pytest.mark.parametrize("krylov", [1, 2])
def test_lockstep_batch(krylov, monkeypatch):
    """Reliable-update even-odd batch of 19 right-hand sides on one lattice:
    the lockstep schedule (groups of up to 16 stepping together, both Schur
    applications of a step in one multi-RHS launch) holds 16 + 3 of them; a
    zero source starts inactive, sources of different structure stop after
    different step counts.  Every solution is checked with the oracle's full
    M, and the step counts against one branch per right-hand side."""
    w = wc()
    dims = (6, 6, 6, 8)
    U = synth.exp_links(dims, 0.3, 1401)
    lat = make_lattice(dims, U, 1.0, 0.124, -1)
    srcs = [synth.point_source(dims, spin=k % 4, colour=k % 3, site=7 * k) for k in range(12)]
    srcs += [synth.gaussian_source(dims, 40 + k) for k in range(5)]
    srcs += [np.zeros_like(srcs[0]), synth.z2_source(dims, 7)]
    bs = [lat.field(0).load(s) for s in srcs]
    monkeypatch.setenv("WC_BATCH_LOCKSTEP", "1")

    def run():
        xs = [lat.field(0) for _ in srcs]
        infos = w.solve_batch([lat] * len(srcs), xs, bs, tol=1e-10, solver=w.SOLVER_RELIABLE, even_odd=True,
                              krylov_prec=krylov, max_iter=3000)
        return infos, [x.store(np.zeros_like(s)) for x, s in zip(xs, srcs)]

    infos, sols = run()
    for info, sol, src in zip(infos, sols, srcs):
        assert info.status == 0 and info.true_rel_resid <= 1e-10
        r = src - oracle.apply_M(dims, -1, 0.124, 1.0, U, sol)
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
    assert np.abs(sols[17]).max() == 0.0
    steps = [i.iters for i in infos]
    assert len(set(steps)) > 1   # the members stop at different steps
    monkeypatch.setenv("WC_BATCH_LOCKSTEP", "0")
    infos0, _ = run()
    for a, b in zip(infos, infos0):
        assert b.status == 0
        assert abs(a.iters - b.iters) <= max(3, 0.1 * b.iters)


@pytest.mark.parametrize("krylov", [1, 2])
def test_near_critical_32x32x32x64_nested_solve(krylov):
    """The 32^3x64 system at kappa 0.128, csw 1.6 (near-critical: plain and
    reliable-update BiCGStab stagnate near 1e-8) solved to 1e-10 by the
    three-level solver on the even-odd operator with FP32 or FP16 inner
    vectors (the configuration's FP16 storage), as the bench runs it; the
    residual checked with the oracle's M on 2000 sampled sites."""
    w = wc()
    dims, U, src, csw, kappa, tbc = synth.config_inputs(3)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    x, b = lat.field(0), lat.field(0).load(src)
    info = lat.solve(x, b, tol=1e-10, solver=w.SOLVER_NESTED, even_odd=True, inner_tol=0.01, inner_iters=100,
                     krylov_prec=krylov, max_iter=60)
    assert info.status == 0 and info.true_rel_resid <= 1e-10
    sol = x.store(np.zeros_like(src))
    sites = np.random.default_rng(5).choice(synth.volume(dims), 2000, replace=False)
    r = src[sites] - oracle.apply_M(dims, tbc, kappa, csw, U, sol, sites=sites)
    # a sample of the residual: bounded by the full residual's scale
    assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(src[sites])


@pytest.mark.parametrize("solver,inner", [(0, 1), (1, 2), (2, 1)])
def test_even_odd_with_ras(solver, inner):
    """The paper's inner configuration: even-odd and RAS together (RAS of the
    full lattice on the even vector extended by zeros, restricted to the
    even sites).  Flexible + FP32 RAS, reliable + FP16 RAS, nested + FP32
    RAS on M^; solutions checked with the oracle's M; the RAS-preconditioned
    flexible solve takes fewer steps than the unpreconditioned one (a
    moderately conditioned system: on near-critical ones the FP32 block
    solves stop paying, as on the full lattice)."""
    w = wc()
    dims, kappa, csw, tbc = (8, 8, 8, 16), 0.124, 1.0, -1
    U = synth.exp_links(dims, 0.3, 151)
    src = synth.gaussian_source(dims, 152)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    x, b = lat.field(0), lat.field(0).load(src)
    info = lat.solve(x, b, tol=1e-10, even_odd=True, precond=w.PRECOND_RAS, inner_prec=inner, solver=solver,
                     block=(4, 4, 4, 4), mr_iters=8, max_iter=2000)
    assert info.status == 0 and info.true_rel_resid <= 1e-10
    sol = x.store(np.zeros_like(src))
    r = src - oracle.apply_M(dims, tbc, kappa, csw, U, sol)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
    if solver == 0:
        plain = lat.solve(lat.field(0), b, tol=1e-10, even_odd=True, max_iter=2000)
        assert info.iters < plain.iters
        # in the batched graph too (explicit block shape)
        xs = [lat.field(0), lat.field(0)]
        infos = w.solve_batch([lat, lat], xs, [b, b], tol=1e-10, even_odd=True, precond=w.PRECOND_RAS,
                              inner_prec=inner, block=(4, 4, 4, 4), mr_iters=8, max_iter=2000)
        for i, xx in zip(infos, xs):
            assert i.status == 0
            r = src - oracle.apply_M(dims, tbc, kappa, csw, U, xx.store(np.zeros_like(src)))
            assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
        with pytest.raises(w.WCError):
            w.solve_batch([lat], [lat.field(0)], [b], tol=1e-10, even_odd=True, precond=w.PRECOND_RAS,
                          block=(0, 0, 0, 0))


@pytest.mark.parametrize("solver,even_odd,precond", [(1, True, 0), (2, True, 0), (1, False, 1), (2, True, 1)])
def test_fp16_krylov_vectors(solver, even_odd, precond):
    """krylov_prec = FP16: the low-precision BiCGStab vectors and operator of
    the reliable-update and nested solvers on FP16 storage (per-site scale,
    FP32 arithmetic), with and without even-odd and RAS; the FP64 true
    residual still reaches 1e-10, checked with the oracle's M; also inside
    the batched graph."""
    w = wc()
    dims, kappa, csw, tbc = (8, 8, 8, 16), 0.124, 1.0, -1
    U = synth.exp_links(dims, 0.3, 161)
    src = synth.gaussian_source(dims, 162)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    x, b = lat.field(0), lat.field(0).load(src)
    kw = dict(tol=1e-10, solver=solver, even_odd=even_odd, precond=precond, krylov_prec=w.F16, max_iter=3000,
              block=(4, 4, 4, 4))
    info = lat.solve(x, b, **kw)
    assert info.status == 0 and info.true_rel_resid <= 1e-10
    sol = x.store(np.zeros_like(src))
    r = src - oracle.apply_M(dims, tbc, kappa, csw, U, sol)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
    if solver == 1:
        xs = [lat.field(0), lat.field(0)]
        infos = w.solve_batch([lat, lat], xs, [b, b], **kw)
        for i, xx in zip(infos, xs):
            assert i.status == 0
            r = src - oracle.apply_M(dims, tbc, kappa, csw, U, xx.store(np.zeros_like(src)))
            assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)


def test_singular_clover_block_is_reported():
    """A constant abelian flux b = pi/2 in the xy plane gives A = 1 + T with
    T = csw kappa sin(b) diag(1,-1,1,-1) (x) diag(1,-1,0) at every site; with
    csw kappa = 1 the blocks of A are singular, so the even-odd operator and
    solves report WC_ERR_BREAKDOWN instead of dividing by (almost) zero,
    while the full-lattice operator still applies."""
    w = wc()
    dims = (4, 4, 2, 2)
    Lx, Ly = dims[0], dims[1]
    b = 2 * np.pi * 4 / (Lx * Ly)
    tau = np.array([1.0, -1.0, 0.0])
    U = synth.unit_links(dims)
    V = synth.volume(dims)
    for s in range(V):
        x, y = s % Lx, (s // Lx) % Ly
        U[s, 1] = np.diag(np.exp(1j * b * x * tau))
        if x == Lx - 1:
            U[s, 0] = np.diag(np.exp(-1j * b * Lx * y * tau))
    lat = make_lattice(dims, U, 8.0, 0.125, -1)
    psi = synth.gaussian_source(dims, 3)
    with pytest.raises(w.WCError) as e:
        lat.apply_schur(lat.field(0), lat.field(0).load(psi))
    assert e.value.status == 5
    with pytest.raises(w.WCError) as e:
        lat.solve(lat.field(0), lat.field(0).load(psi), tol=1e-10, even_odd=True)
    assert e.value.status == 5
    out = lat.field(0)
    lat.apply_M(out, lat.field(0).load(psi))
    ref = oracle.apply_M(dims, -1, 0.125, 8.0, U, psi)
    assert_elementwise(out.store(np.zeros_like(psi)), ref, 1e-12)


def test_batch_pools_survive_clover_reload_and_destroy():
    """The solver states and half-lattice fields a lattice keeps for its
    batches are reused by a batch after a clover reload with another kappa
    (A^-1 rebuilt, same half lattice) and freed with the lattice; the
    solutions stay correct."""
    w = wc()
    dims = (6, 6, 6, 8)
    U = synth.exp_links(dims, 0.3, 1601)
    lat = make_lattice(dims, U, 1.0, 0.124, -1)
    srcs = [synth.point_source(dims, spin=k, colour=k % 3) for k in range(4)]
    for kappa in (0.124, 0.12):
        if kappa != 0.124:
            lat.load_clover(1.0, kappa)
        xs = [lat.field(0) for _ in srcs]
        infos = w.solve_batch([lat] * 4, xs, [lat.field(0).load(s) for s in srcs], tol=1e-10,
                              solver=w.SOLVER_RELIABLE, even_odd=True)
        for info, x, s in zip(infos, xs, srcs):
            assert info.status == 0
            r = s - oracle.apply_M(dims, -1, kappa, 1.0, U, x.store(np.zeros_like(s)))
            assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(s)
    lat.close()


def test_lockstep_member_with_nan_source_does_not_disturb_the_group(monkeypatch):
    """A source with a NaN entry in a lockstep group: that right-hand side
    reports WC_ERR_NAN and skips every step; the other members of its group
    converge to the oracle's solutions."""
    w = wc()
    monkeypatch.setenv("WC_BATCH_LOCKSTEP", "1")
    dims = (6, 6, 6, 8)
    U = synth.exp_links(dims, 0.3, 1701)
    lat = make_lattice(dims, U, 1.0, 0.124, -1)
    srcs = [synth.point_source(dims, spin=k, colour=k % 3) for k in range(4)]
    bad = synth.gaussian_source(dims, 1702)
    bad[5, 1, 2] = np.nan
    srcs.insert(2, bad)
    xs = [lat.field(0) for _ in srcs]
    infos = w.solve_batch([lat] * len(srcs), xs, [lat.field(0).load(s) for s in srcs], tol=1e-10,
                          solver=w.SOLVER_RELIABLE, even_odd=True, check=False)
    assert infos[2].status == 6   # WC_ERR_NAN
    for k, (info, x, s) in enumerate(zip(infos, xs, srcs)):
        if k == 2:
            continue
        assert info.status == 0
        r = s - oracle.apply_M(dims, -1, 0.124, 1.0, U, x.store(np.zeros_like(s)))
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(s)
