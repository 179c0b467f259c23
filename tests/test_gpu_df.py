"""GPU parity of the double-FP32 operator (wc_set_fp64_arith(WC_ARITH_DF32)).

The FP64 operator on FP64 fields, computed with each value carried as the
unevaluated sum of two floats (about 47 significant bits) on the FP32
pipes: M, M^+, H and the Schur complement M^ against the oracle at the FP64
tolerance (1e-12 relative to the largest output), every launch shape, the
full 24^3x32 workload on sampled sites, exact equivariance under
power-of-two scaling of the input (which exercises the integer FP64 <->
float-pair conversions across the exponent range), non-finite inputs, and
solves of every kind whose FP64 operator steps run in this arithmetic,
checked with the oracle's M.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_elementwise, gpu_apply, make_lattice, rel_err, wc
from oracle.evenodd import EvenOdd

pytestmark = pytest.mark.gpu

TOL = 1e-12
CASES = [((4, 4, 4, 4), -1), ((6, 4, 8, 10), -1), ((3, 5, 4, 7), 1), ((2, 2, 2, 2), -1), ((5, 3, 2, 6), -1)]


def _df_lattice(dims, U, csw, kappa, tbc):
    w = wc()
    return make_lattice(dims, U, csw, kappa, tbc).set_fp64_arith(w.ARITH_DF32)


@pytest.mark.parametrize("dims,tbc", CASES)
@pytest.mark.parametrize("kind", ["M", "Mdag", "hop"])
def test_df_apply_matches_oracle(dims, tbc, kind):
    kappa, csw = 0.124, 1.3
    U = synth.exp_links(dims, 0.4, 1100 + sum(dims))
    psi = synth.gaussian_source(dims, 1200 + sum(dims))
    lat = _df_lattice(dims, U, csw, kappa, tbc)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    ref = {"M": lambda: op.M(psi), "Mdag": lambda: op.Mdag(psi),
           "hop": lambda: oracle.apply_hop(dims, tbc, U, psi)}[kind]()
    assert_elementwise(gpu_apply(lat, psi, 0, kind), ref, TOL)


def test_df_every_launch_shape_matches_oracle():
    w = wc()
    dims, kappa, csw, tbc = (8, 8, 4, 4), 0.124, 1.2, -1
    U = synth.exp_links(dims, 0.4, 1301)
    psi = synth.gaussian_source(dims, 1302)
    lat = _df_lattice(dims, U, csw, kappa, tbc)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    ref, refd = op.M(psi), op.Mdag(psi)
    tested = 0
    for i in range(24):
        try:
            lat.apply_shape(0, 0, force=i)
            lat.apply_shape(0, 1, force=i)
        except w.WCError:
            continue
        assert_elementwise(gpu_apply(lat, psi, 0, "M"), ref, TOL)
        assert_elementwise(gpu_apply(lat, psi, 0, "Mdag"), refd, TOL)
        tested += 1
    assert tested == 15   # no register cap, or the 128-register cap


def test_df_full_size_sampled():
    """24^3x32 (442,368 sites, the bench workload's lattice) on sampled
    sites against the oracle."""
    dims, U, src, csw, kappa, tbc = synth.config_inputs(2)
    lat = _df_lattice(dims, U, csw, kappa, tbc)
    out = gpu_apply(lat, src, 0, "M")
    V = synth.volume(dims)
    rng = np.random.default_rng(1401)
    sites = np.concatenate([[0, V - 1], rng.choice(V, 3000, replace=False)])
    ref = oracle.apply_M(dims, tbc, kappa, csw, U, src, sites=sites)
    assert np.max(np.abs(out[sites] - ref)) <= TOL * np.max(np.abs(ref))
    assert rel_err(out[sites], ref) <= TOL


def test_df_power_of_two_scaling_is_exact():
    """M(2^k psi) == 2^k M(psi) bit for bit while every intermediate stays a
    normal float: hi and lo of each converted value, every product and its
    rounding error scale exactly.  Covers input magnitudes ~1e-18 .. 1e27."""
    dims, kappa, csw, tbc = (4, 4, 4, 8), 0.13, 1.1, -1
    U = synth.exp_links(dims, 0.4, 1501)
    psi = synth.gaussian_source(dims, 1502)
    lat = _df_lattice(dims, U, csw, kappa, tbc)
    base = gpu_apply(lat, psi, 0, "M")
    for k in (-60, -20, 30, 90):
        s = 2.0 ** k
        assert np.array_equal(gpu_apply(lat, psi * s, 0, "M"), base * s), k


def test_df_zero_and_non_finite_inputs():
    dims, kappa, csw, tbc = (4, 4, 4, 4), 0.12, 1.0, -1
    U = synth.exp_links(dims, 0.3, 1601)
    lat = _df_lattice(dims, U, csw, kappa, tbc)
    psi = np.zeros((synth.volume(dims), 4, 3), complex)
    assert np.array_equal(gpu_apply(lat, psi, 0, "M"), psi)
    psi = synth.gaussian_source(dims, 1602)
    psi[5, 1, 2] = np.nan
    psi[17, 0, 0] = np.inf
    out = gpu_apply(lat, psi, 0, "M")
    assert not np.all(np.isfinite(out[5])) and not np.all(np.isfinite(out[17]))
    # a site far from both stays finite
    assert np.all(np.isfinite(out[200]))


@pytest.mark.parametrize("dims,tbc", [((4, 4, 4, 4), -1), ((6, 4, 8, 10), 1), ((2, 2, 2, 2), -1)])
@pytest.mark.parametrize("dagger", [False, True])
def test_df_schur_matches_oracle(dims, tbc, dagger):
    kappa, csw = 0.13, 1.4
    U = synth.exp_links(dims, 0.5, 1700 + sum(dims))
    lat = _df_lattice(dims, U, csw, kappa, tbc)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    eo = EvenOdd(dims, tbc, kappa, U, op.T)
    psi = synth.gaussian_source(dims, 1710 + sum(dims))
    fi, fo = lat.field(0).load(psi), lat.field(0)
    lat.apply_schur(fo, fi, dagger)
    out = fo.store(np.zeros_like(psi))
    assert np.abs(out[eo.odd]).max() == 0.0
    assert_elementwise(out, eo.schur(psi, dagger), TOL)


def test_df_mode_switch_reload_and_errors():
    """Switching back to FP64 arithmetic reproduces the FP64 result bit for
    bit; links reloaded in double-FP32 mode are used by the next apply; an
    unknown mode is an argument error."""
    w = wc()
    dims, kappa, csw, tbc = (4, 4, 6, 4), 0.12, 1.2, -1
    U = synth.exp_links(dims, 0.4, 1801)
    psi = synth.gaussian_source(dims, 1802)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    native = gpu_apply(lat, psi, 0, "M")
    lat.set_fp64_arith(w.ARITH_DF32)
    assert rel_err(gpu_apply(lat, psi, 0, "M"), native) <= 1e-13
    lat.set_fp64_arith(w.ARITH_F64)
    assert np.array_equal(gpu_apply(lat, psi, 0, "M"), native)
    lat.set_fp64_arith(w.ARITH_DF32)
    U2 = synth.exp_links(dims, 0.4, 1803)
    lat.load_gauge(U2).load_clover(csw, kappa)
    assert_elementwise(gpu_apply(lat, psi, 0, "M"), oracle.apply_M(dims, tbc, kappa, csw, U2, psi), TOL)
    for bad in (2, -1):
        with pytest.raises(w.WCError) as e:
            lat.set_fp64_arith(bad)
        assert e.value.status == 1


def _check_solution(dims, tbc, kappa, csw, U, src, x, tol):
    sol = x.store(np.zeros_like(src))
    r = src - oracle.apply_M(dims, tbc, kappa, csw, U, sol)
    assert np.linalg.norm(r) <= 1.5 * tol * np.linalg.norm(src)


@pytest.mark.parametrize("mode", ["fp64_plain", "flexible_ras", "reliable_ras", "eo_reliable", "eo_nested",
                                  "eo_plain"])
def test_df_solves_reach_tolerance(mode):
    """Every solver kind with its FP64 operator steps in double-FP32
    arithmetic converges to the requested FP64 true residual, checked with
    the oracle's M, in about the iterations of the FP64-arithmetic solve
    (BiCGStab's iteration count moves by ~10 % under a change of rounding
    alone)."""
    w = wc()
    dims, kappa, csw, tbc = (8, 8, 8, 16), 0.125, 1.0, -1
    U = synth.exp_links(dims, 0.3, 1901)
    src = synth.gaussian_source(dims, 1902)
    kw = {"fp64_plain": dict(),
          "flexible_ras": dict(precond=w.PRECOND_RAS, inner_prec=w.F32),
          "reliable_ras": dict(precond=w.PRECOND_RAS, inner_prec=w.F16, solver=w.SOLVER_RELIABLE),
          "eo_reliable": dict(even_odd=True, solver=w.SOLVER_RELIABLE),
          "eo_nested": dict(even_odd=True, solver=w.SOLVER_NESTED, krylov_prec=w.F16),
          "eo_plain": dict(even_odd=True)}[mode]
    tol = 1e-11
    lat = make_lattice(dims, U, csw, kappa, tbc)
    b = lat.field(0).load(src)
    x64 = lat.field(0)
    info64 = lat.solve(x64, b, tol=tol, **kw)
    lat.set_fp64_arith(w.ARITH_DF32)
    x = lat.field(0)
    info = lat.solve(x, b, tol=tol, **kw)
    assert info.status == 0 and info.true_rel_resid <= tol
    _check_solution(dims, tbc, kappa, csw, U, src, x, tol)
    assert info.iters <= 1.2 * info64.iters + 3


def test_df_batch_and_action():
    """A batched even-odd solve and the pseudofermion action in double-FP32
    mode agree with the FP64-arithmetic ones."""
    w = wc()
    dims, kappa, csw, tbc = (4, 4, 4, 8), 0.12, 1.0, -1
    U = synth.exp_links(dims, 0.3, 2001)
    srcs = [synth.gaussian_source(dims, 2002 + i) for i in range(3)]
    lat = _df_lattice(dims, U, csw, kappa, tbc)
    bs = [lat.field(0).load(s) for s in srcs]
    xs = [lat.field(0) for _ in srcs]
    infos = w.solve_batch([lat] * 3, xs, bs, tol=1e-11, even_odd=True, solver=w.SOLVER_RELIABLE)
    for info, x, s in zip(infos, xs, srcs):
        assert info.status == 0
        _check_solution(dims, tbc, kappa, csw, U, s, x, 1e-11)
    F = np.zeros((synth.volume(dims), 4, 3, 3), complex)
    S = lat.action_force(bs[0], F, tol=1e-13, even_odd=True, solver=w.SOLVER_RELIABLE)
    S_ref, F_ref, _, _ = oracle.action_and_force(oracle.Operator(dims, U, csw, kappa, tbc), srcs[0], tol=1e-14)
    assert abs(S - S_ref) <= 1e-11 * S_ref
    assert np.max(np.abs(F - F_ref)) <= 1e-9 * np.max(np.abs(F_ref))
