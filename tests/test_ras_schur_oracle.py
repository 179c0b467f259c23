"""Pins of the block-Schur-complement RAS oracle (oracle/ras_schur.py)
against things it does not compute itself: the dense M cut to a block and
Schur-complemented by dense linear algebra, the dense block solve, the
full-lattice RAS of the C oracle where both must agree (kappa = 0), and the
gamma5 symmetry of the adjoint."""
import numpy as np
import pytest

import oracle
import synth
from oracle import ras_schur as rs
from oracle.evenodd import parity

DIMS = (6, 6, 6, 6)


def _setup(seed, kappa=0.13, csw=1.2, tbc=-1):
    U = synth.exp_links(DIMS, 0.4, seed)
    T = oracle.clover_field(DIMS, csw, kappa, U)
    return U, T, kappa, csw, tbc


def _dense_block_M(U, T, kappa, csw, tbc, gsite):
    """Columns of M at the block's sites, rows at the block's sites: M cut to
    the extended block (hops leaving it are absent from the cut)."""
    n = len(gsite)
    D = np.zeros((12 * n, 12 * n), dtype=np.complex128)
    for j in range(n):
        for c in range(12):
            psi = np.zeros((oracle.volume(DIMS), 4, 3), dtype=np.complex128)
            psi[gsite[j], c // 3, c % 3] = 1.0
            D[:, 12 * j + c] = oracle.apply_M(DIMS, tbc, kappa, csw, U, psi, T=T, sites=gsite).reshape(-1)
    return D


@pytest.mark.parametrize("block,bc", [((2, 2, 2, 2), (1, 0, 2, 1)), ((2, 2, 2, 2), (0, 2, 1, 0)),
                                      ((2, 2, 3, 2), (0, 2, 1, 2))])
def test_block_schur_apply_is_the_dense_schur_complement(block, bc):
    U, T, kappa, csw, tbc = _setup(71)
    A = np.eye(12)[None] + T
    gsite, gc, lc, e = rs.block_geometry(DIMS, block, 1, bc)
    D = _dense_block_M(U, T, kappa, csw, tbc, gsite)
    ev = np.repeat(gc.sum(axis=1) % 2 == 0, 12)
    S = D[np.ix_(ev, ev)] - D[np.ix_(ev, ~ev)] @ np.linalg.solve(D[np.ix_(~ev, ~ev)], D[np.ix_(~ev, ev)])
    rng = np.random.default_rng(5)
    for dagger in (False, True):
        psi = rng.standard_normal((len(gsite), 4, 3)) + 1j * rng.standard_normal((len(gsite), 4, 3))
        got = rs.block_schur_apply(DIMS, tbc, kappa, U, A, gsite, gc, lc, e, psi, dagger).reshape(-1)
        op = S.conj().T if dagger else S
        want = op @ psi.reshape(-1)[ev]
        assert np.abs(got[~ev]).max() == 0.0
        assert np.abs(got[ev] - want).max() <= 1e-12 * np.abs(want).max()


def test_many_mr_steps_give_the_dense_block_solve():
    """MR_k for large k converges to M^_B^-1 R_B v on every block, which is
    the even part of the dense solve of M_B [x_e; x_o] = [v_e; 0]."""
    U, T, kappa, csw, tbc = _setup(72, kappa=0.11)
    block = (2, 2, 3, 2)
    v = synth.gaussian_source(DIMS, 9)
    z = rs.ras_schur(DIMS, tbc, kappa, U, T, block, 1, 60, v)
    assert np.abs(z[parity(DIMS) == 1]).max() == 0.0
    for bc in [(0, 0, 0, 0), (2, 1, 1, 2)]:
        gsite, gc, lc, e = rs.block_geometry(DIMS, block, 1, bc)
        D = _dense_block_M(U, T, kappa, csw, tbc, gsite)
        ev = gc.sum(axis=1) % 2 == 0
        rhs = np.where(ev[:, None, None], v[gsite], 0.0).reshape(-1)
        x = np.linalg.solve(D, rhs).reshape(-1, 4, 3)
        core = np.all((lc >= 1) & (lc < 1 + np.array(block)), axis=1) & ev
        assert np.abs(z[gsite[core]] - x[core]).max() <= 1e-9 * np.abs(x[core]).max()


def test_kappa_zero_matches_the_full_lattice_ras():
    """At kappa = 0 both block operators are the site-diagonal A: the block
    Schur RAS of v_e equals the C oracle's full-lattice RAS of the
    zero-extended v_e on the even sites (MR on A leaves zeros at zero)."""
    U = synth.exp_links(DIMS, 0.4, 73)
    T = oracle.clover_field(DIMS, 1.5, 0.13, U)
    v = synth.gaussian_source(DIMS, 10)
    par = np.array([(x + y + z + t) % 2 for t in range(6) for z in range(6) for y in range(6) for x in range(6)])
    assert (par == parity(DIMS)).all()
    ve = np.where((par == 0)[:, None, None], v, 0.0)
    for block, k in [((2, 2, 2, 2), 3), ((2, 2, 3, 2), 5)]:
        got = rs.ras_schur(DIMS, -1, 0.0, U, T, block, 1, k, v)
        want = oracle.ras(DIMS, -1, 0.0, U, T, block, 1, k, ve)
        want[par == 1] = 0.0
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_adjoint_is_gamma5_conjugate():
    """MR on gamma5 M^_B gamma5 from gamma5 v is gamma5 times MR on M^_B from
    v (gamma5 is unitary), so RAS^+(v) = gamma5 RAS(gamma5 v)."""
    U, T, kappa, csw, tbc = _setup(74)
    v = synth.gaussian_source(DIMS, 11)
    g5 = oracle.gamma(4)
    a = rs.ras_schur(DIMS, tbc, kappa, U, T, (2, 2, 2, 2), 1, 4, v, dagger=True)
    b = np.einsum("ab,sbc->sac", g5,
                  rs.ras_schur(DIMS, tbc, kappa, U, T, (2, 2, 2, 2), 1, 4, np.einsum("ab,sbc->sac", g5, v)))
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_shapes_that_do_not_fit_are_rejected():
    with pytest.raises(ValueError):
        rs.block_geometry(DIMS, (4, 2, 2, 2), 1, (0, 0, 0, 0))   # 4 does not divide 6
    with pytest.raises(ValueError):
        rs.block_geometry(DIMS, (3, 2, 2, 2), 2, (0, 0, 0, 0))   # 3 + 2 * 2 > 6
