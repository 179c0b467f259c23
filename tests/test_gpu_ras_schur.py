"""GPU RAS on block Schur complements (FP32 arithmetic, FP32 and FP16
storage) against the oracle's FP64 form (oracle/ras_schur.py, pinned to
dense linear algebra), element by element; even-odd solves preconditioned
by it, checked with the oracle's full M."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import make_lattice, rel_err, wc
from oracle import ras_schur as rs
from oracle.evenodd import parity

pytestmark = pytest.mark.gpu


def _ras_schur_gpu(lat, v, prec, block, delta, k, dagger=False):
    fi, fo = lat.field(prec).load(v), lat.field(prec)
    lat.ras_schur(fo, fi, block=block, overlap=delta, mr_iters=k, dagger=dagger)
    return fo.store(np.zeros_like(v))


@pytest.mark.parametrize("dims,block,delta,k", [
    ((8, 8, 8, 8), (4, 4, 4, 4), 1, 4),    # 6^4 extended blocks, the solve shape
    ((6, 6, 6, 6), (2, 2, 2, 2), 1, 4),
    ((6, 6, 6, 6), (2, 2, 3, 2), 1, 3),    # odd core z: block parity alternates along z
    ((8, 6, 6, 8), (4, 2, 3, 2), 1, 5),    # anisotropic
    ((8, 8, 8, 8), (4, 4, 4, 4), 0, 6),    # no overlap
    ((12, 8, 8, 8), (2, 2, 2, 2), 2, 2),   # overlap 2
])
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dagger", [False, True])
def test_ras_schur_matches_oracle(dims, block, delta, k, prec, dagger):
    kappa, csw, tbc = 0.125, 1.0, -1
    U = synth.haar_links(dims, 11 + sum(dims))
    v = synth.z2_source(dims, 12)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    T = oracle.clover_field(dims, csw, kappa, U)
    ref = rs.ras_schur(dims, tbc, kappa, U, T, block, delta, k, v, dagger=dagger)
    out = _ras_schur_gpu(lat, v, prec, block, delta, k, dagger)
    assert np.abs(out[parity(dims) == 1]).max() == 0.0
    tol = 1e-6 if prec == 1 else 1.2e-3
    assert rel_err(out, ref) <= tol
    assert np.max(np.abs(out - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (2, 1.2e-3)])
def test_ras_schur_24x24x24x32_sampled_blocks(prec, tol):
    """The full 24^3x32 launch (1728 blocks of 6^4), compared on the cores of
    a sample of blocks, among them blocks on every lattice boundary."""
    dims, U, src, csw, kappa, tbc = synth.config_inputs(2)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    T = oracle.clover_field(dims, csw, kappa, U)
    out = _ras_schur_gpu(lat, src, prec, (4, 4, 4, 4), 1, 4)
    rng = np.random.default_rng(3)
    blocks = [(0, 0, 0, 0), (5, 5, 5, 7), (0, 5, 0, 7)] + [tuple(int(c) for c in rng.integers(0, [6, 6, 6, 8]))
                                                            for _ in range(5)]
    blocks = list(dict.fromkeys(blocks))
    ref = rs.ras_schur(dims, tbc, kappa, U, T, (4, 4, 4, 4), 1, 4, src, blocks=blocks)
    mask = np.zeros(synth.volume(dims), bool)
    for bc in blocks:
        gsite, gc, lc, e = rs.block_geometry(dims, (4, 4, 4, 4), 1, bc)
        core = np.all((lc >= 1) & (lc < 5), axis=1) & (gc.sum(axis=1) % 2 == 0)
        mask[gsite[core]] = True
    assert mask.sum() == len(blocks) * 128
    assert rel_err(out[mask], ref[mask]) <= tol
    assert np.max(np.abs(out[mask] - ref[mask])) <= tol * np.max(np.abs(ref[mask]))
    assert np.abs(out[parity(dims) == 1]).max() == 0.0


def test_ras_schur_degenerate_cases():
    w = wc()
    dims = (8, 8, 8, 8)
    U = synth.haar_links(dims, 1)
    lat = make_lattice(dims, U, 1.0, 0.12, -1)
    zero = np.zeros((synth.volume(dims), 4, 3), complex)
    assert np.count_nonzero(_ras_schur_gpu(lat, zero, 1, (4, 4, 4, 4), 1, 4)) == 0
    v = synth.gaussian_source(dims, 2)
    assert np.count_nonzero(_ras_schur_gpu(lat, v, 1, (4, 4, 4, 4), 1, 0)) == 0
    for bad in [dict(block=(3, 4, 4, 4)),                # does not divide 8
                dict(block=(4, 4, 4, 4), overlap=2)]:    # extended block as large as the lattice
        with pytest.raises(w.WCError) as e:
            lat.ras_schur(lat.field(1), lat.field(1), **bad)
        assert e.value.status == 1
    lat12 = make_lattice((12, 8, 8, 8), synth.haar_links((12, 8, 8, 8), 2), 1.0, 0.12, -1)
    with pytest.raises(w.WCError) as e:   # odd extended x extent (3 + 2)
        lat12.ras_schur(lat12.field(1), lat12.field(1), block=(3, 4, 4, 4), overlap=1)
    assert e.value.status == 1
    with pytest.raises(w.WCError) as e:   # the block shape is not left to the autotuner
        lat.solve(lat.field(0), lat.field(0).load(v), tol=1e-10, even_odd=True, precond=w.PRECOND_RAS,
                  block=(0, 0, 0, 0), ras_schur=True)
    assert e.value.status == 1


@pytest.mark.parametrize("solver,inner", [(0, 1), (1, 2), (2, 2)])
def test_even_odd_solve_with_ras_schur(solver, inner):
    """Flexible (FP32 storage), reliable and nested (FP16 storage) even-odd
    solves preconditioned by the block-Schur RAS, to 1e-10, checked with the
    oracle's M; the same solves with the zero-extension reading for
    comparison of step counts."""
    w = wc()
    dims = (8, 8, 8, 16)
    U = synth.exp_links(dims, 0.3, 1501)
    lat = make_lattice(dims, U, 1.2, 0.128, -1)
    src = synth.gaussian_source(dims, 3)
    b = lat.field(0).load(src)
    kw = dict(tol=1e-10, even_odd=True, precond=w.PRECOND_RAS, inner_prec=inner, solver=solver,
              block=(4, 4, 4, 4), max_iter=2000)
    x = lat.field(0)
    info = lat.solve(x, b, ras_schur=True, **kw)
    assert info.status == 0 and info.true_rel_resid <= 1e-10
    sol = x.store(np.zeros_like(src))
    r = src - oracle.apply_M(dims, -1, 0.128, 1.2, U, sol)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(src)
    info0 = lat.solve(lat.field(0), b, ras_schur=False, **kw)
    assert info0.status == 0
    # both readings precondition the same system; neither may need many
    # more steps than the other
    assert info.iters <= 2 * info0.iters + 2
