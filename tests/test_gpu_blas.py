"""GPU parity of the fused BLAS-1 reductions (FP64 accumulation) against
numpy on the exported fields."""
import numpy as np
import pytest

import synth
from gpu_common import make_lattice

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 5, 4, 7), (24, 24, 24, 32)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_dot_norm_axpy(dims, prec):
    lat = make_lattice(dims, synth.unit_links(dims), 1.0, 0.1, -1)
    a = synth.gaussian_source(dims, 1)
    b = synth.gaussian_source(dims, 2)
    fa, fb = lat.field(prec).load(a), lat.field(prec).load(b)
    # compare against numpy on the stored (rounded) values
    ra = fa.store(np.zeros_like(a))
    rb = fb.store(np.zeros_like(b))
    d = lat.dot(fa, fb)
    ref = np.vdot(ra, rb)
    assert abs(d - ref) <= 1e-12 * np.linalg.norm(ra) * np.linalg.norm(rb)
    n = lat.norm2(fa)
    assert abs(n - np.vdot(ra, ra).real) <= 1e-12 * n
    alpha = 0.3 - 0.7j
    n2 = lat.axpy_norm(alpha, fa, fb)
    y = fb.store(np.zeros_like(b))
    tol = {0: 1e-13, 1: 1e-6, 2: 2e-3}[prec]
    assert np.linalg.norm(y - (rb + alpha * ra)) <= tol * np.linalg.norm(rb + alpha * ra)
    assert abs(n2 - np.vdot(rb + alpha * ra, rb + alpha * ra).real) <= tol * n2


def test_reductions_are_deterministic():
    dims = (8, 8, 8, 16)
    lat = make_lattice(dims, synth.unit_links(dims), 1.0, 0.1, -1)
    fa = lat.field(0).load(synth.gaussian_source(dims, 3))
    fb = lat.field(0).load(synth.gaussian_source(dims, 4))
    vals = {lat.dot(fa, fb) for _ in range(5)}
    assert len(vals) == 1
