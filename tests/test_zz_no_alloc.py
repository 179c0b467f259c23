"""The allocation-free inner product (wc_dot_noalloc) agrees with wc_dot.

wc_dot_noalloc serves callers that must not allocate device memory; it takes
plain device pointers and keeps its reduction scratch in a fixed array
inside the library.  This file sorts last so that a run stopping at the
first failure has already run every other test; it also passes on its own
in a fresh process.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_dot_noalloc_matches_dot_twice_in_a_row():
    import torch

    import paper_1612_06556_gb300 as wc

    dims = (8, 8, 8, 12)
    a = synth.gaussian_source(dims, 901)
    b = synth.gaussian_source(dims, 902)
    lat = wc.Lattice(dims, -1)
    fa, fb = lat.field(wc.F64).load(a), lat.field(wc.F64).load(b)
    ta = torch.from_numpy(a).cuda()
    tb = torch.from_numpy(b).cuda()
    stream = torch.cuda.current_stream()
    outs = [torch.full((2,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    tol = 1e-12 * np.linalg.norm(a) * np.linalg.norm(b)
    free_after_first = None
    for trial in range(2):
        ref = lat.dot(fa, fb)
        torch.cuda.synchronize()
        wc.dot_noalloc(ta, tb, outs[trial], stream)
        torch.cuda.synchronize()
        # the first call on the device may load the library's module (lazy
        # loading); the second must not change the device's free memory
        free = torch.cuda.mem_get_info()[0]
        if trial == 0:
            free_after_first = free
        else:
            assert free == free_after_first
        got = complex(*outs[trial].cpu().numpy())
        assert abs(got - ref) <= tol, (trial, got, ref)
        assert abs(got - np.vdot(a, b)) <= tol


@pytest.mark.parametrize("n", [0, 1, 4097, 8388608])
def test_dot_noalloc_sizes_against_numpy(n):
    """Empty input (one block, zero result), a ragged last chunk, and the
    largest size the fixed scratch holds (2048 blocks)."""
    import torch

    import paper_1612_06556_gb300 as wc

    rng = np.random.default_rng(n + 5)
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        wc.dot_noalloc(ta, tb, out, torch.cuda.current_stream())
        got = complex(*out.cpu().numpy())
        ref = np.vdot(a, b)
        assert abs(got - ref) <= 1e-12 * max(1.0, np.linalg.norm(a) * np.linalg.norm(b)), (n, got, ref)


def test_dot_noalloc_rejects_sizes_beyond_its_maximum():
    import torch

    import paper_1612_06556_gb300 as wc

    x = torch.zeros(4, dtype=torch.complex128, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = wc._L.wc_dot_noalloc(wc._vp(x.data_ptr()), wc._vp(x.data_ptr()), 8388608 + 1,
                              wc._vp(out.data_ptr()), None)
    assert st == 1
    assert "maximum" in wc._L.wc_last_error(None).decode()
