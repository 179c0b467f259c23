"""GPU parity of the multi-right-hand-side operator (wc_apply_multi).

Every out_r of one launch against the oracle's M (or M^+) of in_r at the
FP32 tolerance 1e-5, for 1, 5, 12 and 16 fields, on lattices whose volume
is not a multiple of the 32-site CTA tile and with both time boundary
conditions; identical to separate single-field applies up to FP32 rounding
order; argument errors before any launch.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_elementwise, gpu_apply, make_lattice, rel_err, wc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,tbc,n", [((4, 4, 4, 8), -1, 12), ((6, 5, 4, 7), 1, 5), ((2, 2, 2, 2), -1, 16),
                                         ((8, 6, 6, 4), -1, 1)])
@pytest.mark.parametrize("dagger", [False, True])
def test_multi_apply_matches_oracle(dims, tbc, n, dagger):
    kappa, csw = 0.126, 1.4
    U = synth.exp_links(dims, 0.4, 500 + n)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    srcs = [synth.gaussian_source(dims, 600 + r) for r in range(n)]
    ins = [lat.field(1).load(s) for s in srcs]
    outs = [lat.field(1) for _ in range(n)]
    lat.apply_multi(outs, ins, dagger)
    for r in range(n):
        ref = op.Mdag(srcs[r]) if dagger else op.M(srcs[r])
        got = outs[r].store(np.zeros_like(srcs[r]))
        assert_elementwise(got, ref, 1e-5)
        single = gpu_apply(lat, srcs[r], 1, "Mdag" if dagger else "M")
        assert rel_err(got, single) <= 1e-6


def test_multi_apply_full_size_sampled():
    """24^3x32 with 12 Z2 sources: sampled sites of every output against the
    oracle."""
    dims, U, _, csw, kappa, tbc = synth.config_inputs(2)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    srcs = [synth.z2_source(dims, 2100 + r) for r in range(12)]
    ins = [lat.field(1).load(s) for s in srcs]
    outs = [lat.field(1) for _ in range(12)]
    lat.apply_multi(outs, ins)
    sites = np.random.default_rng(4).choice(synth.volume(dims), 1000, replace=False)
    for r in (0, 7, 11):
        ref = oracle.apply_M(dims, tbc, kappa, csw, U, srcs[r], sites=sites)
        got = outs[r].store(np.zeros_like(srcs[r]))[sites]
        assert rel_err(got, ref) <= 1e-5


def test_multi_apply_argument_errors():
    w = wc()
    dims = (4, 4, 4, 4)
    lat = make_lattice(dims, synth.unit_links(dims), 1.0, 0.12, -1)
    a = [lat.field(1) for _ in range(17)]
    b = [lat.field(1) for _ in range(17)]
    with pytest.raises(w.WCError) as e:
        lat.apply_multi(a, b)                                   # n > 16
    assert e.value.status == 1
    with pytest.raises(w.WCError) as e:
        lat.apply_multi([], [])                                 # n = 0
    assert e.value.status == 1
    with pytest.raises(w.WCError) as e:
        lat.apply_multi([lat.field(0)], [lat.field(0)])         # FP64
    assert e.value.status == 1
    with pytest.raises(w.WCError) as e:
        lat.apply_multi([a[0], a[1]], [a[1], b[1]])             # out aliases an in
    assert e.value.status == 1
    with pytest.raises(w.WCError) as e:
        lat.apply_multi([a[0], a[0]], [b[0], b[1]])             # repeated out
    assert e.value.status == 1
