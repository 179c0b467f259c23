"""Small odd-extent parity cases run by test_gpu_checked.py in a subprocess
against the checked build of the library (WC_LIBRARY=libwc_checked.so):
every operator launch shape, the even-odd Schur operator, both RAS kernels
and the multi-RHS operator against the oracle, then the count of
out-of-range indices the checked kernels met.  Exits non-zero on a parity
failure or any counted violation."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
import synth  # noqa: E402
from gpu_common import assert_elementwise, gpu_apply, make_lattice, wc  # noqa: E402
from oracle.evenodd import EvenOdd  # noqa: E402

TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3}


def main():
    w = wc()
    assert w.LIB_PATH.endswith("libwc_checked.so"), w.LIB_PATH
    # operator, every launch shape, odd extents
    dims, kappa, csw, tbc = (3, 5, 2, 7), 0.123, 1.1, -1
    U = synth.exp_links(dims, 0.4, 91)
    psi = synth.gaussian_source(dims, 92)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    refs = {"M": op.M(psi), "Mdag": op.Mdag(psi), "hop": oracle.apply_hop(dims, tbc, U, psi)}
    shapes = 0
    for prec in (0, 1, 2):
        for i in range(64):
            try:
                for kind in (0, 1, 2):
                    lat.apply_shape(prec, kind, force=i)
            except w.WCError:
                continue
            for kind, ref in refs.items():
                assert_elementwise(gpu_apply(lat, psi, prec, kind), ref, TOL[prec])
            shapes += 1
    # even-odd Schur operator
    dims2 = (4, 2, 6, 4)
    U2 = synth.exp_links(dims2, 0.35, 93)
    psi2 = synth.gaussian_source(dims2, 94)
    lat2 = make_lattice(dims2, U2, csw, kappa, tbc)
    eo = EvenOdd(dims2, tbc, kappa, U2, oracle.clover_field(dims2, csw, kappa, U2))
    ref = eo.schur(psi2)
    for prec in (0, 1, 2):
        a, b = lat2.field(prec).load(psi2), lat2.field(prec)
        lat2.apply_schur(b, a)
        out = b.store(np.zeros_like(psi2))
        assert np.linalg.norm(out - ref) <= TOL[prec] * np.linalg.norm(ref), prec
    # RAS: the cluster kernel (FP32, even extended t) and the one-CTA kernel
    for dims3, block in (((6, 6, 6, 8), (2, 2, 2, 2)), ((6, 6, 6, 9), (3, 3, 3, 3))):
        U3 = synth.haar_links(dims3, 95)
        v = synth.z2_source(dims3, 96)
        lat3 = make_lattice(dims3, U3, 1.0, 0.125, -1)
        ref = oracle.Operator(dims3, U3, 1.0, 0.125, -1).ras(v, block=block, delta=1, k=3)
        for prec, tol in ((1, 1e-6), (2, 1.2e-3)):
            fi, fo = lat3.field(prec).load(v), lat3.field(prec)
            lat3.ras(fo, fi, block=block, overlap=1, mr_iters=3)
            out = fo.store(np.zeros_like(v))
            assert np.isfinite(out).all(), (dims3, prec)
            assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(ref), (dims3, prec)
    # multi-RHS operator
    srcs = [synth.gaussian_source(dims, 100 + r) for r in range(5)]
    ins = [lat.field(1).load(s) for s in srcs]
    outs = [lat.field(1) for _ in srcs]
    lat.apply_multi(outs, ins)
    for s, o in zip(srcs, outs):
        assert_elementwise(o.store(np.zeros_like(s)), op.M(s), 1e-5)
    n = w.checked_violations()
    print(f"checked build: {shapes} launch shapes, even-odd, RAS, multi-RHS; out-of-range indices: {n}")
    return 0 if n == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
