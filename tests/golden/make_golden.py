"""Write oracle_regression_4x4x4x4.json: values of the FP64 CPU oracle on a
small seeded configuration, so that any later change of the oracle's
arithmetic shows up as a failing regression test (tests/test_oracle_pins.py,
test_oracle_matches_stored_regression_values).  Calls only oracle/ and the
seeded input generators; no value here comes from the GPU library.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle.evenodd import EvenOdd  # noqa: E402

DIMS, TBC, KAPPA, CSW = (4, 4, 4, 4), -1, 0.12, 1.3
SITES = [0, 5, 77, 128, 255]


def compute():
    U = synth.exp_links(DIMS, 0.4, 4401)
    psi = synth.gaussian_source(DIMS, 4402)
    op = oracle.Operator(DIMS, U, CSW, KAPPA, TBC)
    Mpsi = op.M(psi)
    Hpsi = oracle.apply_hop(DIMS, TBC, U, psi)
    T = op.T
    eo = EvenOdd(DIMS, TBC, KAPPA, U, T)
    schur = eo.schur(psi)
    S, F, _, _ = oracle.action_and_force(op, psi, tol=1e-14)

    def cplx(a):
        return [[float(v.real), float(v.imag)] for v in np.asarray(a).reshape(-1)]

    return {
        "config": {"dims": list(DIMS), "t_bc": TBC, "kappa": KAPPA, "csw": CSW,
                   "links": "synth.exp_links(dims, 0.4, 4401)", "psi": "synth.gaussian_source(dims, 4402)"},
        "sites": SITES,
        "M_psi": {str(s): cplx(Mpsi[s]) for s in SITES},
        "H_psi": {str(s): cplx(Hpsi[s]) for s in SITES},
        "schur_psi": {str(s): cplx(schur[s]) for s in SITES},
        "clover_block_site0": cplx(T[0]),
        "norm2_M_psi": float(np.vdot(Mpsi, Mpsi).real),
        "action_S": S,
        "force_link_site0_mu0": cplx(F[0, 0]),
    }


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression_4x4x4x4.json")
    with open(out, "w") as fh:
        json.dump(compute(), fh, indent=1)
    print("wrote", out)
