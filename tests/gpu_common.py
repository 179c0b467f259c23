"""Shared helpers of the GPU parity tests (inputs from synth, references from
the oracle, results through the C ABI binding)."""
import numpy as np
import pytest


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def wc():
    import paper_1612_06556_gb300 as w
    return w


def make_lattice(dims, U, csw, kappa, tbc):
    w = wc()
    return w.Lattice(dims, tbc).load_gauge(U).load_clover(csw, kappa)


def gpu_apply(lat, psi, prec, kind="M"):
    f_in = lat.field(prec).load(psi)
    f_out = lat.field(prec)
    getattr(lat, "apply_" + kind)(f_out, f_in)
    return f_out.store(np.zeros_like(psi))


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def assert_elementwise(out, ref, rel_tol):
    """Every component within rel_tol of the field's largest magnitude, and
    the relative L2 error within rel_tol."""
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(out - ref)) <= rel_tol * scale, np.max(np.abs(out - ref)) / scale
    assert rel_err(out, ref) <= rel_tol, rel_err(out, ref)
