"""CPU oracle for the Wilson-Clover operator and its solvers (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never touches it, and it shares no code with that path.

``wc_oracle.c`` holds the lattice arithmetic (operator, adjoint, clover term,
RAS block solves, force) in plain FP64; this module loads it through ctypes
and adds the solver loops in numpy (``solvers.py``).  Arrays use the canonical
complex128 layouts documented in ``synth``: U[V,4,3,3], psi[V,4,3],
T[V,12,12].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile wc_oracle.c with gcc (portable C99 + OpenMP, no ISA flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)


def _declare(L):
    L.orc_volume.argtypes = [_ip]
    L.orc_volume.restype = ctypes.c_long
    L.orc_gamma.argtypes = [ctypes.c_int, _dp]
    L.orc_clover_field.argtypes = [_ip, ctypes.c_double, ctypes.c_double, _dp, _dp]
    L.orc_leaf_sum.argtypes = [_ip, _dp, ctypes.c_long, ctypes.c_int, ctypes.c_int, _dp]
    L.orc_apply_hop.argtypes = [_ip, ctypes.c_int, _dp, _dp, _dp, ctypes.c_long, _lp]
    L.orc_apply_M.argtypes = [_ip, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp,
                              _dp, _dp, _dp, ctypes.c_long, _lp]
    L.orc_apply_Mdag.argtypes = [_ip, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp]
    L.orc_ras.argtypes = [_ip, ctypes.c_int, ctypes.c_double, _dp, _dp, _ip, ctypes.c_int,
                          ctypes.c_int, _dp, _dp]
    L.orc_ras.restype = ctypes.c_int
    L.orc_force.argtypes = [_ip, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp,
                            _dp, _dp, ctypes.c_int]


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(d) for d in dims])


def _cptr(a: np.ndarray):
    assert a.dtype == np.complex128 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def volume(dims) -> int:
    return int(np.prod([int(d) for d in dims]))


def gamma(mu: int) -> np.ndarray:
    """gamma_mu for mu = 0..3 (x,y,z,t), gamma_5 for mu = 4 (chiral basis)."""
    out = np.zeros((4, 4), dtype=np.complex128)
    lib().orc_gamma(int(mu), _cptr(out))
    return out


def clover_field(dims, csw: float, kappa: float, U) -> np.ndarray:
    """T[V,12,12] = i csw kappa sum_{mu<nu} sigma_munu (x) Fhat_munu."""
    U = _c128(U)
    T = np.zeros((volume(dims), 12, 12), dtype=np.complex128)
    lib().orc_clover_field(_dims(dims), float(csw), float(kappa), _cptr(U), _cptr(T))
    return T


def leaf_sum(dims, U, site: int, mu: int, nu: int) -> np.ndarray:
    U = _c128(U)
    Q = np.zeros((3, 3), dtype=np.complex128)
    lib().orc_leaf_sum(_dims(dims), _cptr(U), int(site), int(mu), int(nu), _cptr(Q))
    return Q


def _sites_arg(sites):
    if sites is None:
        return -1, None, None
    s = np.ascontiguousarray(sites, dtype=np.int64)
    return len(s), s, s.ctypes.data_as(_lp)


def apply_hop(dims, tbc: int, U, psi, sites=None) -> np.ndarray:
    """H psi (all sites, or the listed sites in list order)."""
    U, psi = _c128(U), _c128(psi)
    n, keep, sp = _sites_arg(sites)
    out = np.zeros((volume(dims) if n < 0 else n, 4, 3), dtype=np.complex128)
    lib().orc_apply_hop(_dims(dims), int(tbc), _cptr(U), _cptr(psi), _cptr(out), n, sp)
    return out


def apply_M(dims, tbc: int, kappa: float, csw: float, U, psi, T=None, sites=None):
    """M psi = (1 + T) psi - kappa H psi.  T=None rebuilds the clover per site."""
    U, psi = _c128(U), _c128(psi)
    Tc = None if T is None else _c128(T)
    n, keep, sp = _sites_arg(sites)
    out = np.zeros((volume(dims) if n < 0 else n, 4, 3), dtype=np.complex128)
    lib().orc_apply_M(_dims(dims), int(tbc), float(kappa), float(csw), _cptr(U),
                      None if Tc is None else _cptr(Tc), _cptr(psi), _cptr(out), n, sp)
    return out


def apply_Mdag(dims, tbc: int, kappa: float, U, T, psi) -> np.ndarray:
    """M^+ psi, from explicitly conjugate-transposed blocks of M."""
    U, T, psi = _c128(U), _c128(T), _c128(psi)
    out = np.zeros((volume(dims), 4, 3), dtype=np.complex128)
    lib().orc_apply_Mdag(_dims(dims), int(tbc), float(kappa), _cptr(U), _cptr(T),
                         _cptr(psi), _cptr(out))
    return out


def ras(dims, tbc: int, kappa: float, U, T, block, delta: int, k: int, v) -> np.ndarray:
    """Overlapped RAS: MR_k block solves on extended blocks, core write-back."""
    U, T, v = _c128(U), _c128(T), _c128(v)
    z = np.zeros((volume(dims), 4, 3), dtype=np.complex128)
    b = (ctypes.c_int * 4)(*[int(x) for x in block])
    rc = lib().orc_ras(_dims(dims), int(tbc), float(kappa), _cptr(U), _cptr(T), b,
                       int(delta), int(k), _cptr(v), _cptr(z))
    if rc != 0:
        raise ValueError(f"RAS block {tuple(block)} / overlap {delta} does not fit {dims}")
    return z


def force(dims, tbc: int, kappa: float, csw: float, U, X, Y, hop_only: bool = False):
    """F = TA(G) per link for S = phi^+(M^+M)^-1 phi, given X and Y = M X."""
    U, X, Y = _c128(U), _c128(X), _c128(Y)
    F = np.zeros((volume(dims), 4, 3, 3), dtype=np.complex128)
    lib().orc_force(_dims(dims), int(tbc), float(kappa), float(csw), _cptr(U), _cptr(X),
                    _cptr(Y), _cptr(F), int(bool(hop_only)))
    return F


class Operator:
    """Convenience holder: one gauge field, its clover term, M and M^+."""

    def __init__(self, dims, U, csw: float, kappa: float, tbc: int):
        self.dims = tuple(int(d) for d in dims)
        self.U = _c128(U)
        self.csw, self.kappa, self.tbc = float(csw), float(kappa), int(tbc)
        self.T = clover_field(self.dims, self.csw, self.kappa, self.U)

    def M(self, psi):
        return apply_M(self.dims, self.tbc, self.kappa, self.csw, self.U, psi, T=self.T)

    def Mdag(self, psi):
        return apply_Mdag(self.dims, self.tbc, self.kappa, self.U, self.T, psi)

    def ras(self, v, block=(4, 4, 4, 4), delta=1, k=4):
        return ras(self.dims, self.tbc, self.kappa, self.U, self.T, block, delta, k, v)


from .solvers import bicgstab, action_and_force  # noqa: E402,F401
