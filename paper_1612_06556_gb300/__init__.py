"""GB300 Wilson-Clover operator and RAS-BiCGStab solvers (Python binding).

A thin ctypes layer over ``libwc.so`` (C ABI declared in ``include/wc.h``):
it only marshals arguments.  Every step of the operator, the reductions, the
preconditioner and the solvers runs in the library's CUDA kernels; PyTorch
(when used) only supplies device memory and the CUDA stream.  There is no
CPU fallback: importing this package fails if the library is not built
(``python paper_1612_06556_gb300/build.py`` or ``__graft_entry__.build()``).

Arrays crossing the boundary use the canonical complex128 layouts of
``include/wc.h``: gauge U[V,4,3,3], spinor psi[V,4,3], force F[V,4,3,3],
site = x + Lx*(y + Ly*(z + Lz*t)).  They may be CUDA torch tensors, CPU
torch tensors or numpy arrays (C-contiguous complex128).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# WC_LIBRARY selects another build of the library (the checked build,
# libwc_checked.so, in the tests); default: the in-tree libwc.so
LIB_PATH = os.environ.get("WC_LIBRARY") or os.path.join(_HERE, "libwc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python paper_1612_06556_gb300/build.py); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

F64, F32, F16 = 0, 1, 2
PRECOND_NONE, PRECOND_RAS = 0, 1
ARITH_F64, ARITH_DF32 = 0, 1
SOLVER_FLEXIBLE, SOLVER_RELIABLE, SOLVER_NESTED = 0, 1, 2
STATUS = {0: "WC_OK", 1: "WC_ERR_ARG", 2: "WC_ERR_CUDA", 3: "WC_ERR_STATE", 4: "WC_ERR_NOT_CONVERGED",
          5: "WC_ERR_BREAKDOWN", 6: "WC_ERR_NAN", 7: "WC_ERR_TIMEOUT"}

EXPORTED = [
    "wc_create_lattice", "wc_destroy_lattice", "wc_set_stream", "wc_load_gauge", "wc_load_clover",
    "wc_field_create", "wc_field_destroy", "wc_field_import", "wc_field_export", "wc_field_copy",
    "wc_apply_M", "wc_apply_Mdag", "wc_apply_hop", "wc_dot", "wc_norm2", "wc_axpy_norm",
    "wc_ras_precond", "wc_ras_schur", "wc_solve_bicgstab", "wc_solve_batch", "wc_action_force", "wc_last_error",
    "wc_dot_noalloc", "wc_ras_autotune", "wc_apply_shape", "wc_apply_schur", "wc_apply_multi",
    "wc_force_times_links", "wc_set_fp64_arith", "wc_field_import_f32", "wc_field_export_f32",
    "wc_field_import_async", "wc_field_export_async", "wc_sync",
    "wc_create_subdomain", "wc_halo_bytes", "wc_halo_pack", "wc_apply_interior", "wc_apply_surface",
    "wc_checked_violations", "wc_apply_schur_multi",
]


class RasParams(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int * 4), ("overlap", ctypes.c_int), ("mr_iters", ctypes.c_int),
                ("schur", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("precond", ctypes.c_int), ("inner_prec", ctypes.c_int), ("ras", RasParams),
                ("solver", ctypes.c_int), ("delta", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("inner_iters", ctypes.c_int), ("krylov_prec", ctypes.c_int), ("even_odd", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("true_rel_resid", ctypes.c_double),
                ("seconds", ctypes.c_double), ("status", ctypes.c_int)]

    def __repr__(self):
        return (f"SolveInfo(iters={self.iters}, restarts={self.restarts}, "
                f"true_rel_resid={self.true_rel_resid:.3e}, seconds={self.seconds:.4f}, "
                f"status={STATUS.get(self.status, self.status)})")


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_L = _lib
_L.wc_create_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int, _vp, ctypes.POINTER(_vp)]
_L.wc_destroy_lattice.argtypes = [_vp]
_L.wc_set_stream.argtypes = [_vp, _vp]
_L.wc_set_fp64_arith.argtypes = [_vp, ctypes.c_int]
_L.wc_load_gauge.argtypes = [_vp, _vp]
_L.wc_load_clover.argtypes = [_vp, ctypes.c_double, ctypes.c_double]
_L.wc_field_create.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(_vp)]
_L.wc_field_destroy.argtypes = [_vp]
_L.wc_field_import.argtypes = [_vp, _vp]
_L.wc_field_export.argtypes = [_vp, _vp]
_L.wc_field_import_f32.argtypes = [_vp, _vp]
_L.wc_field_export_f32.argtypes = [_vp, _vp]
_L.wc_field_import_async.argtypes = [_vp, _vp, ctypes.c_int]
_L.wc_field_export_async.argtypes = [_vp, _vp, ctypes.c_int]
_L.wc_sync.argtypes = [_vp]
_L.wc_field_copy.argtypes = [_vp, _vp, ctypes.c_double]
for _n in ("wc_apply_M", "wc_apply_Mdag", "wc_apply_hop"):
    getattr(_L, _n).argtypes = [_vp, _vp, _vp]
_L.wc_dot.argtypes = [_vp, _vp, _vp, _dp]
_L.wc_norm2.argtypes = [_vp, _vp, _dp]
_L.wc_axpy_norm.argtypes = [_vp, _dp, _vp, _vp, _dp]
_L.wc_ras_precond.argtypes = [_vp, _vp, _vp, ctypes.POINTER(RasParams)]
_L.wc_ras_schur.argtypes = [_vp, _vp, _vp, ctypes.POINTER(RasParams), ctypes.c_int]
_L.wc_solve_bicgstab.argtypes = [_vp, _vp, _vp, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo)]
_L.wc_solve_batch.argtypes = [ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                              ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo)]
_L.wc_action_force.argtypes = [_vp, _vp, _dp, _vp, ctypes.POINTER(SolveParams)]
_L.wc_apply_schur.argtypes = [_vp, _vp, _vp, ctypes.c_int]
_L.wc_apply_multi.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int]
_L.wc_force_times_links.argtypes = [_vp, _vp, _vp, ctypes.c_double, _vp]
_L.wc_apply_shape.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
_L.wc_ras_autotune.argtypes = [_vp, _vp, ctypes.POINTER(SolveParams), ctypes.POINTER(RasParams)]
_L.wc_dot_noalloc.argtypes = [_vp, _vp, ctypes.c_longlong, _vp, _vp]
_L.wc_create_subdomain.argtypes = [ctypes.POINTER(ctypes.c_int)] * 3 + [ctypes.c_int, _vp, ctypes.POINTER(_vp)]
_L.wc_halo_bytes.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]
_L.wc_halo_pack.argtypes = [_vp, _vp, ctypes.c_int, ctypes.POINTER(_vp)]
_L.wc_apply_interior.argtypes = [_vp, _vp, _vp, ctypes.c_int]
_L.wc_apply_surface.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(_vp)]
_L.wc_checked_violations.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
_L.wc_apply_schur_multi.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int]
_L.wc_last_error.argtypes = [_vp]
_L.wc_last_error.restype = ctypes.c_char_p
for _n in EXPORTED:
    if _n != "wc_last_error":
        getattr(_L, _n).restype = ctypes.c_int


class WCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(status, handle=None):
    if status != 0:
        msg = _L.wc_last_error(handle)
        raise WCError(status, msg.decode() if msg else "")


def _ptr(a):
    """Data pointer of a C-contiguous complex128 torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.complex128 or not a.is_contiguous():
            raise ValueError("expected a contiguous complex128 tensor")
        return a.data_ptr()
    import numpy as np
    if a.dtype != np.complex128 or not a.flags.c_contiguous:
        raise ValueError("expected a C-contiguous complex128 array")
    return a.ctypes.data


def _nbytes(a):
    return a.numel() * 16 if hasattr(a, "numel") else a.size * 16


def _is_c64(a) -> bool:
    """True for a complex64 torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        import torch
        return a.dtype == torch.complex64
    import numpy as np
    return getattr(a, "dtype", None) == np.complex64


def _ptr64(a):
    """Data pointer of a C-contiguous complex64 torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("expected a contiguous complex64 tensor")
        return a.data_ptr()
    if not a.flags.c_contiguous:
        raise ValueError("expected a C-contiguous complex64 array")
    return a.ctypes.data


def ras_params(block=(4, 4, 4, 4), overlap=1, mr_iters=4, schur=False) -> RasParams:
    return RasParams((ctypes.c_int * 4)(*block), int(overlap), int(mr_iters), int(bool(schur)))


def solve_params(tol=1e-10, max_iter=10000, max_restarts=5, precond=PRECOND_NONE, inner_prec=F32,
                 block=(4, 4, 4, 4), overlap=1, mr_iters=4, solver=SOLVER_FLEXIBLE, delta=0.01, inner_tol=0.01,
                 inner_iters=100, krylov_prec=F32, even_odd=False, ras_schur=False) -> SolveParams:
    return SolveParams(float(tol), int(max_iter), int(max_restarts), int(precond), int(inner_prec),
                       ras_params(block, overlap, mr_iters, ras_schur), int(solver), float(delta), float(inner_tol),
                       int(inner_iters), int(krylov_prec), int(bool(even_odd)))


class Field:
    """A colour-spinor field owned by the library (FP64, FP32 or FP16+scale)."""

    def __init__(self, lattice: "Lattice", prec: int = F64):
        self.lattice = lattice
        self.prec = prec
        h = _vp()
        _check(_L.wc_field_create(lattice.handle, int(prec), ctypes.byref(h)), lattice.handle)
        self.handle = h

    def _size_ok(self, a):
        n = a.numel() if hasattr(a, "numel") else a.size
        if n != self.lattice.volume * 12:
            raise ValueError(f"spinor buffer must hold {self.lattice.volume}*12 complex values")

    def load(self, psi):
        """Import canonical psi[V,4,3], complex128 or complex64 (device or host)."""
        self._size_ok(psi)
        if _is_c64(psi):
            _check(_L.wc_field_import_f32(self.handle, _vp(_ptr64(psi))), self.lattice.handle)
        else:
            _check(_L.wc_field_import(self.handle, _vp(_ptr(psi))), self.lattice.handle)
        return self

    def store(self, out):
        """Export into canonical out[V,4,3], complex128 or complex64 (device or host)."""
        self._size_ok(out)
        if _is_c64(out):
            _check(_L.wc_field_export_f32(self.handle, _vp(_ptr64(out))), self.lattice.handle)
        else:
            _check(_L.wc_field_export(self.handle, _vp(_ptr(out))), self.lattice.handle)
        return out

    def load_async(self, psi):
        """Queue the import of psi[V,4,3] (complex128 or complex64; CUDA or
        page-locked host memory) without waiting; keep psi unchanged until
        Lattice.sync() (see wc_field_import_async)."""
        self._size_ok(psi)
        c64 = _is_c64(psi)
        ptr = _ptr64(psi) if c64 else _ptr(psi)
        _check(_L.wc_field_import_async(self.handle, _vp(ptr), int(c64)), self.lattice.handle)
        return self

    def store_async(self, out):
        """Queue the export into out[V,4,3] (complex128 or complex64; CUDA or
        page-locked host memory); out is valid after Lattice.sync()."""
        self._size_ok(out)
        c64 = _is_c64(out)
        ptr = _ptr64(out) if c64 else _ptr(out)
        _check(_L.wc_field_export_async(self.handle, _vp(ptr), int(c64)), self.lattice.handle)
        return out

    def copy_from(self, src: "Field", scale: float = 1.0):
        _check(_L.wc_field_copy(self.handle, src.handle, float(scale)), self.lattice.handle)
        return self

    def close(self):
        if getattr(self, "handle", None):
            _L.wc_field_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lattice:
    """A 4-D lattice with its gauge field and clover term on the GPU."""

    def __init__(self, dims, t_bc: int = -1, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.volume = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        s = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        h = _vp()
        _check(_L.wc_create_lattice((ctypes.c_int * 4)(*self.dims), int(t_bc), _vp(s), ctypes.byref(h)))
        self.handle = h
        self.t_bc = t_bc

    def set_stream(self, stream):
        s = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        _check(_L.wc_set_stream(self.handle, _vp(s)), self.handle)

    def sync(self):
        """Wait for everything queued on this lattice (see wc_sync)."""
        _check(_L.wc_sync(self.handle), self.handle)
        return self

    def set_fp64_arith(self, arith: int):
        """ARITH_F64 (default) or ARITH_DF32: arithmetic of the FP64 operator
        applications on this lattice (see wc_set_fp64_arith)."""
        _check(_L.wc_set_fp64_arith(self.handle, int(arith)), self.handle)
        return self

    def load_gauge(self, U):
        if _nbytes(U) != self.volume * 36 * 16:
            raise ValueError("gauge buffer must hold V*4*3*3 complex128")
        _check(_L.wc_load_gauge(self.handle, _vp(_ptr(U))), self.handle)
        return self

    def load_clover(self, csw: float, kappa: float):
        _check(_L.wc_load_clover(self.handle, float(csw), float(kappa)), self.handle)
        self.csw, self.kappa = float(csw), float(kappa)
        return self

    def field(self, prec: int = F64) -> Field:
        return Field(self, prec)

    def apply_M(self, out: Field, inp: Field):
        _check(_L.wc_apply_M(self.handle, out.handle, inp.handle), self.handle)

    def apply_Mdag(self, out: Field, inp: Field):
        _check(_L.wc_apply_Mdag(self.handle, out.handle, inp.handle), self.handle)

    def apply_hop(self, out: Field, inp: Field):
        _check(_L.wc_apply_hop(self.handle, out.handle, inp.handle), self.handle)

    def apply_multi(self, outs, inps, dagger: bool = False):
        """outs[r] = M inps[r] (or M^+) for up to 16 FP32 fields in one launch
        (see wc_apply_multi)."""
        n = len(outs)
        if len(inps) != n:
            raise ValueError("outs and inps must have the same length")
        O = (_vp * n)(*[f.handle for f in outs])
        I = (_vp * n)(*[f.handle for f in inps])
        _check(_L.wc_apply_multi(self.handle, n, O, I, int(bool(dagger))), self.handle)

    def apply_schur(self, out: Field, inp: Field, dagger: bool = False):
        """out (even sites) = M^ in (even sites), M^ = A_ee - k^2 H_eo A_oo^-1 H_oe;
        odd sites of out set to zero (see wc_apply_schur)."""
        _check(_L.wc_apply_schur(self.handle, out.handle, inp.handle, int(bool(dagger))), self.handle)

    def apply_schur_multi(self, outs, inps, dagger: bool = False):
        """outs[r] (even sites) = M^ inps[r] for up to 16 FP32 or FP16 fields,
        odd sites zero (see wc_apply_schur_multi)."""
        n = len(outs)
        if len(inps) != n:
            raise ValueError("outs and inps must have the same length")
        O = (_vp * n)(*[f.handle for f in outs])
        I = (_vp * n)(*[f.handle for f in inps])
        _check(_L.wc_apply_schur_multi(self.handle, n, O, I, int(bool(dagger))), self.handle)

    def apply_shape(self, prec: int, kind: int = 0, force: int = -1):
        """(threads, tile, capped) of the operator launch for prec / kind
        (0 M, 1 M^+, 2 H); force >= 0 pins candidate #force."""
        out = (ctypes.c_int * 6)()
        _check(_L.wc_apply_shape(self.handle, int(prec), int(kind), int(force), out), self.handle)
        return out[0], tuple(out[1:5]), out[5]

    def dot(self, a: Field, b: Field) -> complex:
        r = (ctypes.c_double * 2)()
        _check(_L.wc_dot(self.handle, a.handle, b.handle, r), self.handle)
        return complex(r[0], r[1])

    def norm2(self, a: Field) -> float:
        r = ctypes.c_double()
        _check(_L.wc_norm2(self.handle, a.handle, ctypes.byref(r)), self.handle)
        return r.value

    def axpy_norm(self, a: complex, x: Field, y: Field) -> float:
        c = (ctypes.c_double * 2)(a.real, a.imag)
        r = ctypes.c_double()
        _check(_L.wc_axpy_norm(self.handle, c, x.handle, y.handle, ctypes.byref(r)), self.handle)
        return r.value

    def ras(self, out: Field, inp: Field, block=(4, 4, 4, 4), overlap=1, mr_iters=4):
        p = ras_params(block, overlap, mr_iters)
        _check(_L.wc_ras_precond(self.handle, out.handle, inp.handle, ctypes.byref(p)), self.handle)

    def ras_schur(self, out: Field, inp: Field, block=(4, 4, 4, 4), overlap=1, mr_iters=4, dagger=False):
        """RAS on block Schur complements of the even sites of inp (odd sites
        of out zero)."""
        p = ras_params(block, overlap, mr_iters, True)
        _check(_L.wc_ras_schur(self.handle, out.handle, inp.handle, ctypes.byref(p), int(bool(dagger))),
               self.handle)

    def solve(self, x: Field, b: Field, params: SolveParams | None = None, check=True, **kw) -> SolveInfo:
        p = params if params is not None else solve_params(**kw)
        info = SolveInfo()
        st = _L.wc_solve_bicgstab(self.handle, x.handle, b.handle, ctypes.byref(p), ctypes.byref(info))
        if check:
            _check(st, self.handle)
        return info

    def ras_autotune(self, b: Field, params: SolveParams | None = None, **kw):
        """Block shape, overlap and MR steps the batched solver's autotuner
        picks for this lattice (see wc_ras_autotune)."""
        p = params if params is not None else solve_params(**kw)
        out = RasParams()
        _check(_L.wc_ras_autotune(self.handle, b.handle, ctypes.byref(p), ctypes.byref(out)), self.handle)
        return tuple(out.block), out.overlap, out.mr_iters

    def action_force(self, phi: Field, force_out, params: SolveParams | None = None, **kw) -> float:
        p = params if params is not None else solve_params(**kw)
        if _nbytes(force_out) != self.volume * 36 * 16:
            raise ValueError("force buffer must hold V*4*3*3 complex128")
        S = ctypes.c_double()
        _check(_L.wc_action_force(self.handle, phi.handle, ctypes.byref(S), _vp(_ptr(force_out)),
                                  ctypes.byref(p)), self.handle)
        return S.value

    def force_times_links(self, F, U, scale: float, out):
        """out = scale * F U per link (contiguous CUDA complex128 tensors
        [V,4,3,3]); see wc_force_times_links."""
        for t in (F, U, out):
            if not (t.is_cuda and t.numel() == self.volume * 36):
                raise ValueError("F, U and out must be CUDA tensors of V*4*3*3 complex128")
        _check(_L.wc_force_times_links(self.handle, _vp(_ptr(F)), _vp(_ptr(U)), float(scale), _vp(_ptr(out))),
               self.handle)
        return out

    def last_error(self) -> str:
        return _L.wc_last_error(self.handle).decode()

    def close(self):
        if getattr(self, "handle", None):
            _L.wc_destroy_lattice(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dot_noalloc(a, b, out, stream=None):
    """out[0] + i out[1] = <a, b> for CUDA complex128 tensors a, b (same
    number of elements) into the CUDA float64 tensor out (2 elements), with
    no device allocation (see wc_dot_noalloc in wc.h).  Asynchronous on
    stream (default: the legacy default stream)."""
    import torch
    if not (a.is_cuda and b.is_cuda and out.is_cuda):
        raise ValueError("a, b and out must be CUDA tensors")
    if a.dtype != torch.complex128 or b.dtype != torch.complex128 or out.dtype != torch.float64:
        raise ValueError("a and b must be complex128, out float64")
    if a.numel() != b.numel() or out.numel() < 2:
        raise ValueError("a and b must have the same size; out needs 2 elements")
    if not (a.is_contiguous() and b.is_contiguous() and out.is_contiguous()):
        raise ValueError("tensors must be contiguous")
    s = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(_L.wc_dot_noalloc(_vp(a.data_ptr()), _vp(b.data_ptr()), a.numel(), _vp(out.data_ptr()), _vp(s)))
    return out


def solve_batch(lattices, xs, bs, params: SolveParams | None = None, check=True, **kw):
    """Solve M_i x_i = b_i for all i in one batched call; returns SolveInfos."""
    n = len(xs)
    p = params if params is not None else solve_params(**kw)
    L = (_vp * n)(*[lat.handle for lat in lattices])
    X = (_vp * n)(*[x.handle for x in xs])
    B = (_vp * n)(*[b.handle for b in bs])
    infos = (SolveInfo * n)()
    st = _L.wc_solve_batch(n, L, X, B, ctypes.byref(p), infos)
    if st != 0 and check:
        _check(st, None)
    return list(infos)


def _torch_autograd_function():
    import torch

    class PseudofermionAction(torch.autograd.Function):
        """S = phi^+ (M^+ M)^-1 phi as a differentiable function of the gauge
        field U (CUDA complex128 tensor [V,4,3,3], special unitary links).

        forward: loads U into the lattice, builds the clover term, and calls
        wc_action_force (two FP64 solves M^+ Y = phi, M X = Y; S = |Y|^2; F
        the traceless anti-Hermitian force per link).  backward: returns
        grad_U = grad_S * F^+ U = -grad_S * F U, the gradient on the tangent
        space of SU(3): for U -> exp(eps L) U with L in su(3),
        dS/deps = Re sum tr(grad_U^+ L U) = sum tr(L F).  phi is not
        differentiated (its gradient is None)."""

        @staticmethod
        def forward(ctx, U, phi, lattice, csw, kappa, params):
            if not (U.is_cuda and U.dtype == torch.complex128 and U.is_contiguous()):
                raise ValueError("U must be a contiguous CUDA complex128 tensor")
            lattice.load_gauge(U).load_clover(csw, kappa)
            f_phi = lattice.field(F64).load(phi.contiguous())
            F = torch.empty_like(U)
            S = lattice.action_force(f_phi, F, params)
            ctx.save_for_backward(U, F)
            ctx.lattice = lattice
            return torch.tensor(S, dtype=torch.float64, device=U.device)

        @staticmethod
        def backward(ctx, grad_S):
            U, F = ctx.saved_tensors
            grad_U = torch.empty_like(U)
            # grad_U = -grad_S * F U, per link, in the library's kernel
            ctx.lattice.force_times_links(F, U, -float(grad_S), grad_U)
            return grad_U, None, None, None, None, None

    return PseudofermionAction


def pseudofermion_action(U, phi, lattice: Lattice, csw: float, kappa: float, params: SolveParams | None = None,
                         **kw):
    """Differentiable S = phi^+ (M^+ M)^-1 phi (see PseudofermionAction)."""
    p = params if params is not None else solve_params(**kw)
    return _torch_autograd_function().apply(U, phi, lattice, float(csw), float(kappa), p)


def _buf_ptrs(bufs):
    """Eight device buffer pointers (CUDA tensors or None) as a C array."""
    if len(bufs) != 8:
        raise ValueError("need 8 buffers: [2 mu] lower side, [2 mu + 1] upper side, None for uncut mu")
    ptrs = []
    for b in bufs:
        if b is None:
            ptrs.append(None)
        else:
            if not (b.is_cuda and b.is_contiguous()):
                raise ValueError("halo buffers must be contiguous CUDA tensors")
            ptrs.append(b.data_ptr())
    return (_vp * 8)(*ptrs)


class SubDomain(Lattice):
    """One sub-domain of a decomposed lattice: the sites [offset, offset +
    local_dims) of a lattice of extents global_dims, with the overlapped
    operator steps halo_pack / apply_interior / apply_surface (see
    wc_create_subdomain in wc.h)."""

    def __init__(self, local_dims, global_dims, offset, t_bc: int = -1, stream=None):
        self.dims = tuple(int(d) for d in local_dims)
        self.global_dims = tuple(int(d) for d in global_dims)
        self.offset = tuple(int(o) for o in offset)
        self.volume = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        self.split = tuple(l < g for l, g in zip(self.dims, self.global_dims))
        self.ext_dims = tuple(l + 2 * int(c) for l, c in zip(self.dims, self.split))
        s = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        h = _vp()
        c4 = ctypes.c_int * 4
        _check(_L.wc_create_subdomain(c4(*self.dims), c4(*self.global_dims), c4(*self.offset), int(t_bc), _vp(s),
                                      ctypes.byref(h)))
        self.handle = h
        self.t_bc = t_bc

    def load_gauge(self, U_ext):
        """U_ext: the gauge field of the sub-domain extended by one site across
        every cut face (extents ext_dims, canonical layout)."""
        n = self.ext_dims[0] * self.ext_dims[1] * self.ext_dims[2] * self.ext_dims[3]
        if _nbytes(U_ext) != n * 36 * 16:
            raise ValueError(f"extended gauge buffer must hold {n}*4*3*3 complex128")
        _check(_L.wc_load_gauge(self.handle, _vp(_ptr(U_ext))), self.handle)
        return self

    def halo_bytes(self, mu: int) -> int:
        r = ctypes.c_longlong()
        _check(_L.wc_halo_bytes(self.handle, int(mu), ctypes.byref(r)), self.handle)
        return r.value

    def halo_pack(self, inp: Field, send, dagger: bool = False):
        _check(_L.wc_halo_pack(self.handle, inp.handle, int(bool(dagger)), _buf_ptrs(send)), self.handle)

    def apply_interior(self, out: Field, inp: Field, dagger: bool = False):
        _check(_L.wc_apply_interior(self.handle, out.handle, inp.handle, int(bool(dagger))), self.handle)

    def apply_surface(self, out: Field, inp: Field, recv, dagger: bool = False):
        _check(_L.wc_apply_surface(self.handle, out.handle, inp.handle, int(bool(dagger)), _buf_ptrs(recv)),
               self.handle)


def checked_violations() -> int:
    """Out-of-range indices counted by the checked build since it was loaded
    (see wc_checked_violations); raises WCError in the normal build."""
    n = ctypes.c_ulonglong()
    _check(_L.wc_checked_violations(ctypes.byref(n)))
    return n.value
