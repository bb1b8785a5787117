"""Python binding of ``libfpe.so`` (include/fpe.h): fast evaluation of real and
complex polynomials (arXiv 2211.06320, Algorithm A_p) on a GB300 GPU.

Argument marshalling only: every step of preconditioning and evaluation runs
in the C/CUDA library.  Device buffers are torch CUDA tensors (float64 for
points; results as an (n, 3) float64 tensor whose rows are the C struct
fpe_xc64 = {re, im, e}, e stored as int64 bits -- see ``split_xc64``).
There is no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import _build

FPE_OK = 0
FPE_ERR_INVALID_ARG = 1
FPE_ERR_NONFINITE = 2
FPE_ERR_ZERO_POLY = 3
FPE_ERR_OOM = 4
FPE_ERR_CUDA = 5
FPE_ERR_TIMEOUT = 6
FPE_ERR_UNSUPPORTED = 7

FPE_REAL = 1
FPE_WITH_DERIV = 2
FPE_FP32 = 4
FPE_HOST_ONLY = 8
FPE_ACCURATE = 16
FPE_FORCE_DENSE = 32
FPE_FORCE_SPARSE = 64

# every symbol include/fpe.h declares
EXPORTED = [
    "fpe_precondition", "fpe_eval", "fpe_eval_host", "fpe_eval_deriv", "fpe_eval_batch", "fpe_horner",
    "fpe_info", "fpe_get_hull", "fpe_get_good", "fpe_get_windows", "fpe_sync", "fpe_destroy",
    "fpe_status_string", "fpe_last_error", "fpe_profile_enable", "fpe_profile_reset", "fpe_profile_read",
    "fpe_measure_fma_peak", "fpe_eval_noalloc", "fpe_batch_create", "fpe_batch_eval", "fpe_batch_sync",
    "fpe_batch_destroy", "fpe_newton", "fpe_grad_points", "fpe_grad_coeffs", "fpe_to_complex", "fpe_analyse",
    "fpe_set_tuning", "fpe_get_tuning", "fpe_autotune", "fpe_batch_set_tuning", "fpe_batch_autotune",
    "fpe_set_tensor_path", "fpe_get_tensor_path", "fpe_tensor_stats", "fpe_cert_stats", "fpe_measure_mma_peak",
]


class FpeError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


class XC64(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double), ("e", ctypes.c_int64)]


class Tuning(ctypes.Structure):
    """fpe_tuning: launch parameters of the window sums."""
    _fields_ = [("long_window", ctypes.c_int64), ("lane_chunk", ctypes.c_int64), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {"long_window": int(self.long_window), "lane_chunk": int(self.lane_chunk), "ms": float(self.ms)}


_lib = None


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()  # no-op when the in-tree library is up to date
    lib = ctypes.CDLL(path)
    P, I64, I32, U32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_double
    sig = {
        "fpe_precondition": ([P, P, P, I64, I32, U32, ctypes.POINTER(P)], I32),
        "fpe_eval": ([P, P, P, I64, P, P, P, P], I32),
        "fpe_eval_host": ([P, P, P, I64, P, P, P], I32),
        "fpe_eval_deriv": ([P, P, P, I64, P, P], I32),
        "fpe_eval_batch": ([P, I64, P, P, P, P, P], I32),
        "fpe_horner": ([P, P, P, I64, P, I32, P], I32),
        "fpe_info": ([P, P, P, P, P, P], I32),
        "fpe_get_hull": ([P, P, P, I64], I32),
        "fpe_get_good": ([P, P, I64], I32),
        "fpe_get_windows": ([P, I64, P, P, P, P], I32),
        "fpe_sync": ([P, P], I32),
        "fpe_destroy": ([P], None),
        "fpe_status_string": ([I32], ctypes.c_char_p),
        "fpe_last_error": ([], ctypes.c_char_p),
        "fpe_profile_enable": ([I32], None),
        "fpe_profile_reset": ([], None),
        "fpe_profile_read": ([ctypes.c_char_p, ctypes.POINTER(D), ctypes.POINTER(I64)], I32),
        "fpe_measure_fma_peak": ([I32, I32, ctypes.POINTER(D)], I32),
        "fpe_eval_noalloc": ([P, P, P, I64, P, P, P, P], I32),
        "fpe_batch_create": ([P, I64, P, ctypes.POINTER(P)], I32),
        "fpe_batch_eval": ([P, P, P, P, P, P], I32),
        "fpe_batch_sync": ([P, P], I32),
        "fpe_batch_destroy": ([P], None),
        "fpe_newton": ([P, P, P, I64, P, P, P, P], I32),
        "fpe_grad_points": ([P, P, P, I64, P, P, P, P, P], I32),
        "fpe_grad_coeffs": ([P, P, P, I64, P, P, P, P, P], I32),
        "fpe_to_complex": ([P, I64, P, P, P], I32),
        "fpe_analyse": ([P, P, P, I64], I32),
        "fpe_set_tuning": ([P, ctypes.POINTER(Tuning)], I32),
        "fpe_get_tuning": ([P, ctypes.POINTER(Tuning)], I32),
        "fpe_autotune": ([P, P, P, I64, P, ctypes.POINTER(Tuning)], I32),
        "fpe_batch_set_tuning": ([P, ctypes.POINTER(Tuning)], I32),
        "fpe_batch_autotune": ([P, P, P, P, ctypes.POINTER(Tuning)], I32),
        "fpe_set_tensor_path": ([P, I64], I32),
        "fpe_get_tensor_path": ([P, ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_int32)], I32),
        "fpe_tensor_stats": ([P, ctypes.POINTER(I64), I32, P], I32),
        "fpe_cert_stats": ([P, ctypes.POINTER(I64), I32, P], I32),
        "fpe_measure_mma_peak": ([I32, ctypes.POINTER(D)], I32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != FPE_OK:
        lib = _load()
        raise FpeError(st, where, lib.fpe_last_error().decode(errors="replace") or
                       lib.fpe_status_string(st).decode())


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dptr(t):
    """Device pointer of a CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _points(z_re, z_im) -> int:
    """Check the device points before any pointer reaches a kernel: float64,
    one-dimensional, z_im (if given) of the same length and on the same device.
    Returns n.  The kernels read n entries of each array, so a shorter or
    narrower array would be read out of bounds."""
    import torch
    if not isinstance(z_re, torch.Tensor) or z_re.dtype != torch.float64 or z_re.dim() != 1:
        raise ValueError("z_re must be a one-dimensional float64 CUDA tensor")
    if z_im is not None:
        if not isinstance(z_im, torch.Tensor) or z_im.dtype != torch.float64 or z_im.dim() != 1:
            raise ValueError("z_im must be None or a one-dimensional float64 CUDA tensor")
        if z_im.shape[0] != z_re.shape[0] or z_im.device != z_re.device:
            raise ValueError("z_im must have z_re's length and device")
    return int(z_re.shape[0])


def _check_out(out, n: int, device):
    """An (n, 3) float64 fpe_xc64 array on the points' device (the kernels write n rows)."""
    import torch
    if (not isinstance(out, torch.Tensor) or out.dtype != torch.float64 or tuple(out.shape) != (n, 3)
            or out.device != device):
        raise ValueError(f"out must be an ({n}, 3) float64 tensor on {device}")


def _check_vec(t, n: int, device, dtype, name: str):
    """A per-point (or per-coefficient) array of n entries of dtype on device, or None."""
    if t is None:
        return
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or t.numel() != n or t.device != device:
        raise ValueError(f"{name} must be a {dtype} tensor of {n} entries on {device}")


def _check_poly_device(P, device):
    """The handle's arrays live on the device it was preconditioned on."""
    if device.type != "cuda":
        raise ValueError("expected CUDA tensors")
    if P.device is not None and device.index is not None and device.index != P.device:
        raise ValueError(f"tensors are on {device}, the polynomial on cuda:{P.device}")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Poly:
    """A preconditioned polynomial (owns an fpe_poly_t handle)."""

    def __init__(self, handle: int, n_coef: int, device=None):
        self._h = ctypes.c_void_p(handle)
        self.n_coef = n_coef
        self.device = device  # CUDA ordinal the handle's device arrays live on

    @property
    def handle(self):
        return self._h

    def __del__(self):
        try:
            if self._h and self._h.value:
                _load().fpe_destroy(self._h)
                self._h = ctypes.c_void_p(None)
        except Exception:
            pass


def fpe_precondition(re, im=None, e2=None, p: int = 53, flags: int = 0) -> Poly:
    """Preconditioning (preconditioning part of Alg. A_p, §5.1) of a_k = (re[k] + i im[k]) 2^e2[k]; host arrays."""
    lib = _load()
    re = np.ascontiguousarray(re, dtype=np.float64)
    im = None if im is None else np.ascontiguousarray(im, dtype=np.float64)
    e2 = None if e2 is None else np.ascontiguousarray(e2, dtype=np.int64)
    h = ctypes.c_void_p()
    _check(lib.fpe_precondition(_np_ptr(re), _np_ptr(im), _np_ptr(e2), re.shape[0], int(p), int(flags),
                                ctypes.byref(h)), "fpe_precondition")
    dev = None
    if not (int(flags) & FPE_HOST_ONLY):
        try:
            import torch
            dev = torch.cuda.current_device()
        except Exception:  # the handle was built, so a device was current; torch just cannot say which
            dev = None
    return Poly(h.value, re.shape[0], dev)


def empty_out(n: int, device=None):
    import torch
    return torch.empty((n, 3), dtype=torch.float64, device=device or "cuda")


def split_xc64(out):
    """(re, im, e) of an (n, 3) fpe_xc64 array (torch tensor or numpy); e as int64."""
    if isinstance(out, np.ndarray):
        return out[:, 0].copy(), out[:, 1].copy(), np.ascontiguousarray(out[:, 2]).view(np.int64)
    import torch
    return out[:, 0], out[:, 1], out[:, 2].contiguous().view(torch.int64)


def _eval_args(P, z_re, z_im, out=None, nterms=None, bits_lost=None) -> int:
    import torch
    n = _points(z_re, z_im)
    _check_poly_device(P, z_re.device)
    if out is not None:
        _check_out(out, n, z_re.device)
    _check_vec(nterms, n, z_re.device, torch.int32, "nterms")
    _check_vec(bits_lost, n, z_re.device, torch.int32, "bits_lost")
    return n


def fpe_eval(P: Poly, z_re, z_im=None, out=None, nterms=None, bits_lost=None, stream=None):
    """Evaluation (evaluation part of Alg. A_p, §5.2) at device points; returns the (n, 3) result tensor."""
    lib = _load()
    n = _eval_args(P, z_re, z_im, out, nterms, bits_lost)
    if out is None:
        out = empty_out(n, z_re.device)
    _check(lib.fpe_eval(P.handle, _dptr(z_re), _dptr(z_im), n, _dptr(out), _dptr(nterms), _dptr(bits_lost),
                        _stream(stream)), "fpe_eval")
    return out


def fpe_eval_host(P: Poly, z_re: np.ndarray, z_im: Optional[np.ndarray] = None, want_diag: bool = False):
    """fpe_eval on host buffers (copies in, evaluates, copies out, waits)."""
    lib = _load()
    z_re = np.ascontiguousarray(z_re, dtype=np.float64)
    z_im = None if z_im is None else np.ascontiguousarray(z_im, dtype=np.float64)
    n = z_re.shape[0]
    out = np.zeros((n, 3), dtype=np.float64)
    nt = np.zeros(n, dtype=np.int32) if want_diag else None
    bl = np.zeros(n, dtype=np.int32) if want_diag else None
    _check(lib.fpe_eval_host(P.handle, _np_ptr(z_re), _np_ptr(z_im), n, _np_ptr(out), _np_ptr(nt), _np_ptr(bl)),
           "fpe_eval_host")
    return (out, nt, bl) if want_diag else out


def host_eval_raw(P: Poly, z_re_ptr: int, z_im_ptr: Optional[int], n: int, out_ptr: int) -> int:
    """fpe_eval_host on raw host addresses (e.g. pinned torch tensors); returns the status."""
    lib = _load()
    return lib.fpe_eval_host(P.handle, ctypes.c_void_p(z_re_ptr), ctypes.c_void_p(z_im_ptr) if z_im_ptr else None,
                             n, ctypes.c_void_p(out_ptr), None, None)


def fpe_eval_deriv(P: Poly, z_re, z_im=None, out=None, stream=None):
    lib = _load()
    n = _eval_args(P, z_re, z_im, out)
    if out is None:
        out = empty_out(n, z_re.device)
    _check(lib.fpe_eval_deriv(P.handle, _dptr(z_re), _dptr(z_im), n, _dptr(out), _stream(stream)), "fpe_eval_deriv")
    return out


def fpe_eval_batch(polys: Sequence[Poly], pt_offsets, z_re, z_im=None, out=None, stream=None):
    lib = _load()
    npoly = len(polys)
    hs = (ctypes.c_void_p * npoly)(*[p.handle.value for p in polys])
    offs = np.ascontiguousarray(pt_offsets, dtype=np.int64)
    n = int(offs[-1]) if npoly else 0
    if _points(z_re, z_im) != n:
        raise ValueError(f"the points must number pt_offsets[-1] = {n}")
    if out is not None:
        _check_out(out, n, z_re.device)
    if out is None:
        out = empty_out(n, z_re.device)
    _check(lib.fpe_eval_batch(hs, npoly, _np_ptr(offs), _dptr(z_re), _dptr(z_im), _dptr(out), _stream(stream)),
           "fpe_eval_batch")
    return out


def fpe_horner(P: Poly, z_re, z_im=None, compensated: bool = False, out=None, stream=None):
    """GPU Horner over all d+1 terms (plain or compensated)."""
    lib = _load()
    n = _eval_args(P, z_re, z_im, out)
    if out is None:
        out = empty_out(n, z_re.device)
    _check(lib.fpe_horner(P.handle, _dptr(z_re), _dptr(z_im), n, _dptr(out), int(bool(compensated)),
                          _stream(stream)), "fpe_horner")
    return out


def fpe_info(P: Poly) -> dict:
    lib = _load()
    d, v, nh, ng = (ctypes.c_int64() for _ in range(4))
    T = ctypes.c_int()
    _check(lib.fpe_info(P.handle, ctypes.byref(d), ctypes.byref(v), ctypes.byref(nh), ctypes.byref(ng),
                        ctypes.byref(T)), "fpe_info")
    return {"d": d.value, "valuation": v.value, "n_hull": nh.value, "n_good": ng.value, "T": T.value}


def fpe_get_hull(P: Poly):
    lib = _load()
    nh = fpe_info(P)["n_hull"]
    k = np.zeros(nh, dtype=np.int64)
    s = np.zeros(nh, dtype=np.int64)
    _check(lib.fpe_get_hull(P.handle, _np_ptr(k), _np_ptr(s), nh), "fpe_get_hull")
    return k, s


def fpe_get_good(P: Poly):
    lib = _load()
    m = np.zeros(P.n_coef, dtype=np.uint8)
    _check(lib.fpe_get_good(P.handle, _np_ptr(m), P.n_coef), "fpe_get_good")
    return m


def fpe_get_windows(P: Poly, n: int, stream=None):
    import torch
    lib = _load()
    dev = torch.device("cuda", P.device) if P.device is not None else torch.device("cuda")
    l = torch.empty(n, dtype=torch.int64, device=dev)
    r = torch.empty(n, dtype=torch.int64, device=dev)
    N = torch.empty(n, dtype=torch.float64, device=dev)
    _check(lib.fpe_get_windows(P.handle, n, _dptr(l), _dptr(r), _dptr(N), _stream(stream)), "fpe_get_windows")
    return l, r, N


def fpe_sync(P: Poly, stream=None):
    _check(_load().fpe_sync(P.handle, _stream(stream)), "fpe_sync")


def fpe_status_string(st: int) -> str:
    return _load().fpe_status_string(int(st)).decode()


def fpe_profile_enable(on: bool = True):
    _load().fpe_profile_enable(int(bool(on)))


def fpe_profile_reset():
    _load().fpe_profile_reset()


def fpe_profile_read(name: str = ""):
    """(total device ms, launches) of this library's kernels whose name contains `name`."""
    lib = _load()
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    _check(lib.fpe_profile_read(name.encode(), ctypes.byref(ms), ctypes.byref(cnt)), "fpe_profile_read")
    return ms.value, cnt.value


def fpe_measure_fma_peak(precision: int = 64, reps: int = 5) -> float:
    """Measured FMA/s of the current device (FP64 or FP32)."""
    v = ctypes.c_double()
    _check(_load().fpe_measure_fma_peak(int(precision), int(reps), ctypes.byref(v)), "fpe_measure_fma_peak")
    return v.value


NOALLOC_MAX_POINTS = 32768


def fpe_eval_noalloc(P: Poly, z_re, z_im=None, out=None, nterms=None, bits_lost=None, stream=None):
    """fpe_eval without any device allocation (at most NOALLOC_MAX_POINTS points;
    calls share one built-in scratch array and must not overlap on the GPU)."""
    lib = _load()
    n = _eval_args(P, z_re, z_im, out, nterms, bits_lost)
    if out is None:
        out = empty_out(n, z_re.device)
    _check(lib.fpe_eval_noalloc(P.handle, _dptr(z_re), _dptr(z_im), n, _dptr(out), _dptr(nterms),
                                _dptr(bits_lost), _stream(stream)), "fpe_eval_noalloc")
    return out


class Batch:
    """A batch of preconditioned polynomials with fixed point offsets (fpe_batch_t)."""

    def __init__(self, polys: Sequence[Poly], pt_offsets):
        lib = _load()
        self.polys = list(polys)  # keep the handles alive
        self.offsets = np.ascontiguousarray(pt_offsets, dtype=np.int64)
        hs = (ctypes.c_void_p * len(self.polys))(*[p.handle.value for p in self.polys])
        h = ctypes.c_void_p()
        _check(lib.fpe_batch_create(hs, len(self.polys), _np_ptr(self.offsets), ctypes.byref(h)), "fpe_batch_create")
        self._h = h

    @property
    def n(self) -> int:
        return int(self.offsets[-1])

    def __del__(self):
        try:
            if self._h and self._h.value:
                _load().fpe_batch_destroy(self._h)
                self._h = ctypes.c_void_p(None)
        except Exception:
            pass


def fpe_batch_create(polys: Sequence[Poly], pt_offsets) -> Batch:
    return Batch(polys, pt_offsets)


def fpe_batch_eval(B: Batch, z_re, z_im=None, out=None, nterms=None, stream=None):
    import torch
    lib = _load()
    if _points(z_re, z_im) != B.n:
        raise ValueError(f"the batch has {B.n} points")
    if out is not None:
        _check_out(out, B.n, z_re.device)
    _check_vec(nterms, B.n, z_re.device, torch.int32, "nterms")
    if out is None:
        out = empty_out(B.n, z_re.device)
    _check(lib.fpe_batch_eval(B._h, _dptr(z_re), _dptr(z_im), _dptr(out), _dptr(nterms), _stream(stream)),
           "fpe_batch_eval")
    return out


def fpe_batch_sync(B: Batch, stream=None):
    _check(_load().fpe_batch_sync(B._h, _stream(stream)), "fpe_batch_sync")


def fpe_set_tuning(P: Poly, long_window: int, lane_chunk: int):
    t = Tuning(long_window, lane_chunk, 0.0)
    _check(_load().fpe_set_tuning(P.handle, ctypes.byref(t)), "fpe_set_tuning")


def fpe_get_tuning(P: Poly) -> dict:
    t = Tuning()
    _check(_load().fpe_get_tuning(P.handle, ctypes.byref(t)), "fpe_get_tuning")
    return t.as_dict()


def fpe_set_tensor_path(P: Poly, min_window: int):
    """Tensor-core window sums for windows of at least min_window terms (0: off)."""
    _check(_load().fpe_set_tensor_path(P.handle, int(min_window)), "fpe_set_tensor_path")


def fpe_get_tensor_path(P: Poly) -> dict:
    mw, npc = ctypes.c_int64(), ctypes.c_int32()
    _check(_load().fpe_get_tensor_path(P.handle, ctypes.byref(mw), ctypes.byref(npc)), "fpe_get_tensor_path")
    return {"min_window": int(mw.value), "pieces": int(npc.value)}


TENSOR_STATS = ("points", "tiles", "items", "subtiles", "chunk_blocks", "rejected")


def fpe_tensor_stats(P: Poly, stream=None) -> dict:
    """What the tensor-core path did in the handle's last evaluation (all 0 if it did not run)."""
    v = (ctypes.c_int64 * len(TENSOR_STATS))()
    _check(_load().fpe_tensor_stats(P.handle, v, len(TENSOR_STATS), _stream(stream)), "fpe_tensor_stats")
    return dict(zip(TENSOR_STATS, (int(x) for x in v)))


CERT_STATS = ("resummed_windows",)


def fpe_cert_stats(P: Poly, stream=None) -> dict:
    """Windows of the last fpe_eval whose FP64 sums failed their
    rounding-error certificates and were summed again exactly."""
    v = (ctypes.c_int64 * len(CERT_STATS))()
    _check(_load().fpe_cert_stats(P.handle, v, len(CERT_STATS), _stream(stream)), "fpe_cert_stats")
    return dict(zip(CERT_STATS, (int(x) for x in v)))


def fpe_measure_mma_peak(reps: int = 5) -> float:
    """Measured bf16 mma.sync flop/s of the current device (the tensor-core sums' instruction)."""
    v = ctypes.c_double()
    _check(_load().fpe_measure_mma_peak(int(reps), ctypes.byref(v)), "fpe_measure_mma_peak")
    return v.value


def fpe_autotune(P: Poly, z_re, z_im=None, stream=None) -> dict:
    """Time fpe_eval over the tuning grid on these device points; the fastest
    setting stays in the handle and is returned."""
    t = Tuning()
    n = _eval_args(P, z_re, z_im)
    _check(_load().fpe_autotune(P.handle, _dptr(z_re), _dptr(z_im), n, _stream(stream),
                                ctypes.byref(t)), "fpe_autotune")
    return t.as_dict()


def fpe_batch_set_tuning(B: Batch, long_window: int, lane_chunk: int):
    t = Tuning(long_window, lane_chunk, 0.0)
    _check(_load().fpe_batch_set_tuning(B._h, ctypes.byref(t)), "fpe_batch_set_tuning")


def fpe_batch_autotune(B: Batch, z_re, z_im=None, stream=None) -> dict:
    t = Tuning()
    if _points(z_re, z_im) != B.n:
        raise ValueError(f"the batch has {B.n} points")
    _check(_load().fpe_batch_autotune(B._h, _dptr(z_re), _dptr(z_im), _stream(stream), ctypes.byref(t)),
           "fpe_batch_autotune")
    return t.as_dict()


def fpe_newton(P: Poly, z_re, z_im=None, inc=None, z_next_re=None, z_next_im=None, stream=None):
    """One Newton step: returns (inc as (n, 3) fpe_xc64, z_next_re, z_next_im)."""
    import torch
    lib = _load()
    n = _eval_args(P, z_re, z_im, inc)
    _check_vec(z_next_re, n, z_re.device, torch.float64, "z_next_re")
    _check_vec(z_next_im, n, z_re.device, torch.float64, "z_next_im")
    if inc is None:
        inc = empty_out(n, z_re.device)
    if z_next_re is None:
        z_next_re = torch.empty_like(z_re)
    if z_next_im is None and z_im is not None:
        z_next_im = torch.empty_like(z_im)
    _check(lib.fpe_newton(P.handle, _dptr(z_re), _dptr(z_im), n, _dptr(inc), _dptr(z_next_re), _dptr(z_next_im),
                          _stream(stream)), "fpe_newton")
    return inc, z_next_re, z_next_im


def fpe_grad_points(P: Poly, z_re, z_im, g_re, g_im, stream=None):
    import torch
    lib = _load()
    n = _eval_args(P, z_re, z_im)
    if g_re is None:
        raise ValueError("g_re is required")
    _check_vec(g_re, n, z_re.device, torch.float64, "g_re")
    _check_vec(g_im, n, z_re.device, torch.float64, "g_im")
    gz_re = torch.empty_like(z_re)
    gz_im = torch.empty_like(z_re)
    _check(lib.fpe_grad_points(P.handle, _dptr(z_re), _dptr(z_im), n, _dptr(g_re), _dptr(g_im), _dptr(gz_re),
                               _dptr(gz_im), _stream(stream)), "fpe_grad_points")
    return gz_re, gz_im


def fpe_grad_coeffs(P: Poly, z_re, z_im, g_re, g_im, ga_re, ga_im=None, stream=None):
    """Adds dL/da_k into ga_re/ga_im (device float64, n_coef entries)."""
    import torch
    lib = _load()
    n = _eval_args(P, z_re, z_im)
    if g_re is None or ga_re is None:
        raise ValueError("g_re and ga_re are required")
    _check_vec(g_re, n, z_re.device, torch.float64, "g_re")
    _check_vec(g_im, n, z_re.device, torch.float64, "g_im")
    _check_vec(ga_re, P.n_coef, z_re.device, torch.float64, "ga_re")
    _check_vec(ga_im, P.n_coef, z_re.device, torch.float64, "ga_im")
    _check(lib.fpe_grad_coeffs(P.handle, _dptr(z_re), _dptr(z_im), n, _dptr(g_re), _dptr(g_im), _dptr(ga_re),
                               _dptr(ga_im), _stream(stream)), "fpe_grad_coeffs")
    return ga_re, ga_im


def fpe_to_complex(v, stream=None):
    """(re, im) 2^e of an (n, 3) fpe_xc64 tensor as two float64 tensors."""
    import torch
    lib = _load()
    n = int(v.shape[0])
    _check_out(v, n, v.device)
    re = torch.empty(n, dtype=torch.float64, device=v.device)
    im = torch.empty(n, dtype=torch.float64, device=v.device)
    _check(lib.fpe_to_complex(_dptr(v), n, _dptr(re), _dptr(im), _stream(stream)), "fpe_to_complex")
    return re, im


def fpe_analyse(P: Poly):
    """Per coefficient, the log2|z| interval [lam_lo, lam_hi] where it is kept (NaN if never)."""
    lib = _load()
    lo = np.zeros(P.n_coef)
    hi = np.zeros(P.n_coef)
    _check(lib.fpe_analyse(P.handle, _np_ptr(lo), _np_ptr(hi), P.n_coef), "fpe_analyse")
    return lo, hi
