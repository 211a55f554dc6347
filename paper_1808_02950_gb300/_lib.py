"""ctypes binding of libtdct (include/tdct.h): the same names, marshalling only.

Every function takes device tensors (torch, for memory and streams) or plain
integers, converts them to pointers and sizes, calls the C entry point and
raises ``TdctError`` on a non-zero status.  No arithmetic of the codec runs
here; if the CUDA library cannot be loaded, every call fails loudly.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

TDCT_OK, TDCT_EINVAL, TDCT_ENOTORTHO, TDCT_ECUDA = 0, 1, 2, 3
TDCT_ETIMEOUT, TDCT_EDEVICE, TDCT_ENOMEM, TDCT_EUNSUPPORTED = 4, 5, 6, 7
TDCT_U8, TDCT_I16 = 0, 1
TDCT_FP32, TDCT_BF16, TDCT_BF16X3 = 0, 1, 2
TDCT_PATH_AUTO, TDCT_PATH_BUTTERFLY, TDCT_PATH_TENSOR, TDCT_PATH_TENSOR_PIPELINED = 0, 1, 2, 3
TDCT_LOAD_PLAIN, TDCT_LOAD_BULK, TDCT_LOAD_STAGED = 0, 1, 2

# T1 of §4.1 and n = diag(T1 T1^T), the arguments the paper states (S = diag(1/sqrt(n))).
T1 = (
    (1, 1, 1, 1, 1, 1, 1, 1),
    (2, 2, 1, 0, 0, -1, -2, -2),
    (2, 1, -1, -2, -2, -1, 1, 2),
    (1, 0, -2, -2, 2, 2, 0, -1),
    (1, -1, -1, 1, 1, -1, -1, 1),
    (2, -2, 0, 1, -1, 0, 2, -2),
    (1, -2, 2, -1, -1, 2, -2, 1),
    (0, -1, 2, -2, 2, -2, 1, 0),
)
N1 = (8, 18, 20, 18, 8, 18, 20, 18)

EXPORTS = (
    "tdct_forward", "tdct_zonal_inverse", "tdct_codec_error", "tdct_codec_error_batched",
    "tdct_codec_error_batched_noalloc", "tdct_codec_error_batched_host", "tdct_ssim_batched",
    "tdct_search", "tdct_codec_error_jam", "tdct_sweep_batched", "tdct_dct_sweep_batched",
    "tdct_plan_create", "tdct_plan_launch", "tdct_plan_kernel_count", "tdct_plan_config",
    "tdct_plan_groups",
    "tdct_plan_destroy",
    "tdct_dct_codec_error", "tdct_sync_status", "tdct_debug_inject_wait_timeout",
    "tdct_debug_search_hit_cap", "tdct_shutdown",
    "tdct_last_error", "tdct_version",
)


class TdctError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tdct error {code}: {msg}")
        self.code = code


class TdctPlane(ctypes.Structure):
    _fields_ = [
        ("img", ctypes.c_void_p), ("pitch", ctypes.c_int64),
        ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("r", ctypes.c_int32),
        ("dtype", ctypes.c_int32), ("recon", ctypes.c_void_p), ("recon_pitch", ctypes.c_int64),
    ]


class TdctPlanGroup(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("r", ctypes.c_int32), ("load", ctypes.c_int32),
                ("planes", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libtdct.so (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libtdct.so is missing at {_build.LIB}; run build()")
    L = ctypes.CDLL(_build.LIB)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.tdct_forward.argtypes = [vp, i64, i32, i32, i32, vp, vp, vp, vp]
    L.tdct_zonal_inverse.argtypes = [vp, i32, i32, i32, vp, vp, i32, vp, i64, vp]
    L.tdct_codec_error.argtypes = [vp, i64, i32, i32, i32, vp, vp, i32, vp, i64, vp, vp, vp]
    L.tdct_codec_error_batched.argtypes = [vp, i32, vp, vp, vp, vp, i32, vp]
    L.tdct_codec_error_batched_noalloc.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.tdct_codec_error_batched_host.argtypes = [vp, i32, vp, vp, vp, vp, ctypes.c_size_t, vp]
    L.tdct_ssim_batched.argtypes = [vp, i32, vp, vp]
    L.tdct_sweep_batched.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.tdct_dct_sweep_batched.argtypes = [vp, i32, i32, vp, vp, vp]
    L.tdct_search.argtypes = [i32, vp, i32, vp, i32, vp, vp, i32, i32, vp, vp, vp]
    L.tdct_codec_error_jam.argtypes = [vp, i64, i32, i32, i32, i32, vp, vp, i32, vp, i64, vp, vp,
                                       vp]
    L.tdct_plan_create.argtypes = [vp, i32, vp, vp, i32, ctypes.POINTER(ctypes.c_void_p)]
    L.tdct_plan_launch.argtypes = [vp, vp, vp, vp]
    L.tdct_plan_kernel_count.argtypes = [vp]
    L.tdct_plan_config.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_float)]
    L.tdct_plan_groups.argtypes = [vp, ctypes.POINTER(TdctPlanGroup), i32, ctypes.POINTER(ctypes.c_int)]
    L.tdct_plan_destroy.argtypes = [vp]
    L.tdct_plan_destroy.restype = None
    L.tdct_dct_codec_error.argtypes = [vp, i64, i32, i32, i32, i32, i32, vp, vp, i64, vp, vp, vp]
    L.tdct_sync_status.argtypes = [vp]
    L.tdct_shutdown.argtypes = []
    L.tdct_debug_inject_wait_timeout.argtypes = [i32]
    L.tdct_debug_search_hit_cap.argtypes = [i32]
    L.tdct_last_error.restype = ctypes.c_char_p
    L.tdct_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("tdct_plan_destroy", "tdct_last_error", "tdct_version"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int) -> None:
    if rc != TDCT_OK:
        raise TdctError(rc, load().tdct_last_error().decode())


def _T_n(T=None, n=None):
    T = T1 if T is None else T
    n = N1 if n is None else n
    flat = [int(v) for row in T for v in row]
    tb = (ctypes.c_int8 * 64)(*flat)
    nb = (ctypes.c_int32 * 8)(*[int(v) for v in n])
    return tb, nb


def _ptr(t) -> int | None:
    """Device address of a tensor (or an int address, or None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _plane_info(img):
    """(dtype code, H, W, pitch bytes) of a 2-D uint8 / int16 tensor."""
    import torch

    if img.dim() != 2:
        raise ValueError("planes are 2-D tensors")
    if img.dtype == torch.uint8:
        dt = TDCT_U8
    elif img.dtype == torch.int16:
        dt = TDCT_I16
    else:
        raise TypeError("planes are uint8 or int16")
    if img.stride(1) != 1:
        raise ValueError("plane rows must be contiguous")
    return dt, img.shape[0], img.shape[1], img.stride(0) * img.element_size()


def tdct_version() -> str:
    return load().tdct_version().decode()


def tdct_forward(img, coef, T=None, n=None, stream=None) -> None:
    dt, H, W, pitch = _plane_info(img)
    tb, nb = _T_n(T, n)
    _check(load().tdct_forward(_ptr(img), pitch, H, W, dt, tb, nb, _ptr(coef), _stream(stream)))


def tdct_zonal_inverse(coef, r: int, out, T=None, n=None, stream=None) -> None:
    dt, H, W, pitch = _plane_info(out)
    tb, nb = _T_n(T, n)
    _check(load().tdct_zonal_inverse(_ptr(coef), H, W, dt, tb, nb, int(r), _ptr(out), pitch,
                                     _stream(stream)))


def tdct_codec_error(img, r: int, sse, recon=None, psnr=None, T=None, n=None, stream=None) -> None:
    dt, H, W, pitch = _plane_info(img)
    rp = _plane_info(recon)[3] if recon is not None else 0
    tb, nb = _T_n(T, n)
    _check(load().tdct_codec_error(_ptr(img), pitch, H, W, dt, tb, nb, int(r), _ptr(recon), rp,
                                   _ptr(sse), _ptr(psnr), _stream(stream)))


def make_planes(imgs, rs, recons=None):
    """ctypes array of tdct_plane from lists of 2-D tensors and retentions."""
    arr = (TdctPlane * len(imgs))()
    for i, img in enumerate(imgs):
        dt, H, W, pitch = _plane_info(img)
        rec = recons[i] if recons is not None else None
        arr[i] = TdctPlane(_ptr(img), pitch, H, W, int(rs[i]), dt, _ptr(rec),
                           _plane_info(rec)[3] if rec is not None else 0)
    return arr


def make_planes_raw(rows):
    """ctypes array of tdct_plane from (img_ptr, pitch, H, W, r, dtype, recon_ptr, recon_pitch)."""
    arr = (TdctPlane * len(rows))()
    for i, row in enumerate(rows):
        arr[i] = TdctPlane(*row)
    return arr


def tdct_codec_error_batched(planes, sse, psnr=None, path=TDCT_PATH_AUTO, T=None, n=None,
                             stream=None) -> None:
    tb, nb = _T_n(T, n)
    _check(load().tdct_codec_error_batched(ctypes.addressof(planes), len(planes), tb, nb,
                                           _ptr(sse), _ptr(psnr), int(path), _stream(stream)))


NOALLOC_MAX_PLANES = 2048


def tdct_codec_error_batched_noalloc(planes, sse, psnr=None, T=None, n=None, stream=None) -> None:
    """tdct_codec_error_batched without any device allocation (fixed table)."""
    tb, nb = _T_n(T, n)
    _check(load().tdct_codec_error_batched_noalloc(ctypes.addressof(planes), len(planes), tb, nb,
                                                   _ptr(sse), _ptr(psnr), _stream(stream)))


def tdct_codec_error_batched_host(planes, sse, psnr=None, T=None, n=None, chunk_bytes=0,
                                  stream=None) -> None:
    """The batched codec on planes in host memory (``make_planes`` over CPU
    tensors; pinned tensors let the copies overlap the codec); SSE / PSNR
    land in the CPU tensors ``sse`` / ``psnr`` once ``stream`` reaches the
    end of the call's work."""
    tb, nb = _T_n(T, n)
    _check(load().tdct_codec_error_batched_host(ctypes.addressof(planes), len(planes), tb, nb,
                                                _ptr(sse), _ptr(psnr), int(chunk_bytes),
                                                _stream(stream)))


def tdct_sweep_batched(imgs, sse, psnr=None, T=None, n=None, stream=None) -> None:
    """SSE (and PSNR) of every u8 plane of ``imgs`` for each r = 1..64 into
    ``sse[64 * p + r - 1]`` (int64 device tensor of 64 * len(imgs))."""
    planes = make_planes(imgs, [64] * len(imgs))
    tb, nb = _T_n(T, n)
    _check(load().tdct_sweep_batched(ctypes.addressof(planes), len(planes), tb, nb, _ptr(sse),
                                     _ptr(psnr), _stream(stream)))


def tdct_dct_sweep_batched(imgs, sse, psnr=None, precision=TDCT_FP32, stream=None) -> None:
    """The sweep with the exact DCT in FP32 (same layout as tdct_sweep_batched)."""
    planes = make_planes(imgs, [64] * len(imgs))
    _check(load().tdct_dct_sweep_batched(ctypes.addressof(planes), len(planes), int(precision),
                                         _ptr(sse), _ptr(psnr), _stream(stream)))


class TdctSsimPlane(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_void_p), ("x_pitch", ctypes.c_int64),
        ("y", ctypes.c_void_p), ("y_pitch", ctypes.c_int64),
        ("H", ctypes.c_int32), ("W", ctypes.c_int32),
    ]


def tdct_ssim_batched(pairs, mssim, stream=None) -> None:
    """Mean SSIM of each (x, y) pair of 2-D uint8 device tensors into the
    float64 device tensor ``mssim``."""
    arr = (TdctSsimPlane * len(pairs))()
    for i, (x, y) in enumerate(pairs):
        _, H, W, xp = _plane_info(x)
        _, Hy, Wy, yp = _plane_info(y)
        if (H, W) != (Hy, Wy):
            raise ValueError("SSIM pairs need equal shapes")
        arr[i] = TdctSsimPlane(_ptr(x), xp, _ptr(y), yp, H, W)
    _check(load().tdct_ssim_batched(ctypes.addressof(arr), len(pairs), _ptr(mssim),
                                    _stream(stream)))


def tdct_codec_error_jam(img, B: int, T, r: int, sse, recon=None, psnr=None, stream=None) -> None:
    """The codec with B x B blocks (16 or 32) and the JAM matrix T (B x B)."""
    dt, H, W, pitch = _plane_info(img)
    rp = _plane_info(recon)[3] if recon is not None else 0
    flat = [int(v) for row in T for v in row]
    tb = (ctypes.c_int8 * (B * B))(*flat)
    nb = (ctypes.c_int32 * B)(*[sum(int(v) * int(v) for v in row) for row in T])
    _check(load().tdct_codec_error_jam(_ptr(img), pitch, H, W, dt, int(B), tb, nb, int(r),
                                       _ptr(recon), rp, _ptr(sse), _ptr(psnr), _stream(stream)))


def tdct_search(N: int, alphabet, order, fixed=None, tie: str = "small", stream=None):
    """The greedy angle search for one row order on the GPU.  ``order``:
    0-based rows searched in turn; ``fixed``: {row: vector} presets.
    Returns (T as an N x N list of lists, complete)."""
    alph = (ctypes.c_int8 * len(alphabet))(*[int(v) for v in alphabet])
    order = list(order)
    ordb = (ctypes.c_int32 * len(order))(*order)
    fixed = fixed or {}
    frows = (ctypes.c_int32 * max(1, len(fixed)))(*list(fixed.keys()))
    fvals = (ctypes.c_int8 * max(1, N * len(fixed)))(*[int(v) for row in fixed.values()
                                                        for v in row])
    T = (ctypes.c_int8 * (N * N))()
    complete = ctypes.c_int32(0)
    _check(load().tdct_search(N, alph, len(alphabet), ordb, len(order),
                              frows if fixed else None, fvals if fixed else None, len(fixed),
                              {"small": 0, "large": 1}[tie], T, ctypes.byref(complete),
                              _stream(stream)))
    return [[T[i * N + j] for j in range(N)] for i in range(N)], bool(complete.value)


class TdctPlan:
    """Owner of a tdct_plan (tdct_plan_create / _launch / _destroy)."""

    def __init__(self, planes, path=TDCT_PATH_AUTO, T=None, n=None):
        tb, nb = _T_n(T, n)
        h = ctypes.c_void_p()
        _check(load().tdct_plan_create(ctypes.addressof(planes), len(planes), tb, nb, int(path),
                                       ctypes.byref(h)))
        self._h = h
        self.nplanes = len(planes)
        self._planes = planes

    def launch(self, sse, psnr=None, stream=None) -> None:
        _check(load().tdct_plan_launch(self._h, _ptr(sse), _ptr(psnr), _stream(stream)))

    def kernel_count(self) -> int:
        return load().tdct_plan_kernel_count(self._h)

    def config(self) -> dict:
        """The engine, CTAs per SM and tuned time the plan uses."""
        path, cps, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        _check(load().tdct_plan_config(self._h, ctypes.byref(path), ctypes.byref(cps), ctypes.byref(ms)))
        names = {TDCT_PATH_BUTTERFLY: "butterfly", TDCT_PATH_TENSOR: "tensor",
                 TDCT_PATH_TENSOR_PIPELINED: "tensor_pipelined"}
        return {"path": names.get(path.value, path.value), "ctas_per_sm": cps.value,
                "tuned_ms": ms.value}

    def groups(self) -> list:
        """One dict per codec launch: dtype, r, load path, number of planes."""
        n = ctypes.c_int()
        _check(load().tdct_plan_groups(self._h, None, 0, ctypes.byref(n)))
        arr = (TdctPlanGroup * max(n.value, 1))()
        _check(load().tdct_plan_groups(self._h, arr, n.value, ctypes.byref(n)))
        loads = {TDCT_LOAD_PLAIN: "plain", TDCT_LOAD_BULK: "bulk", TDCT_LOAD_STAGED: "staged"}
        return [{"dtype": "u8" if g.dtype == TDCT_U8 else "i16", "r": g.r,
                 "load": loads.get(g.load, g.load), "planes": g.planes} for g in arr[:n.value]]

    def close(self) -> None:
        if self._h:
            load().tdct_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tdct_plan_create(planes, path=TDCT_PATH_AUTO, T=None, n=None) -> TdctPlan:
    return TdctPlan(planes, path, T, n)


def tdct_dct_codec_error(img, r: int, sse, precision=TDCT_FP32, coef=None, recon=None, psnr=None,
                         stream=None) -> None:
    dt, H, W, pitch = _plane_info(img)
    rp = _plane_info(recon)[3] if recon is not None else 0
    _check(load().tdct_dct_codec_error(_ptr(img), pitch, H, W, dt, int(r), int(precision),
                                       _ptr(coef), _ptr(recon), rp, _ptr(sse), _ptr(psnr),
                                       _stream(stream)))


def tdct_debug_inject_wait_timeout(enable: bool = True) -> None:
    _check(load().tdct_debug_inject_wait_timeout(1 if enable else 0))


def tdct_debug_search_hit_cap(cap: int = -1) -> None:
    _check(load().tdct_debug_search_hit_cap(int(cap)))


def tdct_sync_status(stream=None) -> None:
    _check(load().tdct_sync_status(_stream(stream)))


def tdct_shutdown() -> None:
    """Release the library-owned resources (transfer streams); the library
    stays usable afterwards."""
    _check(load().tdct_shutdown())
