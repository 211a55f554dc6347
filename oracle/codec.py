"""Python entry points of the CPU oracle (ctypes over ``tdct_oracle.c``).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
legs of ``bench.py`` may import this module; the product path never does.

``build()`` compiles ``tdct_oracle.c`` with gcc into ``oracle/_build``.  The
numpy wrappers below take plain arrays:

* ``codec_plane(img, T, r)``        -> (sse, recon, coef)   integer path
* ``zonal_inverse_plane(coef, ...)`` -> recon               integer path
* ``dct_codec_plane(img, r)``       -> (sse, recon, coef)   FP64 exact DCT
* ``psnr(sse, npix)``
* ``exact_block_codec(X, T, r)``    -> pure-Python ``Fraction`` brute force of
  one block, used to pin the C oracle (no shared code with it).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from fractions import Fraction
from math import gcd

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdct_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libtdct_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (plain C, -O2) and return the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    if force or not fresh:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u8p = ctypes.c_void_p
        L.orc_zigzag.argtypes = [i32p, i32p]
        L.orc_row_norms.argtypes = [i32p, i64p]
        L.orc_row_norms.restype = ctypes.c_int
        L.orc_forward_block.argtypes = [i64p, i32p, i64p]
        L.orc_forward_block_kron.argtypes = [i64p, i32p, i64p]
        L.orc_codec_plane.argtypes = [
            u8p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            i32p, ctypes.c_int, u8p, ctypes.c_int64, u8p, i64p,
        ]
        L.orc_codec_plane.restype = ctypes.c_int
        L.orc_zonal_inverse_plane.argtypes = [
            u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int,
            u8p, ctypes.c_int64,
        ]
        L.orc_zonal_inverse_plane.restype = ctypes.c_int
        L.orc_dct_codec_plane.argtypes = [
            u8p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_int, u8p, ctypes.c_int64, u8p, i64p,
        ]
        L.orc_dct_codec_plane.restype = ctypes.c_int
        L.orc_psnr.argtypes = [ctypes.c_int64, ctypes.c_int64]
        L.orc_psnr.restype = ctypes.c_double
        L.orc_dct_matrix.argtypes = [ctypes.POINTER(ctypes.c_double)]
        L.orc_ssim_plane.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double)]
        L.orc_ssim_plane.restype = ctypes.c_int
        L.orc_codec_plane_b.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_int64, i64p]
        L.orc_codec_plane_b.restype = ctypes.c_int
        L.orc_zigzag_b.argtypes = [ctypes.c_int, i32p]
        L.orc_zigzag_b.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _T32(T) -> np.ndarray:
    T = np.ascontiguousarray(np.asarray(T), dtype=np.int32)
    assert T.shape == (8, 8)
    return T


def zigzag() -> tuple[np.ndarray, np.ndarray]:
    """(position of scan index, scan index of position), positions p = 8 i + j."""
    a = np.zeros(64, np.int32)
    b = np.zeros(64, np.int32)
    lib().orc_zigzag(_ptr(a, ctypes.c_int32), _ptr(b, ctypes.c_int32))
    return a, b


def row_norms(T) -> np.ndarray | None:
    n = np.zeros(8, np.int64)
    rc = lib().orc_row_norms(_ptr(_T32(T), ctypes.c_int32), _ptr(n, ctypes.c_int64))
    return n if rc == 0 else None


def forward_block(X, T, method: str = "definition") -> np.ndarray:
    X = np.ascontiguousarray(np.asarray(X, dtype=np.int64).reshape(64))
    Z = np.zeros(64, np.int64)
    f = lib().orc_forward_block if method == "definition" else lib().orc_forward_block_kron
    f(_ptr(X, ctypes.c_int64), _ptr(_T32(T), ctypes.c_int32), _ptr(Z, ctypes.c_int64))
    return Z.reshape(8, 8)


def _plane_args(img: np.ndarray):
    img = np.ascontiguousarray(img)
    if img.dtype == np.uint8:
        dtype = 0
    elif img.dtype == np.int16:
        dtype = 1
    else:
        raise TypeError("oracle planes are uint8 or int16")
    H, W = img.shape
    return img, dtype, H, W, img.strides[0]


def codec_plane(img: np.ndarray, T, r: int, want_recon: bool = True, want_coef: bool = False):
    """Integer-path codec of one plane.  Returns (sse, recon or None, coef or None)."""
    img, dtype, H, W, pitch = _plane_args(img)
    recon = np.zeros_like(img) if want_recon else None
    nby, nbx = (H + 7) // 8, (W + 7) // 8
    coef = np.zeros((nby, nbx, 8, 8), np.int64) if want_coef else None
    sse = ctypes.c_int64(0)
    rc = lib().orc_codec_plane(
        img.ctypes.data, pitch, H, W, dtype, _ptr(_T32(T), ctypes.c_int32), r,
        recon.ctypes.data if recon is not None else None,
        recon.strides[0] if recon is not None else 0,
        coef.ctypes.data if coef is not None else None, ctypes.byref(sse),
    )
    if rc != 0:
        raise ValueError(f"oracle codec_plane failed with code {rc}")
    return sse.value, recon, coef


def zonal_inverse_plane(coef: np.ndarray, H: int, W: int, T, r: int, dtype=np.uint8):
    coef = np.ascontiguousarray(coef, dtype=np.int64)
    recon = np.zeros((H, W), dtype=dtype)
    rc = lib().orc_zonal_inverse_plane(
        coef.ctypes.data, H, W, 0 if dtype == np.uint8 else 1,
        _ptr(_T32(T), ctypes.c_int32), r, recon.ctypes.data, recon.strides[0],
    )
    if rc != 0:
        raise ValueError(f"oracle zonal_inverse_plane failed with code {rc}")
    return recon


def dct_codec_plane(img: np.ndarray, r: int, want_recon: bool = True, want_coef: bool = False):
    """FP64 exact-DCT codec of one plane.  Returns (sse, recon or None, coef or None)."""
    img, dtype, H, W, pitch = _plane_args(img)
    recon = np.zeros_like(img) if want_recon else None
    nby, nbx = (H + 7) // 8, (W + 7) // 8
    coef = np.zeros((nby, nbx, 8, 8), np.float64) if want_coef else None
    sse = ctypes.c_int64(0)
    rc = lib().orc_dct_codec_plane(
        img.ctypes.data, pitch, H, W, dtype, r,
        recon.ctypes.data if recon is not None else None,
        recon.strides[0] if recon is not None else 0,
        coef.ctypes.data if coef is not None else None, ctypes.byref(sse),
    )
    if rc != 0:
        raise ValueError(f"oracle dct_codec_plane failed with code {rc}")
    return sse.value, recon, coef


def codec_plane_b(img: np.ndarray, T, B: int, r: int, want_recon: bool = True):
    """The codec with B x B blocks (B = 8, 16, 32) and the B x B matrix T.
    Returns (sse, recon or None)."""
    img, dtype, H, W, pitch = _plane_args(img)
    T = np.ascontiguousarray(np.asarray(T), dtype=np.int32)
    assert T.shape == (B, B)
    recon = np.zeros_like(img) if want_recon else None
    sse = ctypes.c_int64(0)
    rc = lib().orc_codec_plane_b(img.ctypes.data, pitch, H, W, dtype, B,
                                 _ptr(T, ctypes.c_int32), r,
                                 recon.ctypes.data if recon is not None else None,
                                 recon.strides[0] if recon is not None else 0, ctypes.byref(sse))
    if rc != 0:
        raise ValueError(f"orc_codec_plane_b failed ({rc})")
    return sse.value, recon


def zigzag_b(B: int) -> np.ndarray:
    """Scan index of every position (i, j) of a B x B block, as a B x B array."""
    out = np.zeros(B * B, np.int32)
    assert lib().orc_zigzag_b(B, _ptr(out, ctypes.c_int32)) == 0
    return out.reshape(B, B)


def ssim_plane(x: np.ndarray, y: np.ndarray) -> float:
    """MSSIM of two u8 planes (Wang et al. 2004 window and constants, valid
    window positions only); raises ValueError below 11 x 11."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    assert x.shape == y.shape and x.ndim == 2
    out = ctypes.c_double(0.0)
    rc = lib().orc_ssim_plane(x.ctypes.data, x.strides[0], y.ctypes.data, y.strides[0],
                              x.shape[0], x.shape[1], ctypes.byref(out))
    if rc != 0:
        raise ValueError("SSIM needs planes of at least 11 x 11 samples")
    return out.value


def psnr(sse: int, npix: int) -> float:
    return lib().orc_psnr(int(sse), int(npix))


def dct_matrix_c() -> np.ndarray:
    C = np.zeros(64, np.float64)
    lib().orc_dct_matrix(_ptr(C, ctypes.c_double))
    return C.reshape(8, 8)


# ---- pure-Python exact brute force (independent of the C code) ------------


def _zigzag_py():
    """Zig-zag scan generated from its geometric description, independently."""
    seq = []
    for s in range(15):
        diag = [(i, s - i) for i in range(8) if 0 <= s - i < 8]
        # diag runs with increasing row index i; even diagonals are walked
        # from the bottom-left corner upwards.
        if s % 2 == 0:
            diag = diag[::-1]
        seq.extend(diag)
    return seq


def exact_block_codec(X, T, r: int, lo: int = 0, hi: int = 255):
    """One block through C_hat = S T, zonal r, C_hat^T B' C_hat, in Fractions.

    S = diag(1/sqrt(n)) is irrational, so the products are formed with
    S^2 = diag(1/n), which is exact: C_hat^T (M o C_hat X C_hat^T) C_hat =
    T^T S (M o S Z S) S T = T^T (M o Z o (1/n)(1/n)^T) T.  Rounding is half
    away from zero, then clamping to [lo, hi].
    Returns (Z, exact reconstruction as Fractions, rounded reconstruction).
    """
    X = [[int(v) for v in row] for row in np.asarray(X).reshape(8, 8)]
    T = [[int(v) for v in row] for row in np.asarray(T).reshape(8, 8)]
    n = [sum(v * v for v in row) for row in T]
    Z = [[sum(T[i][k] * X[k][l] * T[j][l] for k in range(8) for l in range(8))
          for j in range(8)] for i in range(8)]
    keep = set(_zigzag_py()[:r])
    Wf = [[Fraction(Z[i][j], n[i] * n[j]) if (i, j) in keep else Fraction(0)
           for j in range(8)] for i in range(8)]
    R = [[sum(T[i][k] * Wf[i][j] * T[j][l] for i in range(8) for j in range(8))
          for l in range(8)] for k in range(8)]
    out = []
    for k in range(8):
        row = []
        for l in range(8):
            v = R[k][l]
            a = abs(v)
            m = a.numerator // a.denominator
            if a - m >= Fraction(1, 2):
                m += 1
            x = m if v >= 0 else -m
            row.append(min(max(x, lo), hi))
        out.append(row)
    return np.array(Z, dtype=np.int64), R, np.array(out, dtype=np.int64)


def lcm_list(vals) -> int:
    L = 1
    for v in vals:
        L = L * int(v) // gcd(L, int(v))
    return L
