"""The C ABI loads, exports every declared symbol, and rejects bad arguments
on the host before touching the GPU (runs without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_1808_02950_gb300 as P
from paper_1808_02950_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FAKE = 0x10000  # never dereferenced: validation fails first


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tdct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tdct_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = P.load()
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert set(_lib.EXPORTS) <= set(names)


def test_version():
    assert "sm_103a" in P.tdct_version()


def _call_codec(**kw):
    L = P.load()
    a = dict(img=FAKE, pitch=64, H=16, W=64, dtype=0, r=10, recon=None, rpitch=0, sse=FAKE,
             psnr=None, T=None, n=None)
    a.update(kw)
    tb, nb = _lib._T_n(a["T"], a["n"])
    rc = L.tdct_codec_error(a["img"], a["pitch"], a["H"], a["W"], a["dtype"], tb, nb, a["r"],
                            a["recon"], a["rpitch"], a["sse"], a["psnr"], None)
    return rc, L.tdct_last_error().decode()


@pytest.mark.parametrize(
    "kw,code",
    [
        (dict(img=None), _lib.TDCT_EINVAL),
        (dict(sse=None), _lib.TDCT_EINVAL),
        (dict(sse=FAKE + 4), _lib.TDCT_EINVAL),
        (dict(r=0), _lib.TDCT_EINVAL),
        (dict(r=65), _lib.TDCT_EINVAL),
        (dict(H=0), _lib.TDCT_EINVAL),
        (dict(W=0), _lib.TDCT_EINVAL),
        (dict(W=-8), _lib.TDCT_EINVAL),
        (dict(pitch=63), _lib.TDCT_EINVAL),
        (dict(dtype=2), _lib.TDCT_EINVAL),
        (dict(dtype=1, pitch=64), _lib.TDCT_EINVAL),
        (dict(dtype=1, img=FAKE + 1, pitch=128), _lib.TDCT_EINVAL),
        (dict(recon=FAKE, rpitch=8), _lib.TDCT_EINVAL),
        (dict(n=(8, 18, 20, 18, 8, 18, 20, 17)), _lib.TDCT_ENOTORTHO),
        (dict(T=[[1] * 8] * 8, n=(8,) * 8), _lib.TDCT_ENOTORTHO),
    ],
)
def test_codec_error_rejects(kw, code):
    rc, msg = _call_codec(**kw)
    assert rc == code, msg
    assert msg


T2 = [[1, 1, 1, 1, 1, 1, 1, 1], [2, 1, 2, 0, 0, -2, -1, -2], [2, 1, -1, -2, -2, -1, 1, 2],
      [2, 0, -2, -1, 1, 2, 0, -2], [1, -1, -1, 1, 1, -1, -1, 1], [1, -2, 0, 2, -2, 0, 2, -1],
      [1, -2, 2, -1, -1, 2, -2, 1], [0, -2, 1, -2, 2, -1, 2, 0]]
N2 = (8, 18, 20, 18, 8, 18, 20, 18)


def test_other_orthogonal_T_passes_the_transform_checks():
    # T2 (§4.1) is accepted: the call gets as far as the plane checks
    rc, msg = _call_codec(T=T2, n=N2, img=None)
    assert rc == _lib.TDCT_EINVAL and "NULL plane" in msg, msg


def test_non_orthogonal_and_degenerate_T_rejected():
    # the BAS-2008 matrix of Table 2 as printed is not orthogonal: T T^T has
    # off-diagonal entries, so no diagonal S exists (Eq. (2))
    bas = [[1, 1, 1, 1, 1, 1, 1, 1], [1, 1, 1, 0, 0, -1, -1, -1], [1, 1, -1, -1, -1, -1, 1, 1],
           [1, 0, -1, 0, 0, 1, 0, -1], [1, -1, -1, 1, 1, -1, -1, 1], [1, -1, 1, 0, 0, -1, 1, -1],
           [1, -1, 1, -1, -1, 1, -1, 1], [1, -1, 1, -1, 1, -1, 1, -1]]
    rc, msg = _call_codec(T=bas, n=(8, 6, 8, 4, 8, 6, 8, 8))
    assert rc == _lib.TDCT_ENOTORTHO, msg
    zero_row = [list(r) for r in T2]
    zero_row[7] = [0] * 8
    rc, msg = _call_codec(T=zero_row, n=N2[:7] + (0,))
    assert rc == _lib.TDCT_ENOTORTHO and "zero" in msg, msg


def test_T_beyond_the_exact_32_bit_range_is_unsupported():
    # Walsh-Hadamard rows scaled by 1, 3, 5, 7: orthogonal, n = 8 c^2, and
    # lcm(n) = 8 * 9 * 25 * 49 > 725, outside the exact 32-bit reconstruction
    H = [[1]]
    for _ in range(3):
        H = [row + row for row in H] + [row + [-v for v in row] for row in H]
    c = [1, 3, 5, 7, 1, 3, 5, 7]
    T = [[c[k] * v for v in H[k]] for k in range(8)]
    rc, msg = _call_codec(T=T, n=tuple(8 * ck * ck for ck in c))
    assert rc == _lib.TDCT_EUNSUPPORTED and "lcm" in msg, msg


def test_tensor_engine_rejects_other_T():
    L = P.load()
    tb, nb = _lib._T_n(T2, N2)
    planes = P.make_planes_raw([(FAKE, 64, 16, 64, 10, 0, 0, 0)])
    for path in (_lib.TDCT_PATH_TENSOR, _lib.TDCT_PATH_TENSOR_PIPELINED):
        assert L.tdct_codec_error_batched(ctypes.addressof(planes), 1, tb, nb, FAKE, None, path,
                                          None) == _lib.TDCT_EUNSUPPORTED
        h = ctypes.c_void_p()
        assert L.tdct_plan_create(ctypes.addressof(planes), 1, tb, nb, path, ctypes.byref(h)) \
            == _lib.TDCT_EUNSUPPORTED
        assert not h.value


def test_forward_and_inverse_reject():
    L = P.load()
    tb, nb = _lib._T_n()
    assert L.tdct_forward(FAKE, 64, 16, 64, 0, tb, nb, None, None) == _lib.TDCT_EINVAL
    assert L.tdct_forward(FAKE, 64, 16, 64, 0, tb, nb, FAKE + 2, None) == _lib.TDCT_EINVAL
    assert L.tdct_zonal_inverse(FAKE, 16, 64, 0, tb, nb, 0, FAKE, 64, None) == _lib.TDCT_EINVAL
    assert L.tdct_zonal_inverse(None, 16, 64, 0, tb, nb, 5, FAKE, 64, None) == _lib.TDCT_EINVAL


def test_dct_codec_rejects():
    L = P.load()
    assert L.tdct_dct_codec_error(FAKE, 64, 16, 64, 0, 10, 3, None, None, 0, FAKE, None, None) \
        == _lib.TDCT_EINVAL  # not a tdct_precision
    assert L.tdct_dct_codec_error(FAKE, 128, 16, 64, 1, 10, _lib.TDCT_BF16X3, None, None, 0, FAKE,
                                  None, None) == _lib.TDCT_EUNSUPPORTED  # int16 plane
    assert L.tdct_dct_codec_error(FAKE, 64, 16, 64, 0, 99, 0, None, None, 0, FAKE, None, None) \
        == _lib.TDCT_EINVAL


def test_batched_rejects():
    L = P.load()
    tb, nb = _lib._T_n()
    good = (FAKE, 64, 16, 64, 10, 0, 0, 0)
    planes = P.make_planes_raw([good, (FAKE, 64, 16, 64, 70, 0, 0, 0)])
    rc = L.tdct_codec_error_batched(ctypes.addressof(planes), 2, tb, nb, FAKE, None, 0, None)
    assert rc == _lib.TDCT_EINVAL and "plane 1" in L.tdct_last_error().decode()
    planes = P.make_planes_raw([good])
    assert L.tdct_codec_error_batched(ctypes.addressof(planes), 0, tb, nb, FAKE, None, 0, None) \
        == _lib.TDCT_EINVAL
    assert L.tdct_codec_error_batched(ctypes.addressof(planes), 1, tb, nb, FAKE, None, 9, None) \
        == _lib.TDCT_EUNSUPPORTED
    assert L.tdct_codec_error_batched(ctypes.addressof(planes), 1, tb, nb, FAKE, None, -1, None) \
        == _lib.TDCT_EUNSUPPORTED
    h = ctypes.c_void_p()
    planes = P.make_planes_raw([(FAKE, 64, 16, 64, 10, 3, 0, 0)])
    assert L.tdct_plan_create(ctypes.addressof(planes), 1, tb, nb, 0, ctypes.byref(h)) \
        == _lib.TDCT_EINVAL
    assert not h.value


def test_errors_raise_in_binding():
    import torch

    img = torch.zeros((16, 64), dtype=torch.uint8)
    sse = torch.zeros(1, dtype=torch.int64)
    with pytest.raises(P.TdctError) as e:
        P.tdct_codec_error(img, 0, sse)
    assert e.value.code == _lib.TDCT_EINVAL


def test_named_transforms_agree_with_the_oracle_copies():
    """The library's table of named matrices and the oracle's, typed
    independently from §4.1 and Table 2, agree (LO enters scaled by 2)."""
    import numpy as np

    from oracle import matrices as M
    from paper_1808_02950_gb300 import transforms as tr

    want = {"T1": M.T1, "T2": M.T2, "RDCT": M.T_RDCT, "T6": M.T6, "T4": M.T4,
            "LOx2": 2 * M.T_LO}
    assert set(tr.NAMED) == set(want)
    for name, T in tr.NAMED.items():
        assert np.array_equal(np.array(T), want[name]), name
        assert tr.row_norms(T) == tuple(int(v) for v in np.einsum("ij,ij->i", want[name], want[name]))
    assert tr.T1 == tuple(tuple(r) for r in P.T1)


def test_host_buffer_batch_rejects_before_any_cuda_call():
    L = P.load()
    tb, nb = _lib._T_n()
    good = (FAKE, 64, 16, 64, 10, 0, 0, 0)
    planes = P.make_planes_raw([good, (FAKE, 64, 16, 64, 70, 0, 0, 0)])
    rc = L.tdct_codec_error_batched_host(ctypes.addressof(planes), 2, tb, nb, FAKE, None, 0, None)
    assert rc == _lib.TDCT_EINVAL and "plane 1" in L.tdct_last_error().decode()
    planes = P.make_planes_raw([good])
    assert L.tdct_codec_error_batched_host(ctypes.addressof(planes), 1, tb, nb, None, None, 0,
                                           None) == _lib.TDCT_EINVAL
    assert L.tdct_codec_error_batched_host(ctypes.addressof(planes), 0, tb, nb, FAKE, None, 0,
                                           None) == _lib.TDCT_EINVAL
    planes = P.make_planes_raw([(None, 64, 16, 64, 10, 0, 0, 0)])
    assert L.tdct_codec_error_batched_host(ctypes.addressof(planes), 1, tb, nb, FAKE, None, 0,
                                           None) == _lib.TDCT_EINVAL


def test_ssim_rejects_before_any_cuda_call():
    L = P.load()
    good = _lib.TdctSsimPlane(FAKE, 64, FAKE, 64, 16, 64)
    small = _lib.TdctSsimPlane(FAKE, 64, FAKE, 64, 10, 64)
    arr = (_lib.TdctSsimPlane * 2)(good, small)
    assert L.tdct_ssim_batched(ctypes.addressof(arr), 2, FAKE, None) == _lib.TDCT_EINVAL
    assert "plane 1" in L.tdct_last_error().decode()
    arr = (_lib.TdctSsimPlane * 1)(_lib.TdctSsimPlane(None, 64, FAKE, 64, 16, 64))
    assert L.tdct_ssim_batched(ctypes.addressof(arr), 1, FAKE, None) == _lib.TDCT_EINVAL
    arr = (_lib.TdctSsimPlane * 1)(_lib.TdctSsimPlane(FAKE, 63, FAKE, 64, 16, 64))
    assert L.tdct_ssim_batched(ctypes.addressof(arr), 1, FAKE, None) == _lib.TDCT_EINVAL
    arr = (_lib.TdctSsimPlane * 1)(good)
    assert L.tdct_ssim_batched(ctypes.addressof(arr), 1, FAKE + 4, None) == _lib.TDCT_EINVAL


def test_search_rejects_before_any_cuda_call():
    L = P.load()
    alph = (ctypes.c_int8 * 3)(0, 1, -1)
    order = (ctypes.c_int32 * 2)(0, 1)
    T = (ctypes.c_int8 * 64)()
    c = ctypes.c_int32()
    ok = lambda *a: L.tdct_search(*a)
    assert ok(1, alph, 3, order, 2, None, None, 0, 0, T, ctypes.byref(c), None) == _lib.TDCT_EINVAL
    assert ok(8, alph, 1, order, 2, None, None, 0, 0, T, ctypes.byref(c), None) == _lib.TDCT_EINVAL
    dup = (ctypes.c_int8 * 3)(0, 1, 1)
    assert ok(8, dup, 3, order, 2, None, None, 0, 0, T, ctypes.byref(c), None) == _lib.TDCT_EINVAL
    bad = (ctypes.c_int32 * 2)(0, 0)
    assert ok(8, alph, 3, bad, 2, None, None, 0, 0, T, ctypes.byref(c), None) == _lib.TDCT_EINVAL
    assert ok(8, alph, 3, order, 2, None, None, 0, 2, T, ctypes.byref(c), None) == _lib.TDCT_EINVAL
    wide = (ctypes.c_int8 * 3)(0, 17, -1)
    assert ok(8, wide, 3, order, 2, None, None, 0, 0, T, ctypes.byref(c), None) == _lib.TDCT_EINVAL
    big = (ctypes.c_int8 * 9)(*range(-4, 5))
    assert ok(16, big, 9, order, 2, None, None, 0, 0, T, ctypes.byref(c), None) \
        == _lib.TDCT_EUNSUPPORTED


def test_jam_codec_rejects_before_any_cuda_call():
    import numpy as np

    from oracle import matrices as M

    L = P.load()

    def call(T, B=16, r=10, n=None):
        Tb = (ctypes.c_int8 * (B * B))(*[int(v) for v in np.asarray(T).reshape(-1)])
        nn = n if n is not None else [int(v) for v in np.einsum("ij,ij->i", T, T)]
        nb = (ctypes.c_int32 * B)(*nn)
        return L.tdct_codec_error_jam(FAKE, 64, 16, 64, 0, B, Tb, nb, r, None, 0, FAKE, None, None)

    assert call(M.T16, r=0) == _lib.TDCT_EINVAL
    assert call(M.T16, r=257) == _lib.TDCT_EINVAL
    assert call(M.T1, B=8) == _lib.TDCT_EINVAL
    swapped = M.T16[[1, 0] + list(range(2, 16))]           # orthogonal, not the JAM matrix
    assert call(swapped) == _lib.TDCT_EUNSUPPORTED
    assert call(M.T16, n=[16] * 16) == _lib.TDCT_ENOTORTHO
