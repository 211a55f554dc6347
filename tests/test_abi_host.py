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


def test_other_orthogonal_T_is_unsupported_not_wrong():
    T2 = [[1, 1, 1, 1, 1, 1, 1, 1], [2, 1, 2, 0, 0, -2, -1, -2], [2, 1, -1, -2, -2, -1, 1, 2],
          [2, 0, -2, -1, 1, 2, 0, -2], [1, -1, -1, 1, 1, -1, -1, 1], [1, -2, 0, 2, -2, 0, 2, -1],
          [1, -2, 2, -1, -1, 2, -2, 1], [0, -2, 1, -2, 2, -1, 2, 0]]
    rc, msg = _call_codec(T=T2, n=(8, 18, 20, 18, 8, 18, 20, 18))
    assert rc == _lib.TDCT_EUNSUPPORTED, msg


def test_forward_and_inverse_reject():
    L = P.load()
    tb, nb = _lib._T_n()
    assert L.tdct_forward(FAKE, 64, 16, 64, 0, tb, nb, None, None) == _lib.TDCT_EINVAL
    assert L.tdct_forward(FAKE, 64, 16, 64, 0, tb, nb, FAKE + 2, None) == _lib.TDCT_EINVAL
    assert L.tdct_zonal_inverse(FAKE, 16, 64, 0, tb, nb, 0, FAKE, 64, None) == _lib.TDCT_EINVAL
    assert L.tdct_zonal_inverse(None, 16, 64, 0, tb, nb, 5, FAKE, 64, None) == _lib.TDCT_EINVAL


def test_dct_codec_rejects():
    L = P.load()
    assert L.tdct_dct_codec_error(FAKE, 64, 16, 64, 0, 10, 2, None, None, 0, FAKE, None, None) \
        == _lib.TDCT_EINVAL
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
