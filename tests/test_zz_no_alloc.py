"""tdct_codec_error_batched_noalloc against tdct_codec_error_batched.

The allocation-free entry point serves callers that may not allocate device
memory (their allocator owns the device, or allocation is forbidden once a
real-time pipeline runs).  It keeps the ragged batch's block-offset table in
a fixed array of the library instead.  Two calls in a row, on two different
batches, must give exactly the SSE, PSNR and reconstructions of the
allocating entry point (the integer path is bit-exact, so the tolerance is
zero; PSNR is compared to 1e-12 relative).  The file name sorts last so a
run that stops at the first failure has run every other test already.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1808_02950_gb300 as P
from paper_1808_02950_gb300 import _lib

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _batch(seed):
    rng = np.random.default_rng(seed)
    specs = [(64, 64, 4, torch.uint8), (72, 136, 8, torch.uint8), (13, 11, 16, torch.int16),
             (40, 520, 16, torch.uint8), (8, 8, 64, torch.int16), (33, 65, 32, torch.uint8),
             (16, 1032, 4, torch.int16), (24, 24, int(rng.integers(1, 65)), torch.uint8)]
    views, rs = [], []
    for H, W, r, dt in specs:
        if dt == torch.uint8:
            host = rng.integers(0, 256, (H, W)).astype(np.uint8)
        else:
            host = rng.integers(-255, 256, (H, W)).astype(np.int16)
        views.append(torch.from_numpy(host).to(DEV))
        rs.append(r)
    return views, rs


def _run(fn, views, rs):
    recons = [torch.full_like(v, 3) for v in views]
    planes = P.make_planes(views, rs, recons)
    sse = torch.full((len(views),), -1, dtype=torch.int64, device=DEV)
    psnr = torch.zeros(len(views), dtype=torch.float64, device=DEV)
    fn(planes, sse, psnr)
    torch.cuda.synchronize()
    return sse.cpu().numpy(), psnr.cpu().numpy(), [r.cpu().numpy() for r in recons]


def test_noalloc_matches_allocating_entry_point_twice():
    for seed in (1, 2):  # two calls in a row, different batches
        views, rs = _batch(seed)
        want = _run(P.tdct_codec_error_batched, views, rs)
        got = _run(P.tdct_codec_error_batched_noalloc, views, rs)
        assert np.array_equal(got[0], want[0])
        np.testing.assert_allclose(got[1], want[1], rtol=1e-12)
        for a, b in zip(got[2], want[2]):
            assert np.array_equal(a, b)


def test_noalloc_rejects_more_planes_than_its_table():
    L = P.load()
    tb, nb = _lib._T_n()
    img = torch.zeros((8, 8), dtype=torch.uint8, device=DEV)
    n = _lib.NOALLOC_MAX_PLANES + 1
    planes = P.make_planes_raw([(img.data_ptr(), 8, 8, 8, 10, 0, 0, 0)] * n)
    sse = torch.zeros(n, dtype=torch.int64, device=DEV)
    rc = L.tdct_codec_error_batched_noalloc(ctypes.addressof(planes), n, tb, nb,
                                            sse.data_ptr(), None, None)
    assert rc == _lib.TDCT_EINVAL
    assert "fixed table" in L.tdct_last_error().decode()
