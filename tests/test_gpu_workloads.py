"""The full-size workloads on the GPU against the oracle.

* single_512        -- covered in test_gpu_codec (all outputs).
* batch_1024x1024   -- every image's SSE, sampled reconstructions.
* sweep_64x512      -- SSE for all 64 images x r = 1..64 (T1); exact-DCT FP32
                       PSNR within 0.01 dB of FP64 on a sample.
* ragged_2000       -- every plane's SSE on the GPU; oracle on a sample.
* video_600x1080p   -- int16 residual planes; oracle on sampled frames.
The oracle runs in a thread pool (its C calls release the GIL).
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import paper_1808_02950_gb300 as P
from oracle import codec as oc
from oracle import matrices as M
from paper_1808_02950_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = "cuda"


def _pool_map(fn, items):
    with ThreadPoolExecutor(16) as ex:
        return list(ex.map(fn, items))


def _run_batch(views, rs, with_recon=False):
    recons = [torch.empty_like(v) for v in views] if with_recon else None
    planes = P.make_planes(views, rs, recons)
    sse = torch.zeros(len(views), dtype=torch.int64, device=DEV)
    psnr = torch.zeros(len(views), dtype=torch.float64, device=DEV)
    plan = P.tdct_plan_create(planes)
    plan.launch(sse, psnr)
    torch.cuda.synchronize()
    plan.close()
    return sse.cpu().numpy(), psnr.cpu().numpy(), recons


def test_batch_1024x1024():
    imgs, r = synth.batch_1024x1024(DEV)
    views = [imgs[i] for i in range(imgs.shape[0])]
    sse, psnr, recons = _run_batch(views, [r] * len(views), with_recon=True)
    host = imgs.cpu().numpy()
    sample = set(range(0, 1024, 97)) | {1023}

    def oracle(i):
        s, rec, _ = oc.codec_plane(host[i], M.T1, r, want_recon=i in sample)
        return s, rec

    res = _pool_map(oracle, range(1024))
    for i, (s, rec) in enumerate(res):
        assert sse[i] == s, f"image {i}"
        assert psnr[i] == pytest.approx(oc.psnr(s, 1 << 20), rel=1e-12)
        if i in sample:
            assert np.array_equal(recons[i].cpu().numpy(), rec)


def test_sweep_64x512_all_r():
    imgs, _ = synth.sweep_64x512(DEV)
    n = imgs.shape[0]
    views = [imgs[i] for i in range(n) for _ in range(64)]
    rs = [r for _ in range(n) for r in range(1, 65)]
    sse, _, _ = _run_batch(views, rs)
    host = imgs.cpu().numpy()
    want = _pool_map(lambda ir: oc.codec_plane(host[ir[0]], M.T1, ir[1], want_recon=False)[0],
                     [(i, r) for i in range(n) for r in range(1, 65)])
    assert [int(v) for v in sse] == want
    # exact DCT, FP32 on the GPU vs FP64 oracle, on a sample of (image, r)
    for i in (0, 17, 40, 63):
        for r in (1, 3, 10, 21, 36, 50, 63):
            s = torch.zeros(1, dtype=torch.int64, device=DEV)
            p = torch.zeros(1, dtype=torch.float64, device=DEV)
            P.tdct_dct_codec_error(imgs[i], r, s, precision=P.TDCT_FP32, psnr=p)
            torch.cuda.synchronize()
            s64 = oc.dct_codec_plane(host[i], r, want_recon=False)[0]
            assert abs(float(p.item()) - oc.psnr(s64, 512 * 512)) <= 0.01


def test_ragged_2000():
    buf, offs, H, W, r = synth.ragged_2000(DEV)
    views = [buf[int(offs[i]): int(offs[i]) + int(H[i] * W[i])].view(int(H[i]), int(W[i]))
             for i in range(len(offs))]
    sse, psnr, _ = _run_batch(views, [int(v) for v in r])
    rng = np.random.default_rng(0)
    idx = sorted(set(rng.choice(len(offs), 80, replace=False).tolist()) | {0, len(offs) - 1})
    want = _pool_map(lambda i: oc.codec_plane(views[i].cpu().numpy(), M.T1, int(r[i]),
                                              want_recon=False)[0], idx)
    for i, w in zip(idx, want):
        assert sse[i] == w, f"plane {i} ({H[i]}x{W[i]}, r={r[i]})"
        assert psnr[i] == pytest.approx(oc.psnr(w, int(H[i] * W[i])), rel=1e-12)
    assert np.all(sse > 0)


def test_video_600x1080p():
    Y, U, V = synth.video_600x1080p(DEV)
    views, rs = [], []
    for t in range(Y.shape[0]):
        views += [Y[t], U[t], V[t]]
        rs += [16, 8, 8]
    sse, _, recons = _run_batch(views, rs, with_recon=True)
    frames = [0, 1, 100, 311, 598]
    idx = [3 * t + c for t in frames for c in range(3)]

    def oracle(i):
        return oc.codec_plane(views[i].cpu().numpy(), M.T1, rs[i])

    for i, (s, rec, _) in zip(idx, _pool_map(oracle, idx)):
        assert sse[i] == s, f"plane {i}"
        assert np.array_equal(recons[i].cpu().numpy(), rec)
