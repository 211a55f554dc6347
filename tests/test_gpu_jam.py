"""GPU parity of the 16x16 / 32x32 block codec with the JAM matrices of §6.2
(tdct_codec_error_jam) against the CPU oracle, bit for bit: SSE, PSNR and
reconstruction, u8 and int16 residual planes, ragged edges."""
import numpy as np
import pytest
import torch

import paper_1808_02950_gb300 as P
from oracle import codec as oc
from oracle import matrices as M

pytestmark = pytest.mark.gpu
DEV = "cuda"


def run(host, B, T, r):
    view = torch.from_numpy(host).to(DEV)
    recon = torch.full_like(view, 7)
    sse = torch.zeros(1, dtype=torch.int64, device=DEV)
    psnr = torch.zeros(1, dtype=torch.float64, device=DEV)
    P.tdct_codec_error_jam(view, B, T.tolist(), r, sse, recon=recon, psnr=psnr)
    torch.cuda.synchronize()
    return int(sse.item()), recon.cpu().numpy(), float(psnr.item())


@pytest.mark.parametrize("B,T", [(16, M.T16), (32, M.T32)])
@pytest.mark.parametrize("dtype", [np.uint8, np.int16])
@pytest.mark.parametrize("H,W", [(16, 16), (40, 70), (33, 97), (64, 128), (7, 5)])
def test_jam_codec_matches_oracle(B, T, dtype, H, W):
    rng = np.random.default_rng(B * 1000 + H * 10 + W + (dtype == np.int16))
    if dtype == np.uint8:
        host = rng.integers(0, 256, (H, W)).astype(np.uint8)
    else:
        host = rng.integers(-255, 256, (H, W)).astype(np.int16)
    # kept-extent classes 2, 2, 4, 6, 8, 12, 16, 16 (B = 16) or 24, 32, 32 (B = 32)
    for r in (1, 3, 10, 16, 28, 50, 136, 300 if B == 32 else 200, B * B // 2, B * B):
        sse, rec, psnr = run(host, B, T, r)
        want_sse, want_rec = oc.codec_plane_b(host, T, B, r)
        assert np.array_equal(rec, want_rec), f"B={B} r={r}"
        assert sse == want_sse
        if want_sse:
            assert psnr == pytest.approx(oc.psnr(want_sse, H * W), rel=1e-12)


@pytest.mark.parametrize("B,T", [(16, M.T16), (32, M.T32)])
def test_jam_codec_smooth_image_and_extremes(B, T):
    """A synthetic AR(1) image (the paper's image statistics) and extreme
    blocks (constants, checkerboards, sign patterns of the basis)."""
    from paper_1808_02950_gb300 import synth

    img = synth.ar1_images(1, 128, 256, 0.95, 11, "cpu")[0].numpy()
    for r in (3, 21, 100):
        sse, rec, _ = run(np.ascontiguousarray(img), B, T, r)
        want_sse, want_rec = oc.codec_plane_b(np.ascontiguousarray(img), T, B, r)
        assert sse == want_sse and np.array_equal(rec, want_rec)
    blocks = [np.zeros((B, B)), np.full((B, B), 255),
              (np.indices((B, B)).sum(0) % 2) * 255]
    for i in (0, 1, B // 2 - 1, B - 1):
        s = np.sign(np.outer(T[i], T[(3 * i + 1) % B]))
        blocks.append(np.where(s > 0, 255, 0))
    ext = np.ascontiguousarray(np.concatenate([b.astype(np.uint8) for b in blocks], axis=1))
    for r in (1, 5, 16, 136, B * B):
        sse, rec, _ = run(ext, B, T, r)
        want_sse, want_rec = oc.codec_plane_b(ext, T, B, r)
        assert sse == want_sse and np.array_equal(rec, want_rec)


@pytest.mark.parametrize("B,T", [(16, M.T16), (32, M.T32)])
@pytest.mark.parametrize("dtype", [np.uint8, np.int16])
def test_jam_codec_large_ragged_plane(B, T, dtype):
    """A plane with more blocks than one grid stride covers (each warp steps
    through several blocks and the ring wraps), ragged on both edges, as a
    16-byte aligned plane and as an unaligned pitched view."""
    rng = np.random.default_rng(B + (dtype == np.int16))
    H, W = 3000, 3100
    if dtype == np.uint8:
        host = rng.integers(0, 256, (H, W + 3)).astype(np.uint8)
    else:
        host = rng.integers(-255, 256, (H, W + 3)).astype(np.int16)
    for off in (0, 3):
        view = np.ascontiguousarray(host[:, off:off + W]) if off == 0 else host[:, off:off + W]
        for r in (16, 100):
            dev = torch.from_numpy(host).to(DEV)[:, off:off + W] if off else torch.from_numpy(view).to(DEV)
            recon = torch.full((H, W), 7, dtype=dev.dtype, device=DEV)
            sse = torch.zeros(1, dtype=torch.int64, device=DEV)
            P.tdct_codec_error_jam(dev, B, T.tolist(), r, sse, recon=recon)
            torch.cuda.synchronize()
            want_sse, want_rec = oc.codec_plane_b(np.ascontiguousarray(view), T, B, r)
            assert int(sse.item()) == want_sse, (off, r)
            assert np.array_equal(recon.cpu().numpy(), want_rec), (off, r)
