"""tdct_sweep_batched / tdct_dct_sweep_batched (the zonal sweep of §6.1 from
one read of each plane) against the oracle.

T1: every (plane, r) SSE equals the oracle's codec at that r, bit for bit,
on planes of ragged sizes (edge blocks, units cut by the plane's width),
pitched and unaligned planes, the extreme blocks, and the whole
sweep_64x512 workload (64 images x 64 r).  Exact DCT (FP32): every (plane, r)
PSNR within 0.01 dB of the FP64 oracle.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import paper_1808_02950_gb300 as P
from oracle import codec as oc
from oracle import matrices as M
from paper_1808_02950_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _pool_map(fn, items):
    with ThreadPoolExecutor(16) as ex:
        return list(ex.map(fn, items))


def _oracle_sse(host, dct=False):
    """[64] SSE of the oracle codec for r = 1..64."""
    f = (lambda r: oc.dct_codec_plane(host, r, want_recon=False)[0]) if dct else \
        (lambda r: oc.codec_plane(host, M.T1, r, want_recon=False)[0])
    return np.array([f(r) for r in range(1, 65)], dtype=np.int64)


def _sweep(views, dct=False):
    sse = torch.full((64 * len(views),), -1, dtype=torch.int64, device=DEV)
    psnr = torch.zeros(64 * len(views), dtype=torch.float64, device=DEV)
    if dct:
        P.tdct_dct_sweep_batched(views, sse, psnr)
    else:
        P.tdct_sweep_batched(views, sse, psnr)
    torch.cuda.synchronize()
    return sse.cpu().numpy().reshape(-1, 64), psnr.cpu().numpy().reshape(-1, 64)


SIZES = [(8, 8), (16, 256), (24, 264), (13, 11), (9, 300), (64, 520), (40, 7), (72, 1032),
         (1, 1), (33, 65)]


def test_sweep_t1_ragged_planes_all_r():
    rng = np.random.default_rng(3)
    hosts = [rng.integers(0, 256, s).astype(np.uint8) for s in SIZES]
    views = [torch.from_numpy(h).to(DEV) for h in hosts]
    sse, psnr = _sweep(views)
    want = _pool_map(_oracle_sse, hosts)
    for i, (h, w) in enumerate(zip(hosts, want)):
        assert np.array_equal(sse[i], w), (i, h.shape)
        for r in (1, 16, 64):
            p = oc.psnr(int(w[r - 1]), h.size)
            assert psnr[i, r - 1] == (pytest.approx(p, rel=1e-12) if np.isfinite(p) else p)


@pytest.mark.parametrize("offset,extra", [(0, 0), (3, 5), (8, 8)])
def test_sweep_t1_pitched_and_unaligned(offset, extra):
    rng = np.random.default_rng(offset + 7)
    H, W = 40, 300
    big = torch.from_numpy(rng.integers(0, 256, (H, W + offset + extra)).astype(np.uint8)).to(DEV)
    view = big[:, offset:offset + W]
    sse, _ = _sweep([view])
    assert np.array_equal(sse[0], _oracle_sse(view.cpu().numpy()))


def test_sweep_t1_extreme_blocks():
    """Constants, checkerboards and the sign patterns of T1's outer products
    (the largest coefficients and inverse magnitudes)."""
    plane = synth.adversarial_blocks(DEV)
    sse, _ = _sweep([plane])
    assert np.array_equal(sse[0], _oracle_sse(plane.cpu().numpy()))
    assert sse[0, 63] == 0  # r = 64 is lossless


def test_sweep_t1_equals_codec_per_r_on_gpu():
    """Entry r of the sweep equals the fused codec run with retention r."""
    img, _ = synth.single_512(DEV)
    sse, _ = _sweep([img])
    planes = P.make_planes([img] * 64, list(range(1, 65)))
    ref = torch.zeros(64, dtype=torch.int64, device=DEV)
    P.tdct_codec_error_batched(planes, ref)
    torch.cuda.synchronize()
    assert np.array_equal(sse[0], ref.cpu().numpy())


@pytest.mark.slow
def test_sweep_64x512_every_image_and_r():
    """The sweep_64x512 workload: all 4096 (image, r) SSEs bit-exact."""
    imgs, _ = synth.sweep_64x512(DEV)
    sse, _ = _sweep([imgs[i] for i in range(64)])
    host = imgs.cpu().numpy()
    want = _pool_map(_oracle_sse, [host[i] for i in range(64)])
    for i in range(64):
        assert np.array_equal(sse[i], want[i]), i


def test_dct_sweep_within_tolerance():
    """FP32 exact-DCT sweep: every (plane, r) PSNR within 0.01 dB of FP64."""
    rng = np.random.default_rng(5)
    imgs, _ = synth.sweep_64x512(DEV, n=4)
    views = [imgs[i] for i in range(4)] + [
        torch.from_numpy(rng.integers(0, 256, s).astype(np.uint8)).to(DEV) for s in SIZES[:6]]
    _, psnr = _sweep(views, dct=True)
    hosts = [v.cpu().numpy() for v in views]
    want = _pool_map(lambda h: _oracle_sse(h, dct=True), hosts)
    for i, (h, w) in enumerate(zip(hosts, want)):
        for r in range(1, 65):
            p64 = oc.psnr(int(w[r - 1]), h.size)
            if np.isfinite(p64):
                assert abs(psnr[i, r - 1] - p64) <= 0.01, (i, r, psnr[i, r - 1], p64)
            else:
                assert psnr[i, r - 1] > 60.0 or not np.isfinite(psnr[i, r - 1]), (i, r)


def test_sweep_rejects_what_it_does_not_implement():
    img = torch.zeros((16, 16), dtype=torch.int16, device=DEV)
    sse = torch.zeros(64, dtype=torch.int64, device=DEV)
    with pytest.raises(P.TdctError) as e:
        P.tdct_sweep_batched([img], sse)
    assert e.value.code == 7  # TDCT_EUNSUPPORTED
    u8 = torch.zeros((16, 16), dtype=torch.uint8, device=DEV)
    with pytest.raises(P.TdctError) as e:
        P.tdct_sweep_batched([u8], sse, T=M.T2.tolist(), n=(8, 18, 20, 18, 8, 18, 20, 18))
    assert e.value.code == 7
    with pytest.raises(P.TdctError) as e:
        P.tdct_dct_sweep_batched([u8], sse, precision=P.TDCT_BF16)
    assert e.value.code == 7
