"""GPU parity of tdct_codec_error_batched_host: planes and results in host
memory, copies pipelined with the codec in chunks.  Every SSE, PSNR and
returned reconstruction is compared with the oracle bit for bit; tiny chunk
sizes force many chunks, so both staging buffers are reused several times."""
import numpy as np
import pytest
import torch

import paper_1808_02950_gb300 as P
from oracle import codec as oc
from oracle import matrices as M

pytestmark = pytest.mark.gpu


def host_planes(rng, shapes, pin):
    hosts, tensors = [], []
    for H, W, dt in shapes:
        if dt == np.uint8:
            h = rng.integers(0, 256, (H, W)).astype(np.uint8)
        else:
            h = rng.integers(-255, 256, (H, W)).astype(np.int16)
        t = torch.from_numpy(h.copy())
        tensors.append(t.pin_memory() if pin else t)
        hosts.append(h)
    return hosts, tensors


SHAPES = [(64, 128, np.uint8), (13, 11, np.uint8), (40, 72, np.int16), (8, 1024, np.uint8),
          (33, 65, np.uint8), (16, 32, np.int16), (256, 256, np.uint8), (7, 9, np.int16),
          (128, 80, np.uint8), (24, 1040, np.uint8)]


@pytest.mark.parametrize("pin", [True, False])
@pytest.mark.parametrize("chunk", [0, 1, 40000])
def test_host_batch_matches_oracle(pin, chunk):
    rng = np.random.default_rng(7 + chunk)
    hosts, tens = host_planes(rng, SHAPES, pin)
    rs = [int(v) for v in rng.choice([1, 3, 10, 16, 28, 45, 64], len(SHAPES))]
    recons = [torch.full_like(t, 9) for t in tens]
    recons = [r.pin_memory() if pin else r for r in recons]
    want_recon = [i % 3 != 1 for i in range(len(SHAPES))]  # some planes without reconstruction
    planes = P.make_planes(tens, rs, [recons[i] if want_recon[i] else None
                                      for i in range(len(SHAPES))])
    sse = torch.full((len(SHAPES),), -1, dtype=torch.int64)
    psnr = torch.zeros(len(SHAPES), dtype=torch.float64)
    if pin:
        sse, psnr = sse.pin_memory(), psnr.pin_memory()
    P.tdct_codec_error_batched_host(planes, sse, psnr, chunk_bytes=chunk)
    torch.cuda.synchronize()
    for i, (h, r) in enumerate(zip(hosts, rs)):
        ws, wr, _ = oc.codec_plane(h, M.T1, r)
        assert int(sse[i]) == ws, f"plane {i}"
        p = oc.psnr(ws, h.size)
        assert float(psnr[i]) == (pytest.approx(p, rel=1e-12) if np.isfinite(p) else p)
        if want_recon[i]:
            assert np.array_equal(recons[i].numpy(), wr), f"plane {i}"
        else:
            assert (recons[i].numpy() == 9).all()


def test_host_batch_images_large_and_generic_T():
    """64 pinned 512x512 images in 1 MiB chunks, T1 and T6: equal to the
    device-memory batched call and, sampled, to the oracle."""
    rng = np.random.default_rng(11)
    hosts, tens = host_planes(rng, [(512, 512, np.uint8)] * 64, pin=True)
    rs = [16] * 64
    for T in (None, M.T6):
        Tn = {} if T is None else dict(T=np.asarray(T).tolist(),
                                       n=tuple(int(v) for v in np.einsum("ij,ij->i", T, T)))
        sse_h = torch.zeros(64, dtype=torch.int64).pin_memory()
        P.tdct_codec_error_batched_host(P.make_planes(tens, rs), sse_h, chunk_bytes=1 << 20, **Tn)
        dev = [t.cuda() for t in tens]
        sse_d = torch.zeros(64, dtype=torch.int64, device="cuda")
        P.tdct_codec_error_batched(P.make_planes(dev, rs), sse_d, **Tn)
        torch.cuda.synchronize()
        assert torch.equal(sse_h, sse_d.cpu())
        for i in (0, 37, 63):
            assert int(sse_h[i]) == oc.codec_plane(hosts[i], M.T1 if T is None else T, 16,
                                                   want_recon=False)[0]


def test_shutdown_releases_streams_and_library_stays_usable():
    """tdct_shutdown destroys the library-owned transfer streams; a later
    host-buffer call re-creates them and still matches the oracle, and a
    second shutdown is harmless."""
    rng = np.random.default_rng(21)
    hosts, tens = host_planes(rng, SHAPES[:4], pin=True)
    rs = [10, 16, 8, 28]
    for _ in range(2):
        sse = torch.full((4,), -1, dtype=torch.int64).pin_memory()
        P.tdct_codec_error_batched_host(P.make_planes(tens, rs), sse)
        torch.cuda.synchronize()
        for i, (h, r) in enumerate(zip(hosts, rs)):
            assert int(sse[i]) == oc.codec_plane(h, M.T1, r, want_recon=False)[0]
        P.tdct_shutdown()
    P.tdct_shutdown()
