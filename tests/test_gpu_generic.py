"""GPU parity of the generic-T kernels (any orthogonal integer T) against the
CPU oracle, bit for bit.

The matrices are the other orthogonal approximations of the paper: T2 of
§4.1 and the orthogonal literature matrices of Table 2 (RDCT, T6, T4, and
LO scaled by 2 to integer entries, which leaves C_hat = S T unchanged).
The oracle computes the codec of Eq. (1)-(2) for any orthogonal T with exact
integer arithmetic; the library must reproduce its coefficients,
reconstructions, SSE and PSNR.
"""
import numpy as np
import pytest
import torch

import paper_1808_02950_gb300 as P
from oracle import codec as oc
from oracle import matrices as M

pytestmark = pytest.mark.gpu
DEV = "cuda"

MATS = {
    "T2": M.T2,
    "RDCT": M.T_RDCT,
    "T6": M.T6,
    "T4": M.T4,
    "LOx2": (2 * M.T_LO).astype(np.int64),
}
R_LIST = [1, 2, 3, 5, 6, 8, 10, 13, 16, 21, 28, 32, 36, 45, 55, 63, 64]


def Tn(T):
    T = np.asarray(T, dtype=np.int64)
    return T.tolist(), tuple(int(v) for v in np.einsum("ij,ij->i", T, T))


def rand_plane(rng, H, W, dtype, pitch_extra=0):
    if dtype == np.uint8:
        host = rng.integers(0, 256, (H, W)).astype(np.uint8)
    else:
        host = rng.integers(-255, 256, (H, W)).astype(np.int16)
    tdt = torch.uint8 if dtype == np.uint8 else torch.int16
    buf = torch.zeros((H, W + pitch_extra), dtype=tdt, device=DEV)
    view = buf[:, :W]
    view.copy_(torch.from_numpy(host).to(DEV))
    return host, view


def run(view, r, T, n):
    recon = torch.full_like(view, 77)
    sse = torch.zeros(1, dtype=torch.int64, device=DEV)
    psnr = torch.zeros(1, dtype=torch.float64, device=DEV)
    P.tdct_codec_error(view, r, sse, recon=recon, psnr=psnr, T=T, n=n)
    torch.cuda.synchronize()
    return int(sse.item()), recon.cpu().numpy(), float(psnr.item())


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("dtype", [np.uint8, np.int16])
@pytest.mark.parametrize("H,W", [(8, 8), (13, 11), (40, 136), (24, 1032)])
def test_generic_codec_matches_oracle(name, dtype, H, W):
    T, n = Tn(MATS[name])
    seed = sum(map(ord, name)) * 100003 + H * 1009 + W * 2 + (dtype == np.int16)
    rng = np.random.default_rng(seed)
    host, view = rand_plane(rng, H, W, dtype, pitch_extra=3 if dtype == np.uint8 else 0)
    for r in R_LIST[:: 2 if H * W > 4096 else 1]:
        sse, rec, psnr = run(view, r, T, n)
        want_sse, want_rec, _ = oc.codec_plane(host, MATS[name], r)
        assert np.array_equal(rec, want_rec), f"{name} recon differs at r={r}"
        assert sse == want_sse, f"{name} SSE differs at r={r}"
        if want_sse:
            assert psnr == pytest.approx(oc.psnr(want_sse, H * W), rel=1e-12)
        else:
            assert psnr == float("inf")


def _sign_blocks(T):
    """Extreme u8 blocks for T: constants, checkerboards and the sign patterns
    of the outer products of T's rows (they maximise |Z| and |N|)."""
    T = np.asarray(T)
    blocks = [np.zeros((8, 8)), np.full((8, 8), 255)]
    cb = (np.indices((8, 8)).sum(0) % 2) * 255
    blocks += [cb, 255 - cb]
    for i in range(8):
        for j in range(8):
            s = np.sign(np.outer(T[i], T[j]))
            blocks.append(np.where(s > 0, 255, 0))
            blocks.append(np.where(s >= 0, 255, 0))
    return np.ascontiguousarray(np.concatenate([b.astype(np.uint8) for b in blocks], axis=1))


@pytest.mark.parametrize("name", list(MATS))
def test_generic_extreme_blocks(name):
    T, n = Tn(MATS[name])
    host = _sign_blocks(MATS[name])
    view = torch.from_numpy(host).to(DEV)
    res_host = (host.astype(np.int16) * 2 - 255).astype(np.int16)  # +-255 residuals
    res = torch.from_numpy(res_host).to(DEV)
    for r in (1, 4, 15, 36, 64):
        sse, rec, _ = run(view, r, T, n)
        want_sse, want_rec, _ = oc.codec_plane(host, MATS[name], r)
        assert np.array_equal(rec, want_rec) and sse == want_sse
        sse, rec, _ = run(res, r, T, n)
        want_sse, want_rec, _ = oc.codec_plane(res_host, MATS[name], r)
        assert np.array_equal(rec, want_rec) and sse == want_sse


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("dtype", [np.uint8, np.int16])
def test_generic_forward_and_zonal_inverse(name, dtype):
    T, n = Tn(MATS[name])
    H, W = 37, 203
    rng = np.random.default_rng(len(name) * 7 + (dtype == np.int16))
    host, view = rand_plane(rng, H, W, dtype)
    coef = torch.zeros(((H + 7) // 8, (W + 7) // 8, 8, 8), dtype=torch.int32, device=DEV)
    P.tdct_forward(view, coef, T=T, n=n)
    out = torch.zeros_like(view)
    for r in (1, 6, 16, 37, 64):
        P.tdct_zonal_inverse(coef, r, out, T=T, n=n)
        torch.cuda.synchronize()
        _, want_rec, want_coef = oc.codec_plane(host, MATS[name], r, want_coef=True)
        assert np.array_equal(coef.cpu().numpy().astype(np.int64), want_coef)
        assert np.array_equal(out.cpu().numpy(), want_rec)
        inv = oc.zonal_inverse_plane(want_coef, H, W, MATS[name], r, dtype=dtype)
        assert np.array_equal(inv, want_rec)


@pytest.mark.parametrize("name", ["T2", "T6", "LOx2"])
def test_generic_batched_plan_and_noalloc(name):
    """Ragged mixed batch (u8 and int16, several r) through the batched call,
    a plan (autotune skipped: one engine) and the allocation-free call."""
    T, n = Tn(MATS[name])
    rng = np.random.default_rng(99)
    shapes = [(64, 128, np.uint8, 10), (13, 11, np.uint8, 3), (40, 72, np.int16, 16),
              (8, 1024, np.uint8, 64), (33, 65, np.uint8, 10), (16, 32, np.int16, 1)]
    hosts, views, rs = [], [], []
    for H, W, dt, r in shapes:
        h, v = rand_plane(rng, H, W, dt)
        hosts.append(h)
        views.append(v)
        rs.append(r)
    recons = [torch.full_like(v, 5) for v in views]
    planes = P.make_planes(views, rs, recons)
    want = [oc.codec_plane(h, MATS[name], r) for h, r in zip(hosts, rs)]

    def check(sse, psnr):
        torch.cuda.synchronize()
        for i, (ws, wr, _) in enumerate(want):
            assert int(sse[i]) == ws, f"plane {i}"
            assert np.array_equal(recons[i].cpu().numpy(), wr), f"plane {i}"
            p = oc.psnr(ws, hosts[i].size)
            assert float(psnr[i]) == (pytest.approx(p, rel=1e-12) if np.isfinite(p) else p)
            recons[i].fill_(5)

    sse = torch.zeros(len(views), dtype=torch.int64, device=DEV)
    psnr = torch.zeros(len(views), dtype=torch.float64, device=DEV)
    P.tdct_codec_error_batched(planes, sse, psnr, T=T, n=n)
    check(sse, psnr)
    plan = P.tdct_plan_create(planes, T=T, n=n)
    assert plan.config()["path"] == "butterfly"
    for _ in range(2):
        sse.fill_(-1)
        plan.launch(sse, psnr)
        check(sse, psnr)
    plan.close()
    P.tdct_codec_error_batched_noalloc(planes, sse, psnr, T=T, n=n)
    check(sse, psnr)


def test_generic_large_plane_sampled_rows():
    """A 1024 x 1024 u8 image with T6 at r = 10: SSE of the whole plane and
    the reconstruction of a sample of block rows against the oracle."""
    rng = np.random.default_rng(6)
    host, view = rand_plane(rng, 1024, 1024, np.uint8)
    T, n = Tn(M.T6)
    sse, rec, _ = run(view, 10, T, n)
    want_sse, _, _ = oc.codec_plane(host, M.T6, 10, want_recon=False)
    assert sse == want_sse
    for by in rng.choice(128, 6, replace=False):
        band = np.ascontiguousarray(host[8 * by: 8 * by + 8])
        _, want_band, _ = oc.codec_plane(band, M.T6, 10)
        assert np.array_equal(rec[8 * by: 8 * by + 8], want_band)
