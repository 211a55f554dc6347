"""GPU parity of the CUDA library against the CPU oracle (bit-exact).

Every test calls the C ABI through the thin binding on device tensors and
compares with ``oracle/`` on the same bytes: coefficients, reconstruction
and SSE must be identical; the exact-DCT path must be within the stated
tolerances of the FP64 oracle.
"""
import numpy as np
import pytest
import torch

import paper_1808_02950_gb300 as P
from oracle import codec as oc
from oracle import matrices as M
from paper_1808_02950_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda"
R_LIST = [1, 2, 3, 4, 5, 6, 8, 9, 10, 15, 16, 17, 21, 28, 31, 32, 33, 36, 45, 50, 55, 63, 64]


def rand_plane(rng, H, W, dtype, pitch_extra=0, offset=0):
    """Random plane as a (possibly strided / offset) view of a larger buffer."""
    if dtype == np.uint8:
        host = rng.integers(0, 256, (H, W)).astype(np.uint8)
    else:
        host = rng.integers(-255, 256, (H, W)).astype(np.int16)
    tdt = torch.uint8 if dtype == np.uint8 else torch.int16
    Wp = W + pitch_extra
    buf = torch.zeros(H * Wp + offset + 64, dtype=tdt, device=DEV)
    view = buf[offset: offset + H * Wp].view(H, Wp)[:, :W]
    view.copy_(torch.from_numpy(host).to(DEV))
    return host, view


def run_codec(view, r, want_recon=True):
    recon = torch.full_like(view, 77) if want_recon else None
    sse = torch.zeros(1, dtype=torch.int64, device=DEV)
    psnr = torch.zeros(1, dtype=torch.float64, device=DEV)
    P.tdct_codec_error(view, r, sse, recon=recon, psnr=psnr)
    torch.cuda.synchronize()
    return int(sse.item()), (recon.cpu().numpy() if recon is not None else None), float(psnr.item())


SIZES = [(8, 8), (8, 16), (16, 8), (24, 40), (13, 11), (1, 1), (7, 9), (64, 520), (40, 1032),
         (9, 1025)]


@pytest.mark.parametrize("dtype", [np.uint8, np.int16])
@pytest.mark.parametrize("H,W", SIZES)
def test_codec_small_planes(H, W, dtype):
    rng = np.random.default_rng(H * 1000 + W + (7 if dtype == np.int16 else 0))
    host, view = rand_plane(rng, H, W, dtype)
    for r in R_LIST[:: 2 if H * W > 4096 else 1]:
        sse, rec, psnr = run_codec(view, r)
        want_sse, want_rec, _ = oc.codec_plane(host, M.T1, r)
        assert np.array_equal(rec, want_rec), f"recon differs at r={r}"
        assert sse == want_sse
        assert psnr == pytest.approx(oc.psnr(want_sse, H * W), rel=1e-12) or (
            want_sse == 0 and psnr == float("inf"))


@pytest.mark.parametrize("dtype", [np.uint8, np.int16])
@pytest.mark.parametrize("pitch_extra,offset", [(8, 0), (3, 0), (0, 1), (5, 3), (16, 8)])
def test_codec_strided_and_unaligned(pitch_extra, offset, dtype):
    rng = np.random.default_rng(100 + pitch_extra * 10 + offset)
    host, view = rand_plane(rng, 40, 136, dtype, pitch_extra, offset)
    for r in (1, 10, 16, 64):
        sse, rec, _ = run_codec(view, r)
        want_sse, want_rec, _ = oc.codec_plane(host, M.T1, r)
        assert np.array_equal(rec, want_rec) and sse == want_sse


def test_codec_sse_only():
    rng = np.random.default_rng(5)
    host, view = rand_plane(rng, 64, 1040, np.uint8)
    for r in (3, 16):
        sse, _, _ = run_codec(view, r, want_recon=False)
        assert sse == oc.codec_plane(host, M.T1, r, want_recon=False)[0]


@pytest.mark.parametrize("r", [1, 4, 10, 16, 32, 64])
def test_adversarial_blocks(r):
    blocks = synth.adversarial_blocks(DEV)
    host = blocks.cpu().numpy()
    sse, rec, _ = run_codec(blocks, r)
    want_sse, want_rec, _ = oc.codec_plane(host, M.T1, r)
    assert np.array_equal(rec, want_rec) and sse == want_sse
    # the same sign patterns as int16 residuals at +-255
    res = (blocks.to(torch.int16) * 2 - 255).contiguous()
    sse, rec, _ = run_codec(res, r)
    want_sse, want_rec, _ = oc.codec_plane(res.cpu().numpy(), M.T1, r)
    assert np.array_equal(rec, want_rec) and sse == want_sse


@pytest.mark.parametrize("dtype", [np.uint8, np.int16])
def test_forward_cosimulation_100k_vectors(dtype):
    """100,000 random 8-point vectors through the row and column butterflies
    (12,500 blocks), as the paper's FPGA co-simulation (§5.2) does."""
    rng = np.random.default_rng(2112)
    host, view = rand_plane(rng, 8 * 125, 8 * 100, dtype)
    coef = torch.zeros((125, 100, 8, 8), dtype=torch.int32, device=DEV)
    P.tdct_forward(view, coef)
    torch.cuda.synchronize()
    _, _, want = oc.codec_plane(host, M.T1, 64, want_recon=False, want_coef=True)
    assert np.array_equal(coef.cpu().numpy().astype(np.int64), want)


@pytest.mark.parametrize("H,W", [(8, 8), (13, 11), (40, 520)])
@pytest.mark.parametrize("dtype", [np.uint8, np.int16])
def test_forward_and_zonal_inverse(H, W, dtype):
    rng = np.random.default_rng(H + W)
    host, view = rand_plane(rng, H, W, dtype)
    nby, nbx = (H + 7) // 8, (W + 7) // 8
    coef = torch.zeros((nby, nbx, 8, 8), dtype=torch.int32, device=DEV)
    P.tdct_forward(view, coef)
    out = torch.zeros_like(view)
    for r in (1, 6, 16, 37, 64):
        P.tdct_zonal_inverse(coef, r, out)
        torch.cuda.synchronize()
        _, want_rec, want_coef = oc.codec_plane(host, M.T1, r, want_coef=True)
        assert np.array_equal(coef.cpu().numpy().astype(np.int64), want_coef)
        assert np.array_equal(out.cpu().numpy(), want_rec)


def test_single_512_full():
    """The one-image workload (512x512, rho 0.95, r = 10), bit-exact."""
    img, r = synth.single_512(DEV)
    host = img.cpu().numpy()
    sse, rec, psnr = run_codec(img, r)
    want_sse, want_rec, _ = oc.codec_plane(host, M.T1, r)
    assert np.array_equal(rec, want_rec) and sse == want_sse
    assert psnr == pytest.approx(oc.psnr(want_sse, host.size), rel=1e-12)


def _batch(rng):
    specs = [(64, 64, 4, np.uint8), (72, 136, 8, np.uint8), (13, 11, 16, np.int16),
             (40, 520, 16, np.uint8), (8, 8, 64, np.int16), (33, 65, 32, np.uint8),
             (16, 1032, 4, np.int16), (24, 24, 16, np.uint8)]
    hosts, views, recons, rs = [], [], [], []
    for H, W, r, dt in specs:
        h, v = rand_plane(rng, H, W, dt)
        hosts.append(h)
        views.append(v)
        recons.append(torch.zeros_like(v))
        rs.append(r)
    return hosts, views, recons, rs


def test_batched_matches_oracle():
    rng = np.random.default_rng(77)
    hosts, views, recons, rs = _batch(rng)
    planes = P.make_planes(views, rs, recons)
    sse = torch.zeros(len(views), dtype=torch.int64, device=DEV)
    psnr = torch.zeros(len(views), dtype=torch.float64, device=DEV)
    P.tdct_codec_error_batched(planes, sse, psnr)
    torch.cuda.synchronize()
    for i, h in enumerate(hosts):
        want_sse, want_rec, _ = oc.codec_plane(h, M.T1, rs[i])
        assert int(sse[i]) == want_sse
        assert np.array_equal(recons[i].cpu().numpy(), want_rec)
        assert float(psnr[i]) == pytest.approx(oc.psnr(want_sse, h.size), rel=1e-12)


def test_plan_graph_replay():
    rng = np.random.default_rng(78)
    hosts, views, recons, rs = _batch(rng)
    planes = P.make_planes(views, rs, recons)
    plan = P.tdct_plan_create(planes)
    assert plan.kernel_count() >= 2
    want = [oc.codec_plane(h, M.T1, rs[i])[0] for i, h in enumerate(hosts)]
    for rep in range(3):
        sse = torch.full((len(views),), -1, dtype=torch.int64, device=DEV)
        plan.launch(sse)
        torch.cuda.synchronize()
        assert [int(v) for v in sse.cpu()] == want
    plan.close()


def _dct_rel_err(got, want):
    """Per plane: max |Y_gpu - Y_64| / max |Y_64| (a zero denominator counts as 1)."""
    den = np.abs(want).max()
    return np.abs(got - want).max() / (den if den > 0 else 1.0)


@pytest.mark.parametrize("dtype", [np.uint8, np.int16])
def test_dct_fp32_within_tolerance(dtype):
    rng = np.random.default_rng(300)
    host, view = rand_plane(rng, 64, 136, dtype)
    img, _ = synth.single_512(DEV)
    for h, v in ((host, view), (img.cpu().numpy(), img)):
        Hh, Ww = h.shape
        coef = torch.zeros(((Hh + 7) // 8, (Ww + 7) // 8, 8, 8), dtype=torch.float32, device=DEV)
        for r in (1, 10, 16, 64):
            sse = torch.zeros(1, dtype=torch.int64, device=DEV)
            psnr = torch.zeros(1, dtype=torch.float64, device=DEV)
            P.tdct_dct_codec_error(v, r, sse, precision=P.TDCT_FP32, coef=coef, psnr=psnr)
            torch.cuda.synchronize()
            want_sse, _, want_coef = oc.dct_codec_plane(h, r, want_recon=False, want_coef=True)
            assert _dct_rel_err(coef.cpu().numpy().astype(np.float64), want_coef) <= 1e-5
            p64 = oc.psnr(want_sse, h.size)
            if np.isfinite(p64):
                assert abs(float(psnr.item()) - p64) <= 0.01
            else:
                assert int(sse.item()) <= 2  # r = 64: only rounding ties can differ


def test_dct_bf16_error_is_bounded():
    img, _ = synth.single_512(DEV)
    h = img.cpu().numpy()
    coef = torch.zeros((64, 64, 8, 8), dtype=torch.float32, device=DEV)
    sse = torch.zeros(1, dtype=torch.int64, device=DEV)
    P.tdct_dct_codec_error(img, 16, sse, precision=P.TDCT_BF16, coef=coef)
    torch.cuda.synchronize()
    want_sse, _, want_coef = oc.dct_codec_plane(h, 16, want_recon=False, want_coef=True)
    err = _dct_rel_err(coef.cpu().numpy().astype(np.float64), want_coef)
    # bf16 carries 8 significant bits: two rounded stages stay within a few 2^-8
    assert err <= 2.0**-6
    assert abs(oc.psnr(int(sse.item()), h.size) - oc.psnr(want_sse, h.size)) <= 0.5


def test_status_word_clean():
    P.tdct_sync_status()


@pytest.mark.parametrize("H,W", [(8, 16), (16, 512), (64, 1040), (48, 2048), (8, 4096)])
def test_bulk_copy_ring_planes(H, W):
    """u8 planes with 16-byte aligned rows, W % 16 == 0 and H % 8 == 0 take the
    bulk-copy ring (including a ragged last unit when W is not a multiple of 512)."""
    rng = np.random.default_rng(H * 7 + W)
    host = rng.integers(0, 256, (H, W)).astype(np.uint8)
    img = torch.from_numpy(host).to(DEV)
    for r in (1, 10, 16, 40, 64):
        sse, rec, _ = run_codec(img, r)
        want_sse, want_rec, _ = oc.codec_plane(host, M.T1, r)
        assert np.array_equal(rec, want_rec) and sse == want_sse
        sse2, _, _ = run_codec(img, r, want_recon=False)
        assert sse2 == want_sse


@pytest.mark.parametrize("H,W,extra", [(8, 8, 0), (16, 24, 0), (64, 1032, 0), (48, 2056, 16),
                                       (8, 4104, 0), (40, 520, 32), (64, 1544, 0)])
def test_bulk_copy_ring_rows_8_mod_16(H, W, extra):
    """u8 planes with a 16-byte aligned base, W % 16 == 8, pitch 8 mod 16 and
    H % 8 == 0 take the bulk-copy ring: odd rows start 8 bytes past a 16-byte
    boundary and are copied from 8 bytes earlier; the last pair of each block
    row has one block.  Pitched reconstructions too."""
    rng = np.random.default_rng(H * 13 + W + extra)
    big = rng.integers(0, 256, (H, W + extra)).astype(np.uint8)
    img = torch.from_numpy(big).to(DEV)[:, :W]
    host = big[:, :W]
    planes_r = P.make_planes([img], [16])
    plan = P.tdct_plan_create(planes_r, path=P.TDCT_PATH_BUTTERFLY)
    try:
        assert plan.groups()[0]["load"] == "bulk"
    finally:
        plan.close()
    for r in (1, 10, 16, 40, 64):
        sse, rec, _ = run_codec(img, r)
        want_sse, want_rec, _ = oc.codec_plane(host, M.T1, r)
        assert np.array_equal(rec, want_rec) and sse == want_sse, r
        rec_big = torch.full((H, W + 24), 3, dtype=torch.uint8, device=DEV)
        sse2 = torch.zeros(1, dtype=torch.int64, device=DEV)
        P.tdct_codec_error(img, r, sse2, recon=rec_big[:, :W])
        torch.cuda.synchronize()
        assert int(sse2.item()) == want_sse
        assert np.array_equal(rec_big[:, :W].cpu().numpy(), want_rec)
        assert (rec_big[:, W:].cpu().numpy() == 3).all()


def test_bulk_copy_ring_many_units_per_warp():
    """Enough units that every warp walks its ring many times, across planes."""
    imgs, _ = synth.batch_1024x1024(DEV, n=48)
    r = 16
    recons = torch.empty_like(imgs)
    planes = P.make_planes([imgs[i] for i in range(48)], [r] * 48, [recons[i] for i in range(48)])
    sse = torch.zeros(48, dtype=torch.int64, device=DEV)
    P.tdct_codec_error_batched(planes, sse)
    torch.cuda.synchronize()
    for i in (0, 1, 23, 47):
        want_sse, want_rec, _ = oc.codec_plane(imgs[i].cpu().numpy(), M.T1, r)
        assert int(sse[i]) == want_sse
        assert np.array_equal(recons[i].cpu().numpy(), want_rec)


@pytest.mark.parametrize("H,W", [(8, 8), (16, 24), (64, 1032), (48, 2056), (8, 4104), (13, 16),
                                 (540, 968), (7, 1032), (1, 8)])
def test_staged_copy_ring_planes(H, W):
    """u8 planes with 8-byte aligned rows and W % 8 == 0 that miss the bulk-copy
    conditions (W % 16 == 8 or H % 8 != 0) take the staged-copy ring (the last
    lane of a row may code one block only; rows past the bottom edge are
    zero-filled)."""
    rng = np.random.default_rng(H * 11 + W)
    host = rng.integers(0, 256, (H, W)).astype(np.uint8)
    img = torch.from_numpy(host).to(DEV)
    for r in (1, 10, 16, 40, 64):
        sse, rec, _ = run_codec(img, r)
        want_sse, want_rec, _ = oc.codec_plane(host, M.T1, r)
        assert np.array_equal(rec, want_rec) and sse == want_sse
        sse2, _, _ = run_codec(img, r, want_recon=False)
        assert sse2 == want_sse


@pytest.mark.parametrize("H,W", [(8, 8), (13, 16), (540, 960), (64, 1032), (1080, 1920),
                                 (21, 520)])
def test_int16_bulk_copy_ring_planes(H, W):
    """int16 residual planes with a 16-byte aligned base and pitch and W % 8 ==
    0 take the int16 bulk-copy ring; heights that are not multiples of 8 (the
    540-row chroma planes) are zero-padded in shared memory, widths that are
    not multiples of 512 give a short last unit."""
    rng = np.random.default_rng(H * 13 + W)
    host = rng.integers(-255, 256, (H, W)).astype(np.int16)
    img = torch.from_numpy(host).to(DEV)
    for r in ((8, 16) if H * W > 100000 else (1, 8, 16, 40, 64)):
        sse, rec, _ = run_codec(img, r)
        want_sse, want_rec, _ = oc.codec_plane(host, M.T1, r)
        assert np.array_equal(rec, want_rec) and sse == want_sse
        sse2, _, _ = run_codec(img, r, want_recon=False)
        assert sse2 == want_sse


@pytest.mark.parametrize("H,W", [(8, 16), (13, 24), (540, 968), (64, 1040)])
def test_int16_staged_copy_ring_planes(H, W):
    """int16 residual planes whose first sample sits 8 bytes past a 16-byte
    boundary (rows 8-byte aligned, W % 8 == 0, not bulk-copy eligible) take the
    int16 staged-copy ring; heights that are not multiples of 8 are
    zero-padded in shared memory."""
    rng = np.random.default_rng(H * 17 + W)
    big = rng.integers(-255, 256, (H, W + 4)).astype(np.int16)
    img = torch.from_numpy(big).to(DEV)[:, 4:]
    host = big[:, 4:]
    planes = P.make_planes([img], [16])
    plan = P.tdct_plan_create(planes, path=P.TDCT_PATH_BUTTERFLY)
    try:
        assert plan.groups()[0]["load"] == "staged"
    finally:
        plan.close()
    for r in ((8, 16) if H * W > 100000 else (1, 8, 16, 40, 64)):
        sse, rec, _ = run_codec(img, r)
        want_sse, want_rec, _ = oc.codec_plane(host, M.T1, r)
        assert np.array_equal(rec, want_rec) and sse == want_sse
        sse2, _, _ = run_codec(img, r, want_recon=False)
        assert sse2 == want_sse


def test_staged_bulk_and_plain_planes_in_one_batch():
    """Bulk-copy, staged-copy and plain planes with mixed r in one batch, enough
    units that every warp walks its ring many times."""
    rng = np.random.default_rng(77)
    sizes = [(1024, 1032)] * 10 + [(1024, 1024)] * 10 + [(1023, 1033)] * 3 + [(520, 8), (8, 520)]
    hosts, views, rs = [], [], []
    for i, (H, W) in enumerate(sizes):
        h = rng.integers(0, 256, (H, W)).astype(np.uint8)
        hosts.append(h)
        views.append(torch.from_numpy(h).to(DEV))
        rs.append((4, 8, 16, 32)[i % 4])
    recons = [torch.full_like(v, 5) for v in views]
    sse = torch.zeros(len(views), dtype=torch.int64, device=DEV)
    P.tdct_codec_error_batched(P.make_planes(views, rs, recons), sse)
    torch.cuda.synchronize()
    for i in (0, 9, 10, 19, 20, 22, 23, 24):
        want_sse, want_rec, _ = oc.codec_plane(hosts[i], M.T1, rs[i])
        assert int(sse[i]) == want_sse, i
        assert np.array_equal(recons[i].cpu().numpy(), want_rec), i


def test_plan_routes_planes_to_the_intended_load_paths():
    """Bulk-copy ring for u8 planes with a 16-byte aligned base and H % 8 == 0
    whose rows are 16-byte aligned with W % 16 == 0, or whose pitch is 8 mod 16
    with W % 16 == 8; staged-copy ring for other 8-byte aligned rows with
    W % 8 == 0 (u8 and int16, any height); plain loads otherwise."""
    u8 = lambda H, W: torch.zeros(H, W, dtype=torch.uint8, device=DEV)
    i16 = lambda H, W: torch.zeros(H, W, dtype=torch.int16, device=DEV)
    odd_pitch = torch.zeros(64 * 132, dtype=torch.int16, device=DEV)[2:2 + 64 * 130].view(64, 130)
    base8 = torch.zeros(64 * 1032 + 8, dtype=torch.uint8, device=DEV)[8:].view(64, 1032)
    cases = [(u8(64, 1024), "u8", 3, "bulk"), (u8(64, 1032), "u8", 4, "bulk"),
             (u8(60, 1024), "u8", 5, "staged"), (u8(64, 1030), "u8", 6, "plain"),
             (i16(540, 960), "i16", 7, "bulk"), (odd_pitch[:, :128], "i16", 9, "plain"),
             (torch.zeros(64, 136, dtype=torch.int16, device=DEV)[:, 4:132], "i16", 12, "staged"),
             (base8, "u8", 10, "staged"), (u8(64, 1040)[:, :1032], "u8", 11, "staged")]
    planes = P.make_planes([c[0] for c in cases], [c[2] for c in cases])
    plan = P.tdct_plan_create(planes, path=P.TDCT_PATH_BUTTERFLY)
    try:
        got = {(g["dtype"], g["r"]): (g["load"], g["planes"]) for g in plan.groups()}
        assert len(got) == len(cases)
        for _, dt, r, load in cases:
            assert got[(dt, r)] == (load, 1), (dt, r, got[(dt, r)])
        assert plan.kernel_count() == len(cases) + 1  # + the PSNR kernel
    finally:
        plan.close()


def test_bounded_wait_timeout_is_reported_and_context_survives():
    """A withheld bulk copy makes one warp's bounded wait give up: the library
    reports TDCT_ETIMEOUT through the status word, nothing hangs, and the
    next call is correct."""
    rng = np.random.default_rng(9)
    host = rng.integers(0, 256, (64, 1024)).astype(np.uint8)
    img = torch.from_numpy(host).to(DEV)
    P.tdct_sync_status()  # clean start
    P.tdct_debug_inject_wait_timeout(True)
    sse = torch.zeros(1, dtype=torch.int64, device=DEV)
    P.tdct_codec_error(img, 16, sse)
    with pytest.raises(P.TdctError) as e:
        P.tdct_sync_status()
    assert e.value.code == 4  # TDCT_ETIMEOUT
    P.tdct_sync_status()  # the word was cleared
    got, rec, _ = run_codec(img, 16)
    want_sse, want_rec, _ = oc.codec_plane(host, M.T1, 16)
    assert got == want_sse and np.array_equal(rec, want_rec)
    P.tdct_sync_status()


# ---- the tensor-core forward (tcgen05.mma, exact fp16 inputs, FP32 accumulate) ----


def _run_batch_path(views, rs, path, with_recon=True):
    recons = [torch.full_like(v, 5) for v in views] if with_recon else None
    planes = P.make_planes(views, rs, recons)
    sse = torch.zeros(len(views), dtype=torch.int64, device=DEV)
    psnr = torch.zeros(len(views), dtype=torch.float64, device=DEV)
    P.tdct_codec_error_batched(planes, sse, psnr, path=path)
    torch.cuda.synchronize()
    return sse.cpu().numpy(), psnr.cpu().numpy(), recons


@pytest.mark.parametrize("path", ["tensor", "tensor_pipelined"])
@pytest.mark.parametrize("H,W", [(8, 16), (16, 512), (64, 1040), (48, 2048), (8, 4096)])
def test_tensor_path_matches_oracle(H, W, path):
    path = P.TDCT_PATH_TENSOR if path == "tensor" else P.TDCT_PATH_TENSOR_PIPELINED
    rng = np.random.default_rng(H * 11 + W)
    host = rng.integers(0, 256, (H, W)).astype(np.uint8)
    img = torch.from_numpy(host).to(DEV)
    for r in (1, 3, 8, 9, 10, 16, 17, 32, 33, 64):
        sse, psnr, recons = _run_batch_path([img], [r], path)
        want_sse, want_rec, _ = oc.codec_plane(host, M.T1, r)
        assert sse[0] == want_sse, f"r={r}"
        assert np.array_equal(recons[0].cpu().numpy(), want_rec), f"r={r}"
        sse2, _, _ = _run_batch_path([img], [r], path, with_recon=False)
        assert sse2[0] == want_sse


def test_tensor_path_adversarial_and_mixed_batch():
    blocks = synth.adversarial_blocks(DEV)  # 8 x 1072: eligible for the tensor path
    rng = np.random.default_rng(31)
    odd = torch.from_numpy(rng.integers(0, 256, (13, 11)).astype(np.uint8)).to(DEV)
    res = torch.from_numpy(rng.integers(-255, 256, (16, 32)).astype(np.int16)).to(DEV)
    views = [blocks, odd, res, blocks]
    rs = [16, 10, 8, 64]
    sse, _, recons = _run_batch_path(views, rs, P.TDCT_PATH_TENSOR)
    for i, v in enumerate(views):
        want_sse, want_rec, _ = oc.codec_plane(v.cpu().numpy(), M.T1, rs[i])
        assert sse[i] == want_sse
        assert np.array_equal(recons[i].cpu().numpy(), want_rec)


def test_tensor_path_equals_butterfly_on_many_images():
    imgs, r = synth.batch_1024x1024(DEV, n=64)
    views = [imgs[i] for i in range(64)]
    a, pa, ra = _run_batch_path(views, [r] * 64, P.TDCT_PATH_TENSOR)
    b, pb, rb = _run_batch_path(views, [r] * 64, P.TDCT_PATH_BUTTERFLY)
    c, pc, rc = _run_batch_path(views, [r] * 64, P.TDCT_PATH_TENSOR_PIPELINED)
    assert np.array_equal(a, b) and np.array_equal(pa, pb)
    assert np.array_equal(c, b) and np.array_equal(pc, pb)
    for i in (0, 31, 63):
        assert torch.equal(ra[i], rb[i]) and torch.equal(rc[i], rb[i])
    assert a[0] == oc.codec_plane(imgs[0].cpu().numpy(), M.T1, r, want_recon=False)[0]
    planes = P.make_planes(views, [r] * 64)
    plan = P.tdct_plan_create(planes, path=P.TDCT_PATH_TENSOR)
    sse = torch.zeros(64, dtype=torch.int64, device=DEV)
    for _ in range(2):
        plan.launch(sse)
        torch.cuda.synchronize()
        assert np.array_equal(sse.cpu().numpy(), b)
    plan.close()


@pytest.mark.parametrize("variant", ["tensor", "tensor_pipelined"])
def test_tensor_path_bounded_wait_timeout(variant):
    path = P.TDCT_PATH_TENSOR if variant == "tensor" else P.TDCT_PATH_TENSOR_PIPELINED
    img = torch.from_numpy(np.random.default_rng(3).integers(0, 256, (64, 1024)).astype(np.uint8)).to(DEV)
    P.tdct_sync_status()
    _run_batch_path([img], [16], path)  # tables built, kernel loaded
    P.tdct_debug_inject_wait_timeout(True)
    _run_batch_path([img], [16], path)
    with pytest.raises(P.TdctError) as e:
        P.tdct_sync_status()
    assert e.value.code == 4
    sse, _, recons = _run_batch_path([img], [16], path)
    want_sse, want_rec, _ = oc.codec_plane(img.cpu().numpy(), M.T1, 16)
    assert sse[0] == want_sse and np.array_equal(recons[0].cpu().numpy(), want_rec)
    P.tdct_sync_status()


def test_autotuned_plan_is_correct_and_reports_its_choice():
    rng = np.random.default_rng(41)
    hosts = [rng.integers(0, 256, (64, 1024)).astype(np.uint8) for _ in range(6)]
    views = [torch.from_numpy(h).to(DEV) for h in hosts]
    odd = rng.integers(-255, 256, (13, 24)).astype(np.int16)
    hosts.append(odd)
    views.append(torch.from_numpy(odd).to(DEV))
    rs = [16, 16, 4, 32, 10, 64, 8]
    recons = [torch.zeros_like(v) for v in views]
    plan = P.tdct_plan_create(P.make_planes(views, rs, recons), path=P.TDCT_PATH_AUTO)
    cfg = plan.config()
    assert cfg["path"] in ("butterfly", "tensor") and cfg["tuned_ms"] > 0
    sse = torch.zeros(len(views), dtype=torch.int64, device=DEV)
    plan.launch(sse)
    torch.cuda.synchronize()
    for i, h in enumerate(hosts):
        want_sse, want_rec, _ = oc.codec_plane(h, M.T1, rs[i])
        assert int(sse[i]) == want_sse
        assert np.array_equal(recons[i].cpu().numpy(), want_rec)
    plan.close()


def _extreme_i16_blocks():
    """int16 blocks at the residual bound: constants +-255 and +-255 times the
    sign pattern of every basis image t_i t_j^T of T1 (the inputs that
    maximise |Z_ij|), side by side in one 8-row strip."""
    T = np.array(M.T1, dtype=np.int64)
    blocks = [np.full((8, 8), 255), np.full((8, 8), -255)]
    for i in range(8):
        for j in range(8):
            sgn = np.sign(np.outer(T[i], T[j]))
            sgn[sgn == 0] = 1
            blocks.append(255 * sgn)
            blocks.append(-255 * sgn)
    return np.concatenate(blocks, axis=1).astype(np.int16)


@pytest.mark.parametrize("r", [1, 8, 10, 12, 13, 15, 16, 21, 28, 32, 36, 45, 64])
def test_int16_bulk_ring_extreme_blocks(r):
    """The int16 bulk-copy ring (two blocks per lane through a 16-bit packed
    forward up to class 32, Z_22 in 32 bits) on the blocks that reach the
    coefficient bounds, bit-exact against the oracle."""
    host = _extreme_i16_blocks()
    H, W = host.shape  # 8 x 8 * 130 (W % 8 == 0, rows 16-byte aligned)
    view = torch.from_numpy(host).to(DEV)
    for hh in (8, 16):
        h = np.ascontiguousarray(np.concatenate([host] * (hh // 8), axis=0)[:, ::-1])
        v = torch.from_numpy(h).to(DEV)
        sse, rec, _ = run_codec(v, r)
        want_sse, want_rec, _ = oc.codec_plane(h, M.T1, r)
        assert sse == want_sse and np.array_equal(rec, want_rec), (r, hh)
    sse, rec, _ = run_codec(view, r)
    want_sse, want_rec, _ = oc.codec_plane(host, M.T1, r)
    assert sse == want_sse and np.array_equal(rec, want_rec), r
