"""Batches of u8 planes whose width is not a multiple of 64 blocks: at r > 10
their ring units run on across block rows (64 consecutive blocks in raster
order, up to two row segments per unit).  Bit-exact SSE and reconstruction against
the oracle through the batched call, a plan (graph replay), the host-buffer
call and a forced tensor-engine plan (which keeps units per block row), with
planes of other load paths in the same batch."""
import numpy as np
import pytest
import torch

import paper_1808_02950_gb300 as P
from oracle import codec as oc
from oracle import matrices as M

pytestmark = pytest.mark.gpu
DEV = "cuda"

# (H, W): W % 16 == 0 and W / 8 >= 64 not a multiple of 64 take the wrapping
# units; 1024 and 512 wide planes (whole units per block row), a 504-wide one
# (under 64 blocks) and a 1032-wide one (8 mod 16: the shifted ring) do not
SHAPES = [(8, 528), (16, 1040), (24, 1552), (72, 528), (40, 4112), (520, 1040), (64, 1024),
          (8, 512), (32, 504), (16, 1032), (8, 1040), (2, 528)]


def _planes(seed):
    rng = np.random.default_rng(seed)
    hosts = [rng.integers(0, 256, s).astype(np.uint8) for s in SHAPES]
    # smooth content in one plane so that small r keep most of it
    y, x = np.mgrid[0:SHAPES[1][0], 0:SHAPES[1][1]]
    hosts[1] = (128 + 60 * np.sin(x / 17.0) * np.cos(y / 5.0)).astype(np.uint8)
    return hosts


def _check(hosts, rs, sse, recons):
    for i, (h, r) in enumerate(zip(hosts, rs)):
        want_sse, want_rec, _ = oc.codec_plane(h, M.T1, r)
        assert int(sse[i]) == want_sse, (i, SHAPES[i], r)
        if recons is not None:
            assert np.array_equal(recons[i].cpu().numpy(), want_rec), (i, SHAPES[i], r)


@pytest.mark.parametrize("r", [1, 10, 16, 40, 64])
def test_wrap_units_batched_and_plan(r):
    hosts = _planes(r)
    views = [torch.from_numpy(h).to(DEV) for h in hosts]
    rs = [r if i % 3 else max(1, r // 2) for i in range(len(views))]
    recons = [torch.full_like(v, 7) for v in views]
    planes = P.make_planes(views, rs, recons)
    sse = torch.zeros(len(views), dtype=torch.int64, device=DEV)
    P.tdct_codec_error_batched(planes, sse)
    torch.cuda.synchronize()
    _check(hosts, rs, sse.cpu().numpy(), recons)
    # a plan (autotuned, graph replay), twice; without reconstructions
    plan = P.tdct_plan_create(P.make_planes(views, rs))
    for _ in range(2):
        sse2 = torch.zeros(len(views), dtype=torch.int64, device=DEV)
        plan.launch(sse2, None)
        torch.cuda.synchronize()
        _check(hosts, rs, sse2.cpu().numpy(), None)
    plan.close()


def test_wrap_units_tensor_engine_plan():
    hosts = _planes(3)
    views = [torch.from_numpy(h).to(DEV) for h in hosts]
    rs = [16] * len(views)
    recons = [torch.full_like(v, 7) for v in views]
    plan = P.tdct_plan_create(P.make_planes(views, rs, recons), path=P.TDCT_PATH_TENSOR)
    sse = torch.zeros(len(views), dtype=torch.int64, device=DEV)
    plan.launch(sse, None)
    torch.cuda.synchronize()
    plan.close()
    _check(hosts, rs, sse.cpu().numpy(), recons)


def test_wrap_units_many_units_per_warp():
    """A batch large enough that each warp takes several units (the ring wraps),
    including a plane whose last unit holds fewer than 64 blocks."""
    rng = np.random.default_rng(11)
    shapes = [(1000, 1040)] * 24 + [(8, 528), (504, 2064)]
    hosts = [rng.integers(0, 256, s).astype(np.uint8) for s in shapes]
    views = [torch.from_numpy(h).to(DEV) for h in hosts]
    recons = [torch.full_like(v, 7) for v in views]
    sse = torch.zeros(len(views), dtype=torch.int64, device=DEV)
    P.tdct_codec_error_batched(P.make_planes(views, [16] * len(views), recons), sse)
    torch.cuda.synchronize()
    for i in (0, 13, 23, 24, 25):
        want_sse, want_rec, _ = oc.codec_plane(hosts[i], M.T1, 16)
        assert int(sse[i].item()) == want_sse, i
        assert np.array_equal(recons[i].cpu().numpy(), want_rec), i
    P.tdct_sync_status()


def test_wrap_units_host_buffers():
    hosts = _planes(5)
    cpu = [torch.from_numpy(h).pin_memory() for h in hosts]
    recons = [torch.full_like(c, 7).pin_memory() for c in cpu]
    rs = [16] * len(cpu)
    sse = torch.zeros(len(cpu), dtype=torch.int64).pin_memory()
    P.tdct_codec_error_batched_host(P.make_planes(cpu, rs, recons), sse, chunk_bytes=1 << 20)
    torch.cuda.synchronize()
    _check(hosts, rs, sse.numpy(), recons)
