"""Benchmark of the fused 8x8 T1 block codec on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batch_1024x1024|ragged_2000|video_600x1080p|single_512]

A step is one pass of the whole path -- forward transform, zonal retention
of the first r zig-zag coefficients, inverse, rounding, reconstruction
written back, per-image SSE and PSNR -- over every image of the workload,
with the inputs resident in HBM.  The default workload is 1024 seeded
1024x1024 u8 AR(1) images with r = 16 (16.8 M blocks, 1 GiB in + 1 GiB
reconstruction out, larger than L2, so no flush is needed between steps).

Timing: W untimed steps, then K steps between barriers and device
synchronisation, CUDA events on the launching stream; the max over ranks.
With N > 1 (torchrun) every rank runs its own replica of the workload
(weak scaling, no collective on the data path).  Rank 0 prints one JSON
line.  ``--impl reference`` times the CPU oracle on host cores instead.

Besides the step, the default run reports on the same images: ``e2e`` (the
host-buffer call with its copies; ``e2e_recon`` also returns every
reconstruction), ``ssim`` (mean SSIM of original vs reconstruction), ``jam``
(16x16 and 32x32 blocks with the JAM matrices), ``dct`` (the exact-DCT
comparison codec, FP32 and BF16) and ``search`` (the greedy angle search,
N = 16 and 12); ``configs`` times the other workloads (single_512,
sweep_64x512, ragged_2000, video_600x1080p) each on its own, with its own
oracle parity sample; ``parity`` checks the timed run's per-image SSE against
the oracle on the cpu_baseline sample; ``cpu_baseline`` times the oracle on
all host cores and on one.  ``--no-e2e``, ``--no-ssim``, ``--no-jam``,
``--no-dct``, ``--no-search`` and ``--no-configs`` skip them.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "8×8 blocks/s and HBM GB/s (% of peak), fused fwd+zonal+inv+SSE, bit-exact, 1 GB300"
UNIT = "blocks/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch_1024x1024",
                    choices=["batch_1024x1024", "ragged_2000", "video_600x1080p", "single_512"])
    ap.add_argument("--images", type=int, default=1024,
                    help="images of batch_1024x1024 (smaller only for profiling captures)")
    ap.add_argument("--path", default="auto",
                    choices=["butterfly", "tensor", "tensor_pipelined", "auto"],
                    help="forward-transform engine of the fused codec (auto: the plan autotunes)")
    ap.add_argument("--transform", default="T1", choices=["T1", "T2", "RDCT", "T6", "T4", "LOx2"],
                    help="the 8-point matrix (T1: fused kernels; others: generic kernels)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-jam", action="store_true",
                    help="skip the 16x16 / 32x32 JAM codec timing")
    ap.add_argument("--no-dct", action="store_true",
                    help="skip the exact-DCT comparison codec timing (FP32 and BF16)")
    ap.add_argument("--no-search", action="store_true",
                    help="skip the angle-search timing (N = 16 and N = 12, P = {-1, 0, 1})")
    ap.add_argument("--no-ssim", action="store_true",
                    help="skip the MSSIM measurement (originals vs reconstructions)")
    ap.add_argument("--no-generic", action="store_true",
                    help="skip the generic-T timing (T2, RDCT, T6, T4, LO x 2)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (single_512, sweep_64x512, ragged_2000, "
                         "video_600x1080p)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="CPU-oracle sample budget (seconds of host work, all cores)")
    ap.add_argument("--cpu-seconds-single", type=float, default=4.0,
                    help="CPU-oracle sample budget on one core")
    return ap.parse_args()


# ---- distributed plumbing ---------------------------------------------------------------


class Dist:
    def __init__(self, backend: str):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        return self._reduce(v, "max")

    def sum(self, v: float) -> float:
        return self._reduce(v, "sum")

    def _reduce(self, v, op):
        if not self.pg:
            return v
        import torch

        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---- clocks during the timed region -------------------------------------------------------


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons),
            "samples": len(self.rows),
        }


def kernel_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in ("tdct_device.cuh", "tdct_kernels.cuh"):
        with open(os.path.join(ROOT, "paper_1808_02950_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(images: int):
    """DRAM bytes (read + write) of one launch of the fused codec on the bench
    workload, from the committed ncu summary of a capture of that same launch
    (1024 images); None when the kernel sources changed since the capture or
    the workload differs."""
    import glob
    import re

    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "codec_u8_tma_kernel_*.md"))):
        text = open(path).read()
        m_h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
        m_t = re.search(r"traffic_bytes_per_launch:\s*([0-9.]+)", text)
        m_i = re.search(r"traffic_images:\s*([0-9]+)", text)
        if (m_h and m_t and m_i and m_h.group(1) == kernel_source_hash()
                and int(m_i.group(1)) == images):
            return float(m_t.group(1)), os.path.basename(path)
    return None, None


def aggregate(dist, blocks_local: int, ms_local: float, steps: int):
    """Whole-job throughput of replicas: the units all ranks processed over
    the slowest rank's time.  Returns (blocks/s, max ms, total blocks)."""
    total_ms = dist.max(ms_local)
    blocks_all = dist.sum(blocks_local)
    return blocks_all * steps / (total_ms / 1e3), total_ms, blocks_all


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# Nominal HBM3e bandwidth of one GB300 (8 stacks, 7.9 TB/s), for the fraction
# beside the measured copy bandwidth.
NOMINAL_HBM_GBS = 7900.0


def device_sms() -> int:
    import torch

    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def hbm_figures(algo_bytes: float, ms: float) -> dict:
    """Achieved bandwidth of `algo_bytes` moved in `ms`, against the measured
    copy bandwidth and the nominal HBM3e peak."""
    peak, kind = measured_peaks()
    gbs = algo_bytes / (ms / 1e3) / 1e9
    return {"hbm_gbs": gbs, "frac": gbs / peak, "peak": peak, "peak_kind": kind,
            "frac_of_nominal": gbs / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS}


def time_launches(fn, stream, steps: int, warmup: int = 3) -> float:
    """Mean ms per call of `fn()` over `steps` calls, CUDA events on `stream`
    (the launching stream), after `warmup` untimed calls."""
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


# ---- workloads --------------------------------------------------------------------------------


class Workload:
    """Planes of one workload resident on the GPU, with reconstruction buffers."""

    def __init__(self, name: str, device: str, images: int = 1024):
        import torch

        from paper_1808_02950_gb300 import synth

        self.name = name
        self.planes = []  # (img tensor 2-D, r)
        if name == "batch_1024x1024":
            imgs, r = synth.batch_1024x1024(device, n=images)
            self.storage = [imgs]
            self.planes = [(imgs[i], r) for i in range(imgs.shape[0])]
            self.desc = {"workload": "batch_1024x1024", "images": int(imgs.shape[0]),
                         "H": 1024, "W": 1024, "dtype": "u8", "r": r, "rho": 0.95}
        elif name == "single_512":
            img, r = synth.single_512(device)
            self.storage = [img]
            self.planes = [(img, r)]
            self.desc = {"workload": "single_512", "images": 1, "H": 512, "W": 512, "dtype": "u8",
                         "r": r, "rho": 0.95}
        elif name == "ragged_2000":
            buf, offs, H, W, rr = synth.ragged_2000(device)
            self.storage = [buf]
            for i in range(len(offs)):
                v = buf[int(offs[i]): int(offs[i]) + int(H[i] * W[i])].view(int(H[i]), int(W[i]))
                self.planes.append((v, int(rr[i])))
            self.desc = {"workload": "ragged_2000", "images": len(offs), "dtype": "u8",
                         "H,W": "U{64..4096} step 8", "r": "U{4,8,16,32}"}
        elif name == "video_600x1080p":
            Y, U, V = synth.video_600x1080p(device)
            self.storage = [Y, U, V]
            for t in range(Y.shape[0]):
                self.planes += [(Y[t], 16), (U[t], 8), (V[t], 8)]
            self.desc = {"workload": "video_600x1080p", "frames": int(Y.shape[0]),
                         "planes": len(self.planes), "dtype": "i16 residual", "r": "Y 16, UV 8"}
        else:
            raise ValueError(name)
        self.recons = [torch.empty_like(p) for p, _ in self.planes]
        self.blocks = sum(((p.shape[0] + 7) // 8) * ((p.shape[1] + 7) // 8) for p, _ in self.planes)
        self.in_bytes = sum(p.numel() * p.element_size() for p, _ in self.planes)
        self.out_bytes = sum(p.numel() * p.element_size() for p in self.recons)


def time_ours(args, dist, out):
    import torch

    import paper_1808_02950_gb300 as P
    from paper_1808_02950_gb300 import transforms

    T = transforms.NAMED[args.transform]
    Tn = dict(T=T, n=transforms.row_norms(T))
    dev = f"cuda:{dist.local_rank}"
    torch.cuda.set_device(dev)
    wl = Workload(args.workload, dev, args.images)
    planes = P.make_planes([p for p, _ in wl.planes], [r for _, r in wl.planes], wl.recons)
    n = len(wl.planes)
    sse = torch.zeros(n, dtype=torch.int64, device=dev)
    psnr = torch.zeros(n, dtype=torch.float64, device=dev)
    path = {"butterfly": P.TDCT_PATH_BUTTERFLY, "tensor": P.TDCT_PATH_TENSOR,
            "tensor_pipelined": P.TDCT_PATH_TENSOR_PIPELINED, "auto": P.TDCT_PATH_AUTO}[args.path]
    plan = P.tdct_plan_create(planes, path=path, **Tn)
    plan_cfg = plan.config()
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        plan.launch(sse, psnr, stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    dist.barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(args.steps):
        plan.launch(sse, psnr, stream)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    value, total_ms, blocks_all = aggregate(dist, wl.blocks, ev[0].elapsed_time(ev[args.steps]),
                                            args.steps)
    step_ms = total_ms / args.steps

    # Roofline of the dominant kernel (the fused codec): algorithmic bytes =
    # samples read once + reconstruction written once (+ 16 B per image),
    # over the codec's own launch time: the same plan launched without the
    # PSNR node (the SSE reset memset is a few microseconds), timed with CUDA
    # events on the launching stream right after the timed region.
    algo_bytes = wl.in_bytes + wl.out_bytes + 16 * n
    plan.launch(sse, None, stream)  # instantiates the PSNR-less graph
    kev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    kev[0].record(stream)
    for k in range(args.steps):
        plan.launch(sse, None, stream)
        kev[k + 1].record(stream)
    torch.cuda.synchronize()
    kernel_ms = statistics.mean(kev[k].elapsed_time(kev[k + 1]) for k in range(args.steps))
    peak, peak_kind = measured_peaks()
    achieved = algo_bytes / (kernel_ms / 1e3) / 1e9
    traffic, traffic_src = (profiled_traffic(wl.desc["images"])
                            if args.workload == "batch_1024x1024" and args.transform == "T1"
                            else (None, None))
    wl.sse_host = sse.cpu().numpy()  # the timed configuration's SSE (parity below)
    out.update({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32 (u8 in/out)", "data": "synthetic",
        "config": {**wl.desc, "transform": args.transform,
                   "parallelism": f"replicas{dist.world}", "path": plan_cfg["path"],
                   "ctas_per_sm": plan_cfg["ctas_per_sm"], "autotuned": args.path == "auto",
                   "l2": "inputs larger than L2 (no flush)" if algo_bytes > 256e6 else
                   "inputs smaller than L2"},
        "hbm_gbs": achieved,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                     "peak_kind": peak_kind,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "nominal_peak": NOMINAL_HBM_GBS,
                     "algo_bytes_per_launch": algo_bytes, "kernel_ms": kernel_ms},
        "clocks": clk,
        "gpu_launches": plan.kernel_count() * args.steps,
    })

    # End to end through the public C-ABI call with HOST buffers: every step
    # hands the pinned host planes to tdct_codec_error_batched_host, which
    # copies them to the device in chunks pipelined with the codec, and the
    # per-image SSE and PSNR come back into pinned host arrays.
    if not args.no_e2e:
        host_bufs = [st.cpu().pin_memory() for st in wl.storage]
        rows = []
        for (pl, r) in wl.planes:
            k = next(k for k, st in enumerate(wl.storage)
                     if st.data_ptr() <= pl.data_ptr() < st.data_ptr() + st.numel() * st.element_size())
            hp = host_bufs[k].data_ptr() + (pl.data_ptr() - wl.storage[k].data_ptr())
            dt = P.TDCT_U8 if pl.dtype == torch.uint8 else P.TDCT_I16
            rows.append((hp, pl.stride(0) * pl.element_size(), pl.shape[0], pl.shape[1], r, dt, 0, 0))
        planes_h = P.make_planes_raw(rows)
        sse_h = torch.empty(n, dtype=torch.int64).pin_memory()
        psnr_h = torch.empty(n, dtype=torch.float64).pin_memory()

        def e2e_step():
            P.tdct_codec_error_batched_host(planes_h, sse_h, psnr_h, stream=stream, **Tn)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        ke = max(3, min(args.steps, 10))
        dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ke):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        e_ms = dist.max(e0.elapsed_time(e1))
        out["e2e"] = {"value": blocks_all * ke / (e_ms / 1e3), "unit": UNIT,
                      "h2d_bytes_per_step": int(wl.in_bytes), "d2h_bytes_per_step": 16 * n,
                      "steps": ke, "call": "tdct_codec_error_batched_host",
                      "reconstruction_returned": False}
        # The same call returning every reconstruction to pinned host memory
        # (the device-timed step writes them to HBM): 1 GiB back per step.
        rec_bufs = [torch.empty_like(hb).pin_memory() for hb in host_bufs]
        rows_r = []
        for row, (pl, _) in zip(rows, wl.planes):
            k = next(k for k, st in enumerate(wl.storage)
                     if st.data_ptr() <= pl.data_ptr() < st.data_ptr() + st.numel() * st.element_size())
            rp = rec_bufs[k].data_ptr() + (row[0] - host_bufs[k].data_ptr())
            rows_r.append(row[:6] + (rp, row[1]))
        planes_r = P.make_planes_raw(rows_r)

        def e2e_recon_step():
            P.tdct_codec_error_batched_host(planes_r, sse_h, psnr_h, stream=stream, **Tn)

        for _ in range(2):
            e2e_recon_step()
        torch.cuda.synchronize()
        dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ke):
            e2e_recon_step()
        e1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        r_ms = dist.max(e0.elapsed_time(e1))
        out["e2e_recon"] = {"value": blocks_all * ke / (r_ms / 1e3), "unit": UNIT,
                            "h2d_bytes_per_step": int(wl.in_bytes),
                            "d2h_bytes_per_step": int(wl.out_bytes) + 16 * n, "steps": ke,
                            "call": "tdct_codec_error_batched_host",
                            "reconstruction_returned": True}
        del rec_bufs, host_bufs
    # MSSIM of every image against its reconstruction (the third figure of
    # merit of the paper's image experiment), timed separately: FP32 work on
    # the CUDA cores, reported against the FP32 FMA peak from unit counts and
    # clocks (the device's SMs x 128 lanes x 2 FLOP x max SM clock).
    u8_planes = [(pl, rc) for (pl, _), rc in zip(wl.planes, wl.recons) if pl.dtype == torch.uint8]
    if not args.no_ssim and u8_planes:
        plan.launch(sse, psnr, stream)  # reconstructions of the timed configuration
        mssim = torch.zeros(len(u8_planes), dtype=torch.float64, device=dev)
        for _ in range(2):
            P.tdct_ssim_batched(u8_planes, mssim, stream)
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        ks = 5
        s0.record(stream)
        for _ in range(ks):
            P.tdct_ssim_batched(u8_planes, mssim, stream)
        s1.record(stream)
        torch.cuda.synchronize()
        ms = s0.elapsed_time(s1) / ks
        windows = sum((pl.shape[0] - 10) * (pl.shape[1] - 10) for pl, _ in u8_planes)
        flops = 245.0 * windows  # 5 maps x 11 taps x 2 passes x 2 FLOP + the index
        sm_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
        peak = device_sms() * 128 * 2 * sm_mhz * 1e6 / 1e12
        out["ssim"] = {"value": windows / (ms / 1e3), "unit": "windows/s", "ms": ms,
                       "blocks_per_s": wl.blocks / (ms / 1e3), "mean_mssim": mssim.mean().item(),
                       "roofline": {"bound": "alu", "achieved": flops / (ms / 1e3) / 1e12,
                                    "peak": peak, "unit": "TFLOP/s",
                                    "frac": flops / (ms / 1e3) / 1e12 / peak,
                                    "peak_kind": "FP32 FMA lanes (SMs x 128) x 2 x max SM clock"}}
    # The codec with 16x16 and 32x32 blocks and the JAM matrices of §6.2, on
    # the same images (the batch as one tall plane: 1024 is a multiple of the
    # block sides, so no block straddles two images), reconstruction written.
    if not args.no_jam and args.workload == "batch_1024x1024" and args.transform == "T1":
        big = wl.storage[0].view(-1, wl.storage[0].shape[-1])
        rec_big = torch.empty_like(big)
        jsse = torch.zeros(1, dtype=torch.int64, device=dev)
        jam = {}
        for B in (16, 32):
            T = jam_matrix(B)
            # 3 untimed and 10 timed launches per B
            ms = time_launches(lambda: P.tdct_codec_error_jam(big, B, T, wl.desc["r"], jsse,
                                                              recon=rec_big, stream=stream),
                               stream, 10)
            gbs = 2 * big.numel() / (ms / 1e3) / 1e9
            jam[f"B{B}"] = {"ms": ms, "r": wl.desc["r"], "pixels_per_s": big.numel() / (ms / 1e3),
                            "hbm_gbs": gbs, "frac_of_measured_hbm": gbs / measured_peaks()[0]}
        out["jam"] = jam
    # The exact-DCT comparison codec (orthonormal DCT-II in FP32, or with
    # BF16-rounded inputs, constants and kept coefficients) on the same images
    # as one tall plane, reconstruction written.
    if not args.no_dct and args.workload == "batch_1024x1024" and args.transform == "T1":
        big = wl.storage[0].view(-1, wl.storage[0].shape[-1])
        rec_big = torch.empty_like(big)
        dsse = torch.zeros(1, dtype=torch.int64, device=dev)
        dct = {}
        for name, prec in (("fp32", P.TDCT_FP32), ("bf16", P.TDCT_BF16),
                           ("bf16x3", P.TDCT_BF16X3)):
            # 3 untimed and 10 timed launches per precision
            ms = time_launches(lambda: P.tdct_dct_codec_error(big, wl.desc["r"], dsse,
                                                              precision=prec, recon=rec_big,
                                                              stream=stream),
                               stream, 10)
            blocks = big.numel() // 64
            gbs = 2 * big.numel() / (ms / 1e3) / 1e9
            dct[name] = {"ms": ms, "r": wl.desc["r"], "blocks_per_s": blocks / (ms / 1e3),
                         "hbm_gbs": gbs, "frac_of_measured_hbm": gbs / measured_peaks()[0],
                         "engine": "CUDA cores (FP32 FMA)" if name == "fp32" else
                         "tensor cores (tcgen05.mma kind::f16, bf16 operands, FP32 accumulate)"}
        out["dct"] = dct
    # The generic kernels (NEXT-1: any orthogonal integer T) on the same images,
    # reconstruction written: every orthogonal matrix of Table 2 besides T1.
    if not args.no_generic and args.workload == "batch_1024x1024" and args.transform == "T1":
        gen = {}
        for name in ("T2", "RDCT", "T6", "T4", "LOx2"):
            Tg = transforms.NAMED[name]
            gplan = P.tdct_plan_create(planes, path=P.TDCT_PATH_BUTTERFLY, T=Tg,
                                       n=transforms.row_norms(Tg))
            ms = time_launches(lambda: gplan.launch(sse, None, stream), stream, 10)
            gplan.close()
            gbs = algo_bytes / (ms / 1e3) / 1e9
            gen[name] = {"ms": ms, "blocks_per_s": wl.blocks / (ms / 1e3), "hbm_gbs": gbs,
                         "frac_of_measured_hbm": gbs / measured_peaks()[0]}
        out["generic"] = gen
    plan.close()
    return wl


def oracle_parity(samples, sse_gpu, transform: str = "T1") -> dict:
    """Compare the oracle's SSE of each sampled plane with the GPU's.
    `samples`: (index into sse_gpu, host plane, r); one thread per core."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import codec as oc

    oc.lib()
    T = oracle_matrix(transform)

    def one(item):
        i, img, r = item
        return i, int(oc.codec_plane(img, T, r, want_recon=False)[0])

    threads = max(1, min(os.cpu_count() or 1, len(samples)))
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        got = list(ex.map(one, samples))
    dt = time.perf_counter() - t0
    blocks = sum(((img.shape[0] + 7) // 8) * ((img.shape[1] + 7) // 8) for _, img, _ in samples)
    # one core: the sample planes in order until about a second has passed
    t1 = time.perf_counter()
    b1 = 0
    for _, img, r in samples:
        oc.codec_plane(img, T, r, want_recon=False)
        b1 += ((img.shape[0] + 7) // 8) * ((img.shape[1] + 7) // 8)
        if time.perf_counter() - t1 > 1.0:
            break
    d1 = time.perf_counter() - t1
    bad = [i for i, want in got if int(sse_gpu[i]) != want]
    return {"planes": len(got), "mismatches": len(bad), "first_mismatch": bad[0] if bad else None,
            "check": "per-plane SSE of the timed run vs the C oracle (int64 definition)",
            "oracle_blocks_per_s": blocks / dt, "oracle_cores": threads,
            "oracle_blocks_per_s_1core": b1 / d1}


def time_configs(args, stream) -> dict:
    """The other workloads of the paper's experiments, each timed on its own
    (plan replays, CUDA events on the launching stream, inputs resident in
    HBM) and checked against the oracle on a sample of its planes:
    single_512 (one 512x512 image, r = 10; launch-bound), sweep_64x512 (64
    images x every r = 1..64, SSE per (image, r)), ragged_2000 (2000 images
    of random sizes, r in {4, 8, 16, 32}) and video_600x1080p (1797 int16
    residual planes, r = 16 / 8)."""
    import numpy as np
    import torch

    import paper_1808_02950_gb300 as P
    from paper_1808_02950_gb300 import synth

    dev = "cuda"
    steps = max(5, min(args.steps, 20))
    res = {}

    def plan_entry(planes, n, samples_fn, blocks, algo_bytes, unit_scale=1, unit=UNIT,
                   bound="hbm"):
        plan = P.tdct_plan_create(planes)
        sse = torch.zeros(n, dtype=torch.int64, device=dev)
        psnr = torch.zeros(n, dtype=torch.float64, device=dev)
        ms = time_launches(lambda: plan.launch(sse, psnr, stream), stream, steps)
        torch.cuda.synchronize()
        entry = {"value": blocks * unit_scale / (ms / 1e3), "unit": unit, "ms": ms,
                 "blocks": blocks, "algo_bytes": algo_bytes, "bound": bound,
                 **hbm_figures(algo_bytes, ms), "plan": plan.config(),
                 "launches_per_step": plan.kernel_count(),
                 "groups": len(plan.groups())}
        entry["parity"] = oracle_parity(samples_fn(), sse.cpu().numpy())
        plan.close()
        return entry

    # config 1: one 512x512 u8 image, r = 10 (4096 blocks: launch-bound)
    img, r = synth.single_512(dev)
    rec = torch.empty_like(img)
    res["single_512"] = plan_entry(
        P.make_planes([img], [r], [rec]), 1, lambda: [(0, img.cpu().numpy(), r)], 4096,
        2 * img.numel() + 16, bound="launch")
    res["single_512"]["r"] = r
    del img, rec

    # config 2: 64 images x r = 1..64, SSE per (image, r): the single-read
    # sweep (T1, and the exact DCT in FP32), with the per-r-plane batch of
    # the fused codec (each image read once per r) as the comparison
    imgs, _ = synth.sweep_64x512(dev)
    views = [imgs[i] for i in range(64)]
    host = imgs.cpu().numpy()
    sw_sse = torch.zeros(64 * 64, dtype=torch.int64, device=dev)
    sw_psnr = torch.zeros(64 * 64, dtype=torch.float64, device=dev)
    planes_sw = P.make_planes(views, [64] * 64)
    Tb, nb_ = P._lib._T_n()
    L = P.load()
    stream_h = stream.cuda_stream

    def sweep_t1():
        P._lib._check(L.tdct_sweep_batched(P._lib.ctypes.addressof(planes_sw), 64, Tb, nb_,
                                           sw_sse.data_ptr(), sw_psnr.data_ptr(), stream_h))

    def sweep_dct():
        P._lib._check(L.tdct_dct_sweep_batched(P._lib.ctypes.addressof(planes_sw), 64,
                                               P.TDCT_FP32, sw_sse.data_ptr(),
                                               sw_psnr.data_ptr(), stream_h))

    block_r = 64 * 4096 * 64
    ms_t1 = time_launches(sweep_t1, stream, steps)
    sweep_t1()
    torch.cuda.synchronize()
    got = sw_sse.cpu().numpy()
    sample_imgs = (0, 21, 42, 63)
    par = oracle_parity([(64 * i + r - 1, host[i], r) for i in sample_imgs for r in range(1, 65)],
                        got)
    ms_dct = time_launches(sweep_dct, stream, steps)
    # the comparison: one plane per (image, r) through the fused codec
    plan = P.tdct_plan_create(P.make_planes([v for v in views for _ in range(64)],
                                            [r for _ in range(64) for r in range(1, 65)]))
    pl_sse = torch.zeros(4096, dtype=torch.int64, device=dev)
    ms_planes = time_launches(lambda: plan.launch(pl_sse, None, stream), stream, steps)
    plan.close()
    sms = device_sms()
    res["sweep_64x512"] = {
        "value": block_r / (ms_t1 / 1e3), "unit": "block*r/s", "ms": ms_t1, "blocks": 64 * 4096,
        "r": "1..64", "bound": "alu", "method": "one read per image, incremental reconstruction "
        "(tdct_sweep_batched)", "parity": par,
        "ops_per_block_r": 288, "int_ops_per_s": 288 * block_r / (ms_t1 / 1e3),
        "issue_peak_ops_per_s": sms * 4 * 32 * 2.07e9,
        "dct_fp32": {"value": block_r / (ms_dct / 1e3), "unit": "block*r/s", "ms": ms_dct,
                     "call": "tdct_dct_sweep_batched"},
        "per_r_planes": {"value": block_r / (ms_planes / 1e3), "unit": "block*r/s",
                         "ms": ms_planes, "method": "4096 planes (image, r) in one plan"}}
    del imgs, views

    # config 4: 2000 u8 images of random sizes, r drawn per image
    buf, offs, H, W, rr = synth.ragged_2000(dev)
    rbuf = torch.empty_like(buf)
    views, rviews = [], []
    for i in range(len(offs)):
        o, h, w = int(offs[i]), int(H[i]), int(W[i])
        views.append(buf[o: o + h * w].view(h, w))
        rviews.append(rbuf[o: o + h * w].view(h, w))
    npx = int((H * W).sum())
    idx = list(range(0, len(offs), len(offs) // 32))[:32]
    res["ragged_2000"] = plan_entry(
        P.make_planes(views, [int(v) for v in rr], rviews), len(offs),
        lambda: [(i, views[i].cpu().numpy(), int(rr[i])) for i in idx],
        int(((H + 7) // 8 * ((W + 7) // 8)).sum()), 2 * npx + 16 * len(offs))
    del buf, rbuf, views, rviews

    # config 5: 599 residual frames of 1080p 4:2:0 video (int16), r = 16 (Y) / 8 (U, V)
    Y, U, V = synth.video_600x1080p(dev)
    planes, rs = [], []
    for t in range(Y.shape[0]):
        planes += [Y[t], U[t], V[t]]
        rs += [16, 8, 8]
    recs = [torch.empty_like(p) for p in planes]
    nbytes = sum(p.numel() * p.element_size() for p in planes)
    blocks = sum(((p.shape[0] + 7) // 8) * ((p.shape[1] + 7) // 8) for p in planes)
    idx = list(range(0, len(planes), 61))
    res["video_600x1080p"] = plan_entry(
        P.make_planes(planes, rs, recs), len(planes),
        lambda: [(i, planes[i].cpu().numpy(), rs[i]) for i in idx],
        blocks, 2 * nbytes + 16 * len(planes))
    del Y, U, V, planes, recs
    torch.cuda.empty_cache()
    return res


def jam_matrix(B: int):
    """T_(B) of §6.2 from T1 by the JAM rows: row 2i = [t_i, reverse(t_i)],
    row 2i + 1 = [t_i, -reverse(t_i)] (t_i the rows of the half-size matrix)."""
    from paper_1808_02950_gb300 import transforms as tr

    cur = [list(r) for r in tr.T1]
    while len(cur) < B:
        nxt = []
        for t in cur:
            nxt.append(t + t[::-1])
            nxt.append(t + [-v for v in t[::-1]])
        cur = nxt
    return cur


def time_search(skip_cpu: bool):
    """The greedy angle search on the GPU for one row order (natural order,
    P = {-1, 0, 1}) at N = 16, the case §6.2 times at about 6 minutes on a
    16-core Xeon E5-2630 v3, and at N = 12 with the CPU oracle beside it."""
    import numpy as np
    import torch

    import paper_1808_02950_gb300 as P

    res = {"alphabet": [-1, 0, 1], "order": "natural (rows 0..N-1)"}
    for N in (16, 12):
        P.tdct_search(N, (-1, 0, 1), range(N))  # warm-up (module load, pool)
        ts = []
        for _ in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            T, complete = P.tdct_search(N, (-1, 0, 1), range(N))
            ts.append(time.perf_counter() - t0)
        rows = int(np.count_nonzero(np.abs(np.array(T)).sum(axis=1)))
        res[f"N{N}"] = {"ms": 1e3 * statistics.median(ts), "rows_found": rows,
                        "complete": complete, "candidates": 3 ** N - 1}
    res["N16"]["paper_cpu_seconds"] = 360.0
    res["N16"]["paper_cpu"] = "16-core Xeon E5-2630 v3 @ 2.4 GHz (§6.2, row sequence not stated)"
    if not skip_cpu:
        from oracle import search as S

        t0 = time.perf_counter()
        S.abm_approx_n(12, range(12), S.P1, "small")
        cpu_s = time.perf_counter() - t0
        res["N12"]["cpu_baseline"] = {"seconds": cpu_s, "kind": "oracle", "cores": 1,
                                      "sample": "the whole N = 12 natural-order search, numpy"}
    return res


def oracle_matrix(name: str):
    from oracle import matrices as M

    return (2 * M.T_LO).astype("int64") if name == "LOx2" else M.NAMED[name]


def cpu_oracle_rate(planes_host, budget_s: float, transform: str = "T1", threads: int = 0,
                    sses: dict | None = None):
    """Run the oracle over host planes with `threads` threads (0: one per
    core) until the budget is spent; returns (blocks/s, blocks done, threads,
    planes done).  `sses`, if given, receives {sample position: SSE}."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import codec as oc

    oc.lib()
    T = oracle_matrix(transform)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    done_blocks = 0
    done_planes = 0
    lock = threading.Lock()
    idx = [0]

    def worker():
        nonlocal done_blocks, done_planes
        while True:
            with lock:
                if idx[0] >= len(planes_host) or time.perf_counter() - t0 > budget_s:
                    return
                i = idx[0]
                idx[0] += 1
            img, r = planes_host[i]
            got = oc.codec_plane(img, T, r)[0]
            nb = ((img.shape[0] + 7) // 8) * ((img.shape[1] + 7) // 8)
            with lock:
                done_blocks += nb
                done_planes += 1
                if sses is not None:
                    sses[i] = int(got)

    threads = max(1, min(threads or cores, len(planes_host)))
    with ThreadPoolExecutor(threads) as ex:
        for f in [ex.submit(worker) for _ in range(threads)]:
            f.result()
    dt = time.perf_counter() - t0
    return done_blocks / dt, done_blocks, threads, done_planes


def sample_indices(n: int, max_planes: int) -> list:
    return list(range(0, n, max(1, n // max_planes)))[:max_planes]


def host_sample(wl, max_planes: int):
    """Copy an evenly spaced sample of the workload's planes to host memory."""
    return [(wl.planes[i][0].cpu().numpy(), wl.planes[i][1])
            for i in sample_indices(len(wl.planes), max_planes)]


def main():
    args = parse()
    if args.impl == "reference":
        return main_reference(args)
    import torch  # noqa: F401

    backend = "nccl" if args.gpus > 1 or int(os.environ.get("WORLD_SIZE", "1")) > 1 else "gloo"
    dist = Dist(backend)
    out = {}
    wl = time_ours(args, dist, out)
    if dist.rank == 0 and dist.world == 1 and not args.no_configs and \
            args.workload == "batch_1024x1024" and args.transform == "T1":
        import torch

        out["configs"] = time_configs(args, torch.cuda.current_stream())
    if dist.rank == 0 and not args.no_search:
        out["search"] = time_search(args.no_cpu_baseline or dist.world > 1)
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        idx = sample_indices(len(wl.planes), 256)
        sample = host_sample(wl, 256)
        sses = {}
        rate, nb, cores, npl = cpu_oracle_rate(sample, args.cpu_seconds, args.transform,
                                               sses=sses)
        rate1, nb1, _, npl1 = cpu_oracle_rate(sample, args.cpu_seconds_single, args.transform,
                                              threads=1)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{npl} of {len(wl.planes)} planes ({nb} blocks), "
                                         f"C oracle (int64 definition), one thread per core",
                               "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                                               "sample": f"{npl1} planes ({nb1} blocks)"}}
        # the bit-exactness claim, checked on the run that was timed: the
        # oracle's SSE of every sampled plane against the timed plan's SSE
        bad = [idx[k] for k, v in sses.items() if int(wl.sse_host[idx[k]]) != v]
        out["parity"] = {"planes": len(sses), "mismatches": len(bad),
                         "first_mismatch": bad[0] if bad else None,
                         "check": "per-plane SSE of the timed run vs the C oracle (int64 "
                                  "definition), planes of the cpu_baseline sample"}
    if dist.rank == 0:
        print(json.dumps(out))
    dist.close()


def main_reference(args):
    """The oracle as it stands, timed on host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch

    from oracle import codec as oc

    oc.lib()
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    wl = Workload(args.workload, dev, args.images)
    # every plane of the workload: a step is one pass over the whole workload
    # when the per-step budget allows it (about 1.2 s on 16 host cores for
    # the 1024 images), else the planes the budget covers
    sample = host_sample(wl, len(wl.planes))
    per_step_budget = max(2.0, 240.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_oracle_rate(sample, per_step_budget, args.transform)
    rates, blocks, cores, planes = [], 0, 1, 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rate, nb, cores, npl = cpu_oracle_rate(sample, per_step_budget, args.transform)
        rates.append(rate)
        blocks += nb
        planes += npl
    wall = time.perf_counter() - t0
    value = blocks / wall
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {**wl.desc, "transform": args.transform, "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{planes / max(1, args.steps):.0f} of the workload's "
                                   f"{len(sample)} planes per step ({per_step_budget:.1f} s "
                                   f"budget per step)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
