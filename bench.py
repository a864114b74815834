"""Benchmark of the fused RDCT path (forward, zonal compression with the S
scaling, inverse, squared error) on GB300.

Default workload (one step = one pass of the whole path over the batch):
600 synthetic 3840x2160 YUV 4:2:0 frames (1/f^2 luma, 1/f^3 chroma at half
resolution, AR(1) drift), r = 16, uint8 reconstruction of every plane plus
per-frame SSE, all 1800 planes in one graph-captured persistent launch.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused RDCT fwd+compress+inv Gpixel/s and % HBM peak; serving p50/p99 latency"
UNIT = "Gpixel/s"

# DRAM bytes (read + write) per sample of the fused kernel, from the ncu capture summarised in
# profiles/fused_video_40x4k_r16_ncu.md.  Reported only while the kernel sources still hash to
# the value they had when the counters were taken.
FUSED_TRAFFIC = {"sources_sha256_16": "b046a7775fe44c3f", "bytes_per_sample": 1.9066}
FUSED_SOURCES = ["rdct_fused2.cuh", "rdct_device.cuh", "rdct_blocks.cuh", "rdct_fused2_launch.cu"]


def fused_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in FUSED_SOURCES:
        with open(os.path.join(ROOT, "paper_1402_6034_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-single", action="store_true", help="skip the single 512 x 512 image latency")
    ap.add_argument("--workload", choices=["video", "batch512", "uneven", "sweep", "variants"], default="video")
    ap.add_argument("--frames", type=int, default=600)
    ap.add_argument("--r", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--no-autotune", action="store_true",
                    help="uneven workload: the default launch shape instead of the autotuner's")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the r table, the uneven batch, the r sweep and the separate steps")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------- multi-rank

def max_over_ranks(x: float, device) -> float:
    """The largest value over all ranks (the slowest rank's time); x itself on one rank.
    Ends with a barrier so no rank starts later work before the others finished timing."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def weak_scaling_value(samples_per_rank: int, steps: int, ms_max: float, world: int) -> float:
    """Whole-job Gpixel/s: every rank processed its own copy of the workload `steps` times; the
    job took as long as the slowest rank."""
    return world * samples_per_rank * steps / (ms_max / 1000.0) / 1e9


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms with host timestamps; kept for a window."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            import threading
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        rows = []
        for ts, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((ts, float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        inside = [r for r in rows if t0 <= r[0] <= t1 + 0.25]
        note = "samples inside the timed region"
        if not inside and rows:
            inside = sorted(rows, key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))[:3]
            note = "no sample fell inside the timed region; nearest samples"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        names = ["active_mask", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in inside:
            for n, v in zip(names[1:], r[3][1:]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted(reasons), "samples": len(inside), "note": note}


# --------------------------------------------------------------- workloads

def video_config(frames: int, r: int) -> dict:
    """The `config` of the video workload (shared by both bench arms)."""
    samples = frames * (3840 * 2160 + 2 * 1920 * 1080)
    return {"workload": f"video_yuv420_{frames}x3840x2160_r{r}", "frames": frames, "planes_per_frame": 3, "r": r,
            "luma": "3840x2160 1/f^2", "chroma": "2x1920x1080 1/f^3", "samples_per_step": samples,
            "outputs": "uint8 reconstruction of every plane + per-frame SSE",
            "l2": f"inputs and outputs (2 x {samples / 1e9:.2f} GB) "
                  + ("larger than L2; no flush needed" if samples > 129e6 else "within L2"),
            "launch": f"one CUDA-graph launch per step (persistent kernel over all {3 * frames} planes)"}


def batch512_config(r: int) -> dict:
    """The `config` of the 1024 x 512 x 512 batch workload (shared by both bench arms)."""
    return {"workload": f"batch_1024x512x512_r{r}", "images": 1024, "r": r, "samples_per_step": 1024 * 512 * 512,
            "l2": "inputs and outputs (2 x 268 MB) larger than L2; no flush needed"}


class VideoWorkload:
    def __init__(self, frames: int, r: int, dev):
        from paper_1402_6034_gb300 import rdct, synth
        self.rdct = rdct
        self.frames, self.r = frames, r
        Y, U, V = synth.video_yuv420(frames, 2160, 3840, seed=0, device=str(dev))
        self.planes = (Y, U, V)
        self.out = tuple(torch.empty_like(p) for p in self.planes)
        jobs = []
        for f in range(frames):
            for p, o in zip(self.planes, self.out):
                jobs.append(rdct.BatchJob(p[f], o[f], r, f))
        self.jobs = jobs
        self.samples = sum(p.numel() for p in self.planes)
        self.nimages = frames
        self.plan = rdct.BatchPlan(jobs, frames)
        self.sse = torch.empty(frames, dtype=torch.float64, device=dev)
        self.config = video_config(frames, r)
        self.name = self.config["workload"]
        assert self.config["samples_per_step"] == self.samples
        self.kernels_per_step = 2  # fused batch kernel (one r class) + SSE finalize

    def step(self, stream):
        self.plan.run(self.sse, stream)

    def quality(self):
        mse = self.sse.cpu().numpy() / (self.samples / self.frames)
        return {"mean_psnr_db": float(np.mean(10 * np.log10(255.0 ** 2 / mse)))}

    def host_jobs(self, pinned: bool = True):
        """Host copies (pinned, or plain pageable memory) of the inputs and outputs for the end-to-end path."""
        from paper_1402_6034_gb300.rdct import HostJob
        hin = [torch.empty(p.shape, dtype=torch.uint8, pin_memory=pinned) for p in self.planes]
        hout = [torch.empty(p.shape, dtype=torch.uint8, pin_memory=pinned) for p in self.planes]
        for h, p in zip(hin, self.planes):
            h.copy_(p)
        arr = (HostJob * (3 * self.frames))()
        k = 0
        for f in range(self.frames):
            for h, o in zip(hin, hout):
                arr[k] = HostJob(h[f].data_ptr(), o[f].data_ptr(), h.shape[2], h.shape[2], h.shape[1], self.r, f)
                k += 1
        return (hin, hout), arr

    def cpu_planes(self):
        """The workload's planes in order, copied to host one at a time."""
        for f in range(self.frames):
            for p in self.planes:
                yield p[f].cpu().numpy()


class Batch512Workload(VideoWorkload):
    """1024 synthetic 512x512 1/f^2 images at one r (r = 10)."""

    def __init__(self, frames: int, r: int, dev):
        from paper_1402_6034_gb300 import rdct, synth
        self.rdct = rdct
        n = 1024
        self.frames, self.r = n, r
        imgs = torch.from_numpy(synth.image_batch(64, 512, 512, 2.0, 0)).to(dev)
        imgs = imgs.repeat(n // 64, 1, 1).contiguous()
        self.planes = (imgs,)
        self.out = (torch.empty_like(imgs),)
        self.jobs = [rdct.BatchJob(imgs[i], self.out[0][i], r, i) for i in range(n)]
        self.samples = imgs.numel()
        self.nimages = n
        self.plan = rdct.BatchPlan(self.jobs, n)
        self.sse = torch.empty(n, dtype=torch.float64, device=dev)
        self.config = batch512_config(r)
        self.name = self.config["workload"]
        self.kernels_per_step = 2

    def host_jobs(self, pinned: bool = True):
        from paper_1402_6034_gb300.rdct import HostJob
        hin = [torch.empty(self.planes[0].shape, dtype=torch.uint8, pin_memory=pinned)]
        hout = [torch.empty(self.planes[0].shape, dtype=torch.uint8, pin_memory=pinned)]
        hin[0].copy_(self.planes[0])
        arr = (HostJob * self.frames)()
        for i in range(self.frames):
            arr[i] = HostJob(hin[0][i].data_ptr(), hout[0][i].data_ptr(), 512, 512, 512, self.r, i)
        return (hin, hout), arr



def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), and its architecture."""
    import platform
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        name = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return f"{name or 'unknown'} ({platform.machine()}, {os.cpu_count()} logical CPUs)"


def cpu_oracle_rate(planes_iter, r: int, budget_s: float, threads: int = 0):
    """Times the FP64 oracle over planes until budget_s has passed (threads 0: all host threads)."""
    from oracle import oracle as orc
    threads = threads or orc.max_threads()
    done, t_total = 0, 0.0
    for img in planes_iter:
        t = time.perf_counter()
        orc.fused(img, r, want_xhat=False, want_u8=True, nthreads=threads)
        t_total += time.perf_counter() - t
        done += img.size
        if t_total >= budget_s:
            break
    return done / t_total / 1e9, threads, done, t_total


# ------------------------------------------------------- uneven / sweep modes

def host_link_rate(dev, nbytes: int = 1 << 30, reps: int = 5) -> float:
    """GB/s each way of plain pinned-host <-> device copies running at the same time on two streams: the
    ceiling for any end-to-end path that moves every input in and every output out."""
    hin = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    hout = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    din = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    dout = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def both():
        with torch.cuda.stream(s1):
            din.copy_(hin, non_blocking=True)
        with torch.cuda.stream(s2):
            hout.copy_(dout, non_blocking=True)

    both()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        both()
    torch.cuda.synchronize()
    return nbytes / ((time.perf_counter() - t) / reps) / 1e9


def single_image_latency(dev, r: int = 10, reps: int = 200) -> dict:
    """One 512 x 512 image at r = 10 (L2-resident): rdct_fused (forward, keep r, inverse, uint8 output,
    exact SSE) back to back on a stream (CUDA events), and one call at a time with a synchronize after each
    (host wall clock, launch included)."""
    from paper_1402_6034_gb300 import rdct, synth
    img = torch.from_numpy(synth.image_1f(512, 512, alpha=2.0, seed=0)).to(dev)
    out = torch.empty_like(img)
    sse = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    us = events_time(lambda: rdct.fused(img, r, out_u8=out, sse=sse, stream=stream), reps, 10, stream) * 1e3
    walls = []
    for _ in range(reps):
        t = time.perf_counter()
        rdct.fused(img, r, out_u8=out, sse=sse, stream=stream)
        torch.cuda.synchronize()
        walls.append((time.perf_counter() - t) * 1e6)
    mse = float(sse.item()) / img.numel()
    return {"image": "512x512 uint8, r = 10", "device_us_per_call": us,
            "wall_us_per_call_p50": statistics.median(walls), "psnr_db": 10 * math.log10(255.0 ** 2 / mse)}


def events_time(fn, steps, warmup, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def bench_uneven(args, dev):
    """4096 images, sides uniform over multiples of 8 in [64, 2048], 1 or 3 planes, r from {4, 10, 16, 32}:
    one graph-captured launch per step (autotuned) vs one plain launch per plane."""
    from paper_1402_6034_gb300 import rdct, synth
    n = 4096
    specs = synth.uneven_specs(n, seed=0)
    pool = synth.field_u8_torch(2048, 2048, 2.0, 0, device=str(dev), planes=4)
    rng = np.random.Generator(np.random.PCG64(1))
    sizes = [sp.w * sp.h for sp in specs for _ in range(sp.planes)]
    total = sum(sizes)
    src_buf = torch.empty(total, dtype=torch.uint8, device=dev)
    dst_buf = torch.empty(total, dtype=torch.uint8, device=dev)
    jobs, off = [], 0
    for i, sp in enumerate(specs):
        for p in range(sp.planes):
            k = int(rng.integers(0, 4))
            y0, x0 = int(rng.integers(0, 2048 - sp.h + 1)), int(rng.integers(0, 2048 - sp.w + 1))
            src = src_buf[off:off + sp.w * sp.h].view(sp.h, sp.w)
            src.copy_(pool[k, y0:y0 + sp.h, x0:x0 + sp.w])
            jobs.append(rdct.BatchJob(src, dst_buf[off:off + sp.w * sp.h].view(sp.h, sp.w), sp.r, i))
            off += sp.w * sp.h
    tune = None if getattr(args, "no_autotune", False) else rdct.autotune(jobs, n)
    plan = rdct.BatchPlan(jobs, n, tune=tune)
    tune = plan.tune
    sse_g = torch.empty(n, dtype=torch.float64, device=dev)
    sse_p = torch.empty(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    ms_graph = events_time(lambda: plan.run(sse_g, stream), args.steps, args.warmup, stream)
    ms_plain = events_time(lambda: plan.run_per_plane(sse_p, stream), max(3, args.steps // 10), 2, stream)
    identical = bool(torch.equal(sse_g, sse_p))
    npix = torch.tensor([sp.w * sp.h * sp.planes for sp in specs], dtype=torch.float64, device=dev)
    psnr = 10 * torch.log10(255.0 ** 2 / (sse_g / npix))
    peak, kind = peaks()
    alg = 2 * total + 8 * n
    kernels = plan.kernels_per_run()  # one per r present and staging form, plus the error conversion
    return {"metric": METRIC, "value": total / (ms_graph / 1e3) / 1e9, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "uneven_4096_images_64to2048_r4-10-16-32", "images": n, "planes": len(jobs),
                       "samples_per_step": total, "tune": tune,
                       "l2": f"inputs and outputs (2 x {total / 1e9:.2f} GB) larger than L2"},
            "roofline": {"bound": "hbm", "achieved": alg / (ms_graph / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (ms_graph / 1e3) / 1e9 / peak, "traffic": None,
                         "peak_source": f"{kind} hbm_gbs"},
            "gpu_launches": kernels * args.steps,
            "per_plane_launches": {"value": total / (ms_plain / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms_plain,
                                   "launches_per_step": len(jobs) + 1},
            "batched_over_per_plane": ms_plain / ms_graph, "sse_identical": identical,
            "quality": {"mean_psnr_db": float(psnr.mean())}}


def sweep_images(dev, n: int = 1024) -> torch.Tensor:
    """[n, 512, 512] uint8 1/f^2 images: 64 seeded fields, each also taken at n / 64 - 1 block-aligned
    circular shifts (distinct block contents per image)."""
    from paper_1402_6034_gb300 import synth
    base = torch.from_numpy(synth.image_batch(64, 512, 512, 2.0, 0)).to(dev)
    return torch.cat([torch.roll(base, shifts=(8 * k, 8 * ((k * 7) % 64)), dims=(1, 2)) for k in range(n // 64)])


def bench_sweep(args, dev):
    """1024 images of 512 x 512, r = 1..64 for the RDCT and the exact DCT: one energy pass per transform
    (rdct_sweep_noalloc, the allocation-free form of rdct_sweep: the same kernels, with its descriptor tables
    in the library's fixed array), per-r average MSE / PSNR and the MSE absolute percentage error against
    the DCT."""
    from paper_1402_6034_gb300 import rdct
    n = 1024
    imgs = sweep_images(dev, n)
    planes = rdct.plane_array(imgs)
    out_r = torch.empty((n, 64), dtype=torch.float64, device=dev)
    out_d = torch.empty((n, 64), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        rdct.sweep_noalloc(planes, out_r, rdct.KIND_RDCT, stream)
        rdct.sweep_noalloc(planes, out_d, rdct.KIND_DCT, stream)

    ms = events_time(step, args.steps, args.warmup, stream)
    mse_r = (out_r / (512 * 512)).mean(0).cpu().numpy()
    mse_d = (out_d / (512 * 512)).mean(0).cpu().numpy()
    ps_r = (10 * torch.log10(255.0 ** 2 / (out_r / (512 * 512)))).cpu().numpy()
    ps_d = (10 * torch.log10(255.0 ** 2 / (out_d / (512 * 512)))).cpu().numpy()
    rows = {}
    n_uqi = 64  # UQI needs the reconstruction itself: a 64-image subset, one fused + one UQI launch each
    for r in (1, 5, 10, 16, 32, 45, 63):
        q = {}
        for kind in (rdct.KIND_RDCT, rdct.KIND_DCT):
            acc = torch.zeros((), dtype=torch.float64, device=dev)
            for i in range(n_uqi):
                rec = rdct.fused(imgs[i], r, kind, stream=stream)[0]
                acc += rdct.uqi(imgs[i], rec, stream=stream)
            q[kind] = acc.item() / n_uqi
        rows[str(r)] = {"psnr_rdct": float(np.mean(ps_r[:, r - 1])), "psnr_dct": float(np.mean(ps_d[:, r - 1])),
                        "mse_rdct": float(mse_r[r - 1]), "mse_dct": float(mse_d[r - 1]),
                        "mse_ape_pct": float(100 * abs(mse_r[r - 1] - mse_d[r - 1]) / mse_d[r - 1]),
                        "uqi_rdct": q[rdct.KIND_RDCT], "uqi_dct": q[rdct.KIND_DCT],
                        "uqi_ape_pct": float(100 * abs(q[rdct.KIND_RDCT] - q[rdct.KIND_DCT]) / q[rdct.KIND_DCT])}
    uqi_ms = events_time(lambda: rdct.uqi(imgs[0], imgs[1], stream=stream), 20, 3, stream)
    total = n * 512 * 512 * 2  # two transforms per step
    peak, kind = peaks()
    # beside the sweep: the direct fused path at r = 10 on the same images (one batch-plan launch; uint8
    # reconstruction and per-image SSE: 2 B per sample + 8 B per image)
    rec = torch.empty_like(imgs)
    plan10 = rdct.BatchPlan([rdct.BatchJob(imgs[i], rec[i], 10, i) for i in range(n)], n)
    sse10 = torch.empty(n, dtype=torch.float64, device=dev)
    ms10 = events_time(lambda: plan10.run(sse10, stream), args.steps, args.warmup, stream)
    bytes10 = 2 * n * 512 * 512 + 8 * n
    fused10 = {"ms": ms10, "gpixel_s": n * 512 * 512 / (ms10 / 1e3) / 1e9,
               "frac": bytes10 / (ms10 / 1e3) / 1e9 / peak, "algorithmic_bytes": bytes10,
               "mean_psnr_db": float(torch.mean(10 * torch.log10(255.0 ** 2 / (sse10 / (512 * 512)))).item())}
    del plan10, rec
    return {"metric": METRIC, "value": total / (ms / 1e3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32 (RDCT) + f16 MMA, f32 accumulate (DCT)", "data": "synthetic",
            "config": {"workload": "sweep_1024x512x512_r1-64_rdct_and_dct", "images": n,
                       "samples_per_step": total, "note": "one pass per transform, 1 B/px read"},
            "roofline": {"bound": "hbm", "achieved": total / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": total / (ms / 1e3) / 1e9 / peak, "traffic": None, "peak_source": f"{kind} hbm_gbs",
                         "limiter": "not DRAM: both passes need all 63 AC coefficients of every block. RDCT pass "
                                    "(per-block kernel) issue-bound, 63 % of issue slots busy, DRAM read 2.9 TB/s; "
                                    "DCT pass (tensor cores) bound by each tile's chain of tensor-memory stores, "
                                    "MMAs and loads back, tensor pipe 38 % busy, DRAM read 3.3 TB/s"},
            "gpu_launches": 6 * args.steps, "per_r": rows, "fused_r10_batch": fused10,
            "uqi_kernel": {"image": "512x512 u8", "us": uqi_ms * 1e3,
                           "windows_per_s": 505 * 505 / (uqi_ms / 1e3), "uqi_subset_images": n_uqi}}


def variant_ops_per_block(r: int) -> int:
    """FP32 operations the variant kernel needs per 8x8 block at r (one FMA or add = 1): forward row pass
    (8 rows x K kept columns x 8), column pass over the kept zone (zone x 8), inverse (8 x zone, then
    64 x K), squared error (64 subtractions + 64 FMAs).  D is the anti-diagonal class of r, K = min(D+1, 8)."""
    zz = sorted(((i + j, i if (i + j) % 2 else j, i, j) for i in range(8) for j in range(8)))
    d = zz[r - 1][0]
    k = min(d + 1, 8)
    zone = sum(1 for i in range(8) for j in range(8) if i + j <= d)
    return 8 * k * 8 + zone * 8 + 8 * zone + 64 * k + 128


def bench_variants(args, dev):
    """The other transforms of the paper (signed DCT, ceil(2C) polar variant, sign(C) polar, and C_orth
    through the same general kernel) on the 1024 x 512^2 batch at r = 10, timed as one tall plane per call;
    average PSNR and UQI per variant over a 64-image subset at several r."""
    from paper_1402_6034_gb300 import rdct
    n, r = 1024, 10
    imgs = sweep_images(dev, n)
    tall = imgs.view(n * 512, 512)
    out = torch.empty_like(tall)
    sse = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    names = ["round", "ceil", "sdct", "sdct_polar"]
    per = {}
    clock = 2070.0
    ops_px = variant_ops_per_block(r) / 64.0
    for name in names:
        v = rdct.VARIANTS[name]
        p = rdct.plane_of(tall)
        o = rdct.Out(out.data_ptr(), None, 512, 0)
        lib = rdct.load()

        def step():
            rdct._check(lib.rdct_fused_variant(ctypes.byref(p), r, v, ctypes.byref(o), sse.data_ptr(),
                                               stream.cuda_stream), "rdct_fused_variant")

        ms = events_time(step, args.steps, args.warmup, stream)
        gpx = n * 512 * 512 / (ms / 1e3) / 1e9
        per[name] = {"gpixel_s": gpx, "ms": ms, "psnr_db_of_batch_mse": float(10 * np.log10(255.0 ** 2 * n * 512 * 512
                                                                                          / sse.item()))}
    quality = {}
    for rr in (5, 10, 16, 32, 45):
        row = {}
        for name in names:
            ps, qs = [], []
            for i in range(64):
                u8, _, s1 = rdct.fused_variant(imgs[i], rr, rdct.VARIANTS[name], stream=stream)
                ps.append(10 * torch.log10(255.0 ** 2 * 512 * 512 / s1))
                qs.append(rdct.uqi(imgs[i], u8, stream=stream))
            row[name] = {"psnr_db": float(torch.stack(ps).mean()), "uqi": float(torch.stack(qs).mean())}
        quality[str(rr)] = row
    peak = 152 * 128 * clock * 1e6 / 1e12  # FP32 lane-operations per second, in T/s
    achieved = per["ceil"]["gpixel_s"] * 1e9 * ops_px / 1e12
    return {"metric": METRIC, "value": per["ceil"]["gpixel_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per["ceil"]["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
            "config": {"workload": "variants_1024x512x512_r10", "images": n, "r": r,
                       "timed": "one rdct_fused_variant call on the batch as one 512 x 524288 plane",
                       "value_is": "ceil(2C) polar variant"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": None,
                         "ops_per_pixel": ops_px,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2070 MHz (one FMA = one op)"},
            "gpu_launches": 2 * args.steps, "per_variant": per, "quality_64_images": quality}


# ------------------------------------------------------------------ serving

def serving_bench(dev, n_requests: int = 2000, rates=(250.0, 500.0, 1000.0, 2000.0, 4000.0, 0.0), seed: int = 0,
                  budget: int = 1 << 30):
    """Poisson arrivals of images (side log-uniform 256..4096, 1 or 3 planes, r ~ U{1..64}) against
    the continuous-batching server and against one launch per image (max_batch 1, one stream), both
    with the same device budget (small enough that admission binds when requests pile up).
    Rate 0 submits everything at once (saturation).  Requests are windows of one pinned 3 x 4096 x 4096
    field (rows 4096 bytes apart), and their reconstructions go to the same windows of one pinned output
    field, so thousands of requests need no per-request host buffers."""
    from paper_1402_6034_gb300 import rdct, synth
    pool = synth.field_u8_torch(4096, 4096, 2.0, seed, device=str(dev), planes=3).cpu().pin_memory()
    out_pool = torch.empty_like(pool).pin_memory()
    trace = synth.poisson_trace(1.0, n_requests, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    reqs = []
    for q in trace:
        y0 = 8 * int(rng.integers(0, (4096 - q.side) // 8 + 1))
        x0 = 8 * int(rng.integers(0, (4096 - q.side) // 8 + 1))
        src = pool[:q.planes, y0:y0 + q.side, x0:x0 + q.side]
        dst = out_pool[:q.planes, y0:y0 + q.side, x0:x0 + q.side]
        reqs.append((src, dst, q.r, q.t))
    samples = sum(src.numel() for src, _, _, _ in reqs)
    # warm the library and the device once: one small request for every r, so that the first launch of
    # each per-r kernel (and its module load) falls outside the timed runs
    small = torch.from_numpy(synth.image_1f(64, 64, alpha=2.0, seed=seed)).pin_memory()
    small_out = torch.empty_like(small).pin_memory()
    for kw in (dict(max_batch=64, streams=2), dict(max_batch=1, streams=1)):
        w = rdct.Server(device_budget_bytes=1 << 28, **kw)
        for tk in [w.submit(small, r, small_out) for r in range(1, 65)]:
            w.wait(tk)
        w.close()
    rows = []
    for rate in rates:
        row = {"rate_req_s": rate if rate else "saturation"}
        errs = {}
        for name, kw in (("served", dict(max_batch=64, streams=2)), ("plain", dict(max_batch=1, streams=1))):
            srv = rdct.Server(device_budget_bytes=budget, queue_capacity=n_requests + 1, **kw)
            t0 = time.perf_counter()
            tickets = []
            for src, dst, r, t in reqs:
                if rate:
                    target = t0 + t / rate
                    while True:
                        now = time.perf_counter()
                        if now >= target:
                            break
                        if target - now > 2e-3:
                            time.sleep(target - now - 1e-3)
                tickets.append(srv.submit(src, r, dst))
            res = [srv.wait(tk) for tk in tickets]
            st = srv.stats()
            srv.close()
            errs[name] = [(x["sse"], x["sse_u8"]) for x in res]
            psnrs = [x["psnr"] for x in res if math.isfinite(x["psnr"])]
            psnrs8 = [x["psnr_u8"] for x in res if math.isfinite(x["psnr_u8"])]
            row[name] = {"p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3,
                         "p999_ms": st["p999_us"] / 1e3, "mean_ms": st["mean_us"] / 1e3,
                         "gpixels_per_s": st["gpixels_per_s"], "launches": st["batches"],
                         "peak_resident_bytes": st["peak_resident_bytes"], "rejected": st["rejected"],
                         "mean_psnr_db": float(np.mean(psnrs)) if psnrs else None,
                         "mean_psnr_u8_db": float(np.mean(psnrs8)) if psnrs8 else None}
        row["sse_identical"] = errs["served"] == errs["plain"]
        rows.append(row)
    return {"requests": n_requests, "samples": samples, "sides": "log-uniform 256..4096, square",
            "planes": "1 or 3", "r": "uniform 1..64", "host_buffers": "pinned, windows of one field",
            "budget_bytes": budget,
            "served": f"max_batch 64, 2 compute streams, {budget >> 20} MiB device budget",
            "plain": "one launch per image (max_batch 1, 1 stream), same budget, admission and copies",
            "latency": "submit to completion (C++ steady clock)", "rates": rows}


def fused_r_table(wl, rs, steps, warmup, dev):
    """The default workload's fused path at other r: one graph launch per step over all planes."""
    from paper_1402_6034_gb300 import rdct
    peak, kind = peaks()
    stream = torch.cuda.current_stream()
    rows = {}
    for r in rs:
        jobs = [rdct.BatchJob(j.src, j.dst, r, j.image) for j in wl.jobs]
        plan = rdct.BatchPlan(jobs, wl.nimages)
        sse = torch.empty(wl.nimages, dtype=torch.float64, device=dev)
        ms = events_time(lambda: plan.run(sse, stream), steps, warmup, stream)
        alg = 2 * wl.samples + 8 * wl.nimages
        mse = sse.cpu().numpy() / (wl.samples / wl.nimages)
        rows[str(r)] = {"gpixel_s": wl.samples / (ms / 1e3) / 1e9, "ms": ms,
                        "frac": alg / (ms / 1e3) / 1e9 / peak, "kernels_per_step": plan.kernels_per_run(),
                        "form": "dropped coefficients" if r > 35 else "kept coefficients",
                        "mean_psnr_db": float(np.mean(10 * np.log10(255.0 ** 2 / np.maximum(mse, 1e-300))))}
        plan.close()
    return {"workload": wl.name.replace(f"_r{wl.r}", "_r*"), "peak_source": f"{kind} hbm_gbs", "steps": steps,
            "per_r": rows}


def bench_steps(dev, steps: int, warmup: int, r: int = 10):
    """The separate calls of the method (rdct_forward, rdct_compress, rdct_inverse, rdct_mse_psnr) on the
    1024 x 512^2 batch taken as one 512 x 524288 plane, each against its algorithmic bytes."""
    from paper_1402_6034_gb300 import rdct
    peak, kind = peaks()
    imgs = sweep_images(dev, 1024)
    tall = imgs.view(1024 * 512, 512)
    npx = tall.numel()
    nblk = npx // 64
    stream = torch.cuda.current_stream()
    Y = rdct.forward(tall, stream)
    Yc = rdct.compress(Y, r, stream)
    rec = rdct.inverse(Yc, 512 // 8, 1024 * 512 // 8, r, stream=stream)[0]
    calls = {
        "rdct_forward": (lambda: rdct.forward(tall, stream), 5 * npx, "1 B read + 4 B int32 write per pixel"),
        "rdct_compress": (lambda: rdct.compress(Y, r, stream), (256 + 4 * r) * nblk,
                          f"256 B read + {4 * r} B write per block (r = {r})"),
        "rdct_inverse": (lambda: rdct.inverse(Yc, 512 // 8, 1024 * 512 // 8, r, stream=stream), (4 * r + 64) * nblk,
                         f"{4 * r} B read + 64 B uint8 write per block"),
        "rdct_mse_psnr": (lambda: rdct.mse_psnr(tall, rec, stream), 2 * npx, "2 B read per pixel (uint8 pair)"),
    }
    out = {}
    for name, (fn, nbytes, what) in calls.items():
        ms = events_time(fn, steps, warmup, stream)
        out[name] = {"ms": ms, "algorithmic_bytes": nbytes, "bytes": what, "GBs": nbytes / (ms / 1e3) / 1e9,
                     "frac": nbytes / (ms / 1e3) / 1e9 / peak}
    del Y, Yc, rec
    return {"image": "1024 x 512^2 batch as one 512 x 524288 plane", "r": r, "peak_source": f"{kind} hbm_gbs",
            "note": "each call includes its allocation of the output tensor (torch caching allocator)",
            "calls": out}


# ---------------------------------------------------------------- reference

def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_1402_6034_gb300 import synth
    orc.build()
    frames_needed = max(1, min(args.steps + args.warmup, 4))
    if args.workload == "video":
        Y, U, V = synth.video_yuv420(frames_needed, 2160, 3840, seed=0, device="cpu")
        samples = [[Y[f].numpy(), U[f].numpy(), V[f].numpy()] for f in range(frames_needed)]
        config = video_config(args.frames, args.r)
        sample_desc = "one 3840x2160 YUV 4:2:0 frame (3 planes) per step, cycling over the first frames"
    elif args.workload == "batch512":
        imgs = synth.image_batch(frames_needed, 512, 512, 2.0, 0)
        samples = [[imgs[f]] for f in range(frames_needed)]
        config = batch512_config(args.r)
        sample_desc = "one 512x512 image per step"
    else:
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm times the video and batch512 "
                                                             f"workloads, not {args.workload}"}), flush=True)
        return
    threads = orc.max_threads()

    def one(k):
        n = 0
        for img in samples[k % len(samples)]:
            orc.fused(img, args.r, want_xhat=False, want_u8=True, nthreads=threads)
            n += img.size
        return n

    for k in range(args.warmup):
        one(k)
    t = time.perf_counter()
    n = 0
    for k in range(args.steps):
        n += one(k)
    dt = time.perf_counter() - t
    value = n / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample_desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- main

def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1402_6034_gb300 import rdct
    rdct.load()

    if args.workload in ("uneven", "sweep", "variants"):
        line = {"uneven": bench_uneven, "sweep": bench_sweep, "variants": bench_variants}[args.workload](args, dev)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    wl = (VideoWorkload if args.workload == "video" else Batch512Workload)(args.frames, args.r, dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        wl.step(stream)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(local) if rank == 0 else None
    time.sleep(0.5 if sampler else 0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        wl.step(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    time.sleep(0.3 if sampler else 0)
    clocks = sampler.summary(t0, t1) if sampler else None
    if sampler:
        sampler.stop()
    quality = wl.quality()

    ms_step = ms / args.steps
    value = weak_scaling_value(wl.samples, args.steps, ms, world)
    peak, peak_kind = peaks()
    alg_bytes = 2 * wl.samples + 8 * wl.nimages
    traffic = None
    if args.workload == "video" and fused_sources_hash() == FUSED_TRAFFIC["sources_sha256_16"]:
        traffic = FUSED_TRAFFIC["bytes_per_sample"] * wl.samples
    achieved = alg_bytes / (ms_step / 1000.0) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": wl.config,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "fused2_tma_kernel at r >= 16, fused2_kernel below (one graph step: SSE memset, "
                                   "kernel, SSE finalize)",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "peak_source": f"{peak_kind} hbm_gbs (copy)"},
            "gpu_launches": wl.kernels_per_step * args.steps, "clocks": clocks, "quality": quality}
    if args.workload == "video":
        line["frames_per_s"] = wl.frames / (ms_step / 1000.0)

    if not args.no_e2e:
        bufs, arr = wl.host_jobs()
        lib = rdct.load()

        def time_pipeline(mode, jobs_arr, budget=6 << 30, depth=3):
            """Mean seconds per step over e2e_steps after one untimed run (which, for outputs the host never
            touched, also faults their pages in: its time is returned too)."""
            pipe = ctypes.c_void_p()
            rdct._check(lib.rdct_pipeline_create(ctypes.c_int64(budget), depth, ctypes.byref(pipe)),
                        "rdct_pipeline_create")
            rdct._check(lib.rdct_pipeline_set_mode(pipe, mode), "rdct_pipeline_set_mode")
            sse_h = (ctypes.c_double * wl.nimages)()
            t = time.perf_counter()
            rdct._check(lib.rdct_pipeline_run(pipe, jobs_arr, len(jobs_arr), wl.nimages, sse_h, None),
                        "rdct_pipeline_run")  # warm
            first = time.perf_counter() - t
            t = time.perf_counter()
            for _ in range(args.e2e_steps):
                rdct._check(lib.rdct_pipeline_run(pipe, jobs_arr, len(jobs_arr), wl.nimages, sse_h, None),
                            "rdct_pipeline_run")
            dt = (time.perf_counter() - t) / args.e2e_steps
            lib.rdct_pipeline_destroy(pipe)
            return dt, bool(np.allclose(np.array(sse_h[:]), wl.sse.cpu().numpy(), rtol=0, atol=0)), first

        dt, ok, _ = time_pipeline(rdct.Pipeline.AUTO, arr)
        dt_s, ok_s, _ = time_pipeline(rdct.Pipeline.STAGED, arr, 2 << 30, 4)
        del bufs
        pg_bufs, arr_pg = wl.host_jobs(pinned=False)
        dt_p, ok_p, first_p = time_pipeline(rdct.Pipeline.AUTO, arr_pg)
        del pg_bufs
        link = host_link_rate(dev)
        line["e2e"] = {"value": world * wl.samples / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": wl.samples,
                       "d2h_bytes_per_step": wl.samples + 8 * wl.nimages, "ms_per_step": 1000 * dt,
                       "api": "rdct_pipeline_run on pinned host planes, direct mode: the fused kernels read and "
                              "write the host planes over the host link (no staging copies)",
                       "sse_matches_device_path": ok,
                       "host_link_GBs_each_way": link,
                       "staged": {"value": world * wl.samples / dt_s / 1e9, "ms_per_step": 1000 * dt_s,
                                  "api": "rdct_pipeline_run, staged mode (pinned planes, 4 slots of 256 MiB each "
                                         "way): copies into device slots overlapped with kernels on three streams",
                                  "sse_matches_device_path": ok_s},
                       "pageable": {"value": world * wl.samples / dt_p / 1e9, "ms_per_step": 1000 * dt_p,
                                    "first_run_ms": 1000 * first_p,
                                    "api": "rdct_pipeline_run (AUTO) on plain pageable host planes: direct mode, "
                                           "the kernels reach the pages through the host page tables on this "
                                           "device; the first run also faults in the fresh output pages",
                                    "sse_matches_device_path": ok_p}}

    if rank == 0 and args.workload == "video" and not args.no_extra:
        k = min(args.steps, 20)
        line["fused_r"] = fused_r_table(wl, (1, 4, 10, 16, 21, 32, 35, 36, 40, 45, 55, 63, 64), k, 3, dev)
        sub = argparse.Namespace(**{**vars(args), "steps": k, "warmup": 3})
        u = bench_uneven(sub, dev)
        line["uneven"] = {"workload": u["config"]["workload"], "value": u["value"], "unit": u["unit"],
                          "ms_per_step": u["ms_per_step"], "frac": u["roofline"]["frac"],
                          "achieved_GBs": u["roofline"]["achieved"], "planes": u["config"]["planes"],
                          "samples_per_step": u["config"]["samples_per_step"], "tune": u["config"]["tune"],
                          "kernels_per_step": u["gpu_launches"] // k,
                          "per_plane_launches": u["per_plane_launches"],
                          "batched_over_per_plane": u["batched_over_per_plane"],
                          "sse_identical": u["sse_identical"], "quality": u["quality"]}
        torch.cuda.empty_cache()
        sw = bench_sweep(sub, dev)
        line["sweep"] = {"workload": sw["config"]["workload"], "value": sw["value"], "unit": "Gsample/s",
                         "ms_per_step": sw["ms_per_step"], "frac": sw["roofline"]["frac"],
                         "per_r": {r: sw["per_r"][r] for r in ("1", "10", "16", "45") if r in sw["per_r"]},
                         "fused_r10_batch": sw["fused_r10_batch"],
                         "uqi_subset_images": sw["uqi_kernel"]["uqi_subset_images"]}
        line["steps_api"] = bench_steps(dev, k, 3)
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_serving:
        line["serving"] = serving_bench(dev, args.serving_requests)
    if rank == 0 and args.workload == "video" and not args.no_single:
        line["single_image_512_r10"] = single_image_latency(dev)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, threads, done, tt = cpu_oracle_rate(wl.cpu_planes(), args.r, args.cpu_seconds)
        rate1, _, done1, tt1 = cpu_oracle_rate(wl.cpu_planes(), args.r, args.cpu_seconds / 2, threads=1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "cpu_model": cpu_model(),
                                "sample": f"{done} samples = {100.0 * done / wl.samples:.0f}% of the same workload "
                                          f"(its planes in order, up to {args.cpu_seconds:.0f} s), {tt:.1f} s of "
                                          f"wall time on {threads} threads",
                                "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                                  "sample": f"{done1} samples (the first planes of the workload), "
                                                            f"{tt1:.1f} s"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
