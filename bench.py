#!/usr/bin/env python3
"""Throughput of the 4DGS rendering routine and its adjoint on one GB300.

One step = the whole hot path over one batch: fgs4d_slice_project ->
fgs4d_bin_sort -> fgs4d_render -> fgs4d_render_backward for every view of
the batch.  Workload (the one the headline metric is quoted on): 1M 4D
Gaussians with clustered means, SH degree 3 x 2 Fourier frequencies, a batch
of 20 cameras on a forward-facing arc at 1352x1014, each at its own time out
of 300 frames (seeded synthetic data standing in for Plenoptic-Video-like
scenes).  The parameters (644 MB) are larger than L2, so no flush is needed.

Precision (default ``mixed``): 4DSH coefficients stored in BF16 and conics
in 16-bit records, with FP32 arithmetic and accumulation; ``--precision fp32``
stores everything in FP32.

Printed: one JSON line.  ``value`` is forward+backward Mpix/s with inputs
resident in HBM, each step replayed as one CUDA graph (by default the views
as two groups on two streams inside it, ``--groups``); ``e2e`` is the same
step through the C ABI with host buffers (parameters and dL/dimage copied in,
image and gradients copied out inside the timed region).  ``stage_ms`` and
``fwd_mpix_s`` come from eager launches bracketed by events; ``batched_fp32``
is the whole batch in plain FP32 and ``single_view`` the plain FP32 path one
view per call, both on the same GPU.

``--impl reference`` times the FP64 CPU oracle instead (a bounded crop sample
of the same workload on the host cores).
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
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="4dgs-render-fwd+bwd", gaussians=1_000_000, clustered=True, sh_degree=3, n_freq=2,
                views=20, width=1352, height=1014, frames=300)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fgs4d", choices=["fgs4d", "reference"])
    ap.add_argument("--n", type=int, default=None, help="override the number of Gaussians (smoke runs)")
    ap.add_argument("--views", type=int, default=None)
    ap.add_argument("--scale", type=float, default=1.0, help="image scale (smoke runs only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-train", action="store_true", help="skip the training-step key of the default run")
    ap.add_argument("--no-aux", action="store_true", help="skip the depth/flow-map key of the default run")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the No-4DRot / static-3DGS stage times of the default run")
    ap.add_argument("--no-batching", action="store_true",
                    help="skip the uneven-batch key (300k Gaussians, 100 views, batched vs one by one)")
    ap.add_argument("--workload", default="render", choices=["render", "train"],
                    help="render: forward+backward of the 1M-Gaussian batch (the headline); train: the full "
                         "training step (loss, adjoint, Adam) on 3M Gaussians x 8 views")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32"],
                    help="mixed: BF16 4DSH coefficients + 16-bit conic records; fp32: plain FP32 storage")
    ap.add_argument("--no-graph", action="store_true", help="launch the timed steps eagerly, not as a CUDA graph")
    ap.add_argument("--groups", type=int, default=0,
                    help="view groups of the timed step, each on a stream of its own (1: one batch on one stream; "
                         "0: the autotuner times 1 and 2)")
    ap.add_argument("--tile", default="auto", choices=["auto", "16", "32"],
                    help="compositing tile side; auto: the autotuner times both on this workload")
    ap.add_argument("--bin-size", default="auto", choices=["auto", "16", "32", "64"],
                    help="binning tile side (a multiple of the compositing tile); auto: picked with the tile size")
    ap.add_argument("--batch-depth", default="auto", choices=["auto", "32", "64", "128", "256"],
                    help="splat records staged per shared-memory batch; auto: picked with the tile size")
    return ap.parse_args()


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi during the timed region (median SM clock, reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for nm, val in zip(names, r[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM traffic of the dominant kernel comes from a committed ncu summary; it is
# reported only while the kernel's sources hash to the value recorded there.
KERNEL_SOURCES = ("paper_2310_10642_gb300/csrc/render.cu", "paper_2310_10642_gb300/csrc/fgs4d_internal.cuh")
STAGE_PROFILE = {"render_backward_2d": "render_bwd_kernel_1M_2views_1352x1014.md",
                 "render": "render_fwd_kernel_1M_2views_1352x1014.md"}
# launch shape of those captures: their traffic applies to runs with this shape only
PROFILED_SHAPE = dict(tile_size=32, bin_size=64, batch_depth=256)


def profiled_traffic(stage: str):
    """(DRAM bytes per full-size launch, note) for a stage's kernel, or (None, why)."""
    import hashlib
    import re
    name = STAGE_PROFILE.get(stage)
    if not name:
        return None, "no ncu summary for this kernel"
    try:
        text = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None, f"profiles/{name} missing"
    fields = dict(re.findall(r"^\s*(sources_sha1|dram_bytes_per_launch_full_workload):\s*(\S+)\s*$", text, re.M))
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if fields.get("sources_sha1") != h.hexdigest():
        return None, f"profiles/{name} is stale: the kernel changed since the capture"
    if "dram_bytes_per_launch_full_workload" not in fields:
        return None, f"profiles/{name} has no traffic line"
    return int(fields["dram_bytes_per_launch_full_workload"]), f"profiles/{name} (2-view capture scaled to 20 views)"


def block_diagonal_pair(q):
    """Per Gaussian the quaternion pair (q_l, q_r) whose rotation
    L(q_l) R(q_r) (Eq. 8) is blockdiag(R3(q), 1), R3 the usual rotation of the
    unit quaternion q = (w, x, y, z): the No-4DRot model written as a general
    4D one, so that the 4D kernels render exactly the scene of the spatial
    fast path.  With x -> q_l x q_r and e0 = its image of 1, x -> q_l x
    conj(q_l) is x -> (M x) conj(e0), a conjugation whose 3x3 block gives q_l
    (Shepperd's method); then q_r = conj(q_l) e0.  Host-side input
    preparation for a timing comparison, float64 numpy."""
    import numpy as np

    def ham(p_, q_):
        a1, b1, c1, d1 = p_
        a2, b2, c2, d2 = q_
        return np.stack([a1 * a2 - b1 * b2 - c1 * c2 - d1 * d2, a1 * b2 + b1 * a2 + c1 * d2 - d1 * c2,
                         a1 * c2 - b1 * d2 + c1 * a2 + d1 * b2, a1 * d2 + b1 * c2 - c1 * b2 + d1 * a2])

    conj = np.array([1.0, -1.0, -1.0, -1.0])[:, None]
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q, axis=0)
    n = q.shape[1]
    M = np.zeros((4, 4, n))
    M[:3, :3] = [[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                 [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                 [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]]
    M[3, 3] = 1.0
    e0 = M[:, 0]
    R = np.stack([ham(M[:, k], e0 * conj)[1:] for k in (1, 2, 3)], axis=1)
    tr = R[0, 0] + R[1, 1] + R[2, 2]
    s_ = [2 * np.sqrt(np.maximum(v, 1e-30)) for v in (tr + 1, 1 + R[0, 0] - R[1, 1] - R[2, 2],
                                                      1 + R[1, 1] - R[0, 0] - R[2, 2], 1 + R[2, 2] - R[0, 0] - R[1, 1])]
    cand = [np.stack([s_[0] / 4, (R[2, 1] - R[1, 2]) / s_[0], (R[0, 2] - R[2, 0]) / s_[0], (R[1, 0] - R[0, 1]) / s_[0]]),
            np.stack([(R[2, 1] - R[1, 2]) / s_[1], s_[1] / 4, (R[0, 1] + R[1, 0]) / s_[1], (R[0, 2] + R[2, 0]) / s_[1]]),
            np.stack([(R[0, 2] - R[2, 0]) / s_[2], (R[0, 1] + R[1, 0]) / s_[2], s_[2] / 4, (R[1, 2] + R[2, 1]) / s_[2]]),
            np.stack([(R[1, 0] - R[0, 1]) / s_[3], (R[0, 2] + R[2, 0]) / s_[3], (R[1, 2] + R[2, 1]) / s_[3], s_[3] / 4])]
    pick = np.where(tr > 0, 0, np.where((R[0, 0] > R[1, 1]) & (R[0, 0] > R[2, 2]), 1,
                                        np.where(R[1, 1] > R[2, 2], 2, 3)))
    a = np.zeros((4, n))
    for k in range(4):
        a[:, pick == k] = cand[k][:, pick == k]
    return a, ham(a * conj, e0)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def job_throughput(pixels_per_step: int, steps: int, local_ms: float, dist=None, device="cpu") -> tuple:
    """Whole-job Mpix/s of N replicas: every rank renders pixels_per_step per
    step; the job takes as long as its slowest rank (max over ranks of the
    timed region).  Returns (Mpix/s over all ranks, max ms)."""
    import torch
    world = dist.get_world_size() if dist else 1
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return pixels_per_step * world * steps / (ms * 1e-3) / 1e6, ms


# ---------------------------------------------------------------------------- reference arm
def workload_inputs(n=None, views=None, scale=1.0):
    from paper_2310_10642_gb300 import inputs as I
    c = I.config(3, n=n, scale=scale)
    vs = c["views"][: (views or WORKLOAD["views"])]
    return c["gaussians"], vs, c["options"]


def host_cpu() -> dict:
    """Core count and CPU model of the host running the oracle."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return dict(cores=int(cores), model=model)


def _as_f64(G):
    """The parameters in float64 once, so that every oracle call reads them in place."""
    import numpy as np
    return {k: (np.ascontiguousarray(v, dtype=np.float64) if isinstance(v, np.ndarray) else v) for k, v in G.items()}


def _oracle_crop(G64, v, crop, seed):
    """One oracle forward + backward on the crop x crop window at the view's centre."""
    import numpy as np
    from oracle import oracle as O
    x0 = v["width"] // 2 - crop // 2
    y0 = v["height"] // 2 - crop // 2
    win = (x0, y0, crop, crop)
    O.render(G64, v, window=win, prefilter=True)
    O.backward(G64, v, np.random.default_rng(seed).normal(size=(3, crop, crop)), window=win, prefilter=True)
    return crop * crop


def oracle_sample(G, views, budget_s=20.0, crop=32, threads=1):
    """FP64 oracle forward+backward on crop x crop windows at the centre of
    successive views until ~budget_s of wall time; returns (Mpix/s, sample).
    threads > 1 splits the work over pixels: each thread renders whole
    windows (one oracle call at a time per thread; the C oracle has no shared
    mutable state and ctypes releases the interpreter lock during its calls)."""
    from concurrent.futures import ThreadPoolExecutor
    G64 = _as_f64(G)
    t0 = time.perf_counter()
    pix = done = 0
    if threads <= 1:
        for v in views:
            pix += _oracle_crop(G64, v, crop, done)
            done += 1
            if time.perf_counter() - t0 > budget_s:
                break
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            while time.perf_counter() - t0 <= budget_s and done < 64 * threads:
                batch = [views[(done + i) % len(views)] for i in range(threads)]
                pix += sum(ex.map(lambda a: _oracle_crop(G64, a[1], crop, a[0]), enumerate(batch, done)))
                done += threads
    dt = time.perf_counter() - t0
    return pix / dt / 1e6, (f"{done} views x {crop}x{crop} centre crop, forward+backward, "
                            f"{G['logit'].shape[0]} Gaussians, {threads} thread{'s' if threads > 1 else ''}")


def cpu_baseline_both(G, views, budget_s=12.0) -> dict:
    """The oracle on one host core and on all of them, in the same run."""
    host = host_cpu()
    v1, s1 = oracle_sample(G, views, budget_s=budget_s, threads=1)
    vn, sn = oracle_sample(G, views, budget_s=budget_s, threads=host["cores"])
    return dict(value=vn, unit="Mpix/s", cores=host["cores"], kind="oracle", sample=sn, cpu_model=host["model"],
                single_thread=dict(value=v1, unit="Mpix/s", cores=1, sample=s1))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    G, views, _ = workload_inputs(args.n, args.views, args.scale)
    vals = []
    sample = ""
    host = host_cpu()
    for _ in range(args.warmup):
        oracle_sample(G, views[:1], budget_s=0.0, crop=16)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, sample = oracle_sample(G, views, budget_s=30.0 / max(1, args.steps), crop=32, threads=host["cores"])
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.median(vals)
    out = dict(metric="Mpix/s fwd+bwd (4DGS render, 1M Gaussians, 1352x1014)", value=value, unit="Mpix/s",
               n_gpus=args.gpus, steps=args.steps, warmup=args.warmup, ms_per_step=wall * 1e3 / args.steps,
               higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
               config=dict(WORKLOAD, l2="inputs larger than L2"), impl="reference",
               cpu_baseline=dict(value=value, unit="Mpix/s", cores=host["cores"], kind="oracle", sample=sample,
                                 cpu_model=host["model"]),
               e2e=dict(value=value, unit="Mpix/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0), gpu_launches=0)
    print(json.dumps(out))
    return 0


# ---------------------------------------------------------------------------- GPU arm
TRAIN_WORKLOAD = dict(workload="4dgs-train-step", gaussians=3_000_000, clustered=True, sh_degree=3, n_freq=2,
                      views="4 x 1352x1014 + 4 x 800x800", loss="0.8 L1 + 0.2 (1 - SSIM)", optimizer="Adam")


def measure_train(args, dist=None, world=1, rank=0, steps=None, per_view=True, e2e=True) -> dict:
    """Training-step throughput on the 3M-Gaussian, 8-view workload: one CUDA
    graph replay = forward, loss, adjoint and Adam over all parameters.
    Returns the numbers; the caller prints them."""
    import torch
    from paper_2310_10642_gb300 import inputs as I
    from paper_2310_10642_gb300 import native as N
    from paper_2310_10642_gb300 import render as R
    from paper_2310_10642_gb300.train import TrainStep
    steps = steps or args.steps
    c = I.config(4, n=args.n, n_views=args.views, scale=args.scale)
    G, views = c["gaussians"], c["views"]
    n = G["logit"].shape[0]
    mixed = args.precision == "mixed"
    tile = 32 if args.tile == "auto" else int(args.tile)
    depth = 256 if args.batch_depth == "auto" else int(args.batch_depth)
    binsz = max(tile, 64) if args.bin_size == "auto" else int(args.bin_size)
    opts = dict(c["options"], tile_size=tile, bin_size=binsz, batch_depth=depth)
    tg_host = torch.cat([torch.as_tensor(t).reshape(-1) for t in I.random_target(views, 44)]).pin_memory()
    tg = tg_host.cuda()
    p = R.params_to_device(G)
    # one group: with 8 views over 3M Gaussians the per-Gaussian stages, run once per group, outweigh
    # the overlap (two groups measured 20.9 vs 19.4 ms per step)
    ts = TrainStep(p, views, tg, opts, mixed=mixed, groups=1)
    npix = ts.frame.total_pixels
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        ts.step()
    torch.cuda.synchronize()
    l0 = N.fgs4d_launch_count()
    ts.capture()
    per_step = N.fgs4d_launch_count() - l0
    for _ in range(2):
        ts.replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        ts.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    value, total_ms = job_throughput(npix, steps, e0.elapsed_time(e1), dist, device="cuda")
    cnt = ts.frame.counters()
    status = max(c_.status for c_ in cnt) if isinstance(cnt, list) else cnt.status

    # end to end: this step's targets copied in from pinned host memory, the loss read back
    e2e_d = None
    if e2e:
        loss_host = torch.empty(1, dtype=torch.float32).pin_memory()
        ks = max(1, min(steps, 5))
        e0.record(stream)
        for _ in range(ks):
            ts.targets.copy_(tg_host, non_blocking=True)
            ts.replay()
            loss_host.copy_(ts.loss, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / ks
        e2e_d = dict(value=npix * world / (ms * 1e-3) / 1e6, unit="Mpix/s", h2d_bytes_per_step=int(tg_host.numel() * 4),
                     d2h_bytes_per_step=4, ms_per_step=ms)

    # plain FP32 per-view path: each view rendered, scored and differentiated on its own (gradients
    # summed over views), then one Adam step
    single = None
    if per_view and rank == 0:
        p32 = R.params_to_device(G)
        tsv = [TrainStep(p32, [v], tgv.reshape(-1).cuda(), dict(opts, record_fp16=0), mixed=False)
               for v, tgv in zip(views, [torch.as_tensor(t) for t in I.random_target(views, 44)])]
        acc = {k: torch.zeros_like(p32[k]) for k in tsv[0].grads}

        def per_view_step():
            for k in acc:
                acc[k].zero_()
            for t in tsv:
                fr = t.frame
                fr.slice_project(t.render_params)
                fr.bin_sort()
                fr.render()
                N.fgs4d_loss_l1_dssim(fr.c_views, fr.nv, fr.image.data_ptr(), t.targets.data_ptr(), t.lam,
                                      t.loss.data_ptr(), t.dL.data_ptr(), t.scratch.data_ptr(), t.scratch_bytes,
                                      stream.cuda_stream)
                fr.backward(t.render_params, t.dL, t.grads)
                for k in acc:
                    acc[k].add_(t.grads[k])
            for k in acc:
                tsv[0].grads[k].copy_(acc[k])
            N.fgs4d_adam_step(tsv[0]._groups, tsv[0].lrs.data_ptr(), 0.9, 0.999, 1e-15,
                              tsv[0].step_count.data_ptr(), tsv[0].bias.data_ptr(), stream.cuda_stream)

        for _ in range(2):
            per_view_step()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            per_view_step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms1 = e0.elapsed_time(e1) / 3
        single = dict(mpix_s=round(npix / (ms1 * 1e-3) / 1e6, 3), ms_per_step=round(ms1, 3),
                      path="plain FP32, one view per call (render, loss, adjoint), gradients summed, one Adam step")
        del tsv, acc, p32
    out = dict(value=round(value, 3), ms_per_step=round(total_ms / steps, 4),
               steps_per_s=round(1e3 * steps / total_ms, 3), pixels_per_step=npix,
               config=dict(TRAIN_WORKLOAD, n=n, n_views=len(views), tile=tile, bin=binsz, batch_depth=depth,
                           view_groups=[[0, len(views)]],
                           precision="BF16 4DSH copy + 16-bit conic records, FP32 master weights" if mixed
                           else "FP32", cuda_graph=True, pixels_per_step=npix,
                           l2="inputs larger than L2 (1.9 GB FP32 parameters + Adam state)",
                           parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
               per_view_fp32=single,
               train_vs_per_view_fp32=round(value / world / single["mpix_s"], 3) if single else None,
               final_loss=float(ts.loss.item()), status=int(status), e2e=e2e_d, clocks=clk,
               gpu_launches=int(per_step * steps))
    del ts, p, tg
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def main_train(args):
    """Training-step throughput as the headline (``--workload train``)."""
    import torch
    from paper_2310_10642_gb300 import native as N
    N.build()
    N.lib()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    r = measure_train(args, dist, world, rank, e2e=not args.no_e2e)
    if rank == 0:
        out = dict(metric="Mpix/s training step (4DGS, 3M Gaussians, 8 views)", value=r["value"], unit="Mpix/s",
                   n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=r["ms_per_step"],
                   steps_per_s=r["steps_per_s"], higher_is_better=True, scaling="weak", vs_baseline=None,
                   dtype="f32", data="synthetic", config=r["config"], per_view_fp32=r["per_view_fp32"],
                   train_vs_per_view_fp32=r["train_vs_per_view_fp32"], final_loss=r["final_loss"],
                   status=r["status"], e2e=r["e2e"], clocks=r["clocks"], gpu_launches=r["gpu_launches"])
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "train":
        return main_train(args)
    import torch
    from paper_2310_10642_gb300 import autotune as A
    from paper_2310_10642_gb300 import native as N
    from paper_2310_10642_gb300 import render as R

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    N.build()
    N.lib()

    G, views, opts = workload_inputs(args.n, args.views, args.scale)
    n = G["logit"].shape[0]
    mixed = args.precision == "mixed"
    p32 = R.params_to_device(G)
    p = R.params_to_device(G, shs_dtype=torch.bfloat16) if mixed else p32
    opts = dict(opts, record_fp16=int(mixed))
    tiles = A.TILE_SIZES if args.tile == "auto" else (int(args.tile),)
    depths = A.BATCH_DEPTHS if args.batch_depth == "auto" else (int(args.batch_depth),)
    cands = [c for c in A.candidates(tiles, depths)
             if args.bin_size == "auto" or c["bin_size"] == int(args.bin_size)]
    if not cands:
        raise SystemExit("--bin-size must be a multiple of the tile size")
    tune_table = None
    if len(cands) > 1:  # launch shape from the autotuner, timed on this workload (untimed here)
        opts, tune_table = A.tune(p, views, opts, cands=cands, cache=None)
    else:
        opts = dict(opts, **cands[0])
    groups_table = None
    if args.groups <= 0:  # one batch or two view groups, timed on this workload with the chosen shape
        args.groups, groups_table = A.tune_groups(p, views, opts)
    opts_fp32 = dict(opts, record_fp16=0)
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device="cuda").manual_seed(1234)
    grads = {k: torch.empty(p32[k].shape, device="cuda", dtype=torch.float32) for k in R.PARAM_KEYS}
    stages = ["slice_project", "bin_sort", "render", "render_backward_2d", "project_backward"]

    def sized_frame(vs, o, params):
        """Frame whose pair capacity is sized once, outside the timed region, with headroom."""
        fr = R.Frame(n, vs, o)
        fr.forward(params, check=True)
        c = fr.last_counters
        if c.n_pairs * 1.1 > fr.pair_capacity:
            fr._alloc(int(c.n_pairs * 1.15) + 4096)
            fr.forward(params, check=True)
        return fr

    def make_step(fr, params, dLv, events=None, gr=None):
        gr = grads if gr is None else gr

        def step():
            if events is not None:
                events[0].record(stream)
            fr.slice_project(params)
            if events is not None:
                events[1].record(stream)
            fr.bin_sort()
            if events is not None:
                events[2].record(stream)
            fr.render()
            if events is not None:
                events[3].record(stream)
            if events is None:
                fr.backward(params, dLv, gr)  # both adjoint steps in one call
            else:
                fr.backward_2d(dLv)
                events[4].record(stream)
                fr.project_backward(params, gr)
                events[5].record(stream)
        return step

    def capture(step):
        """One whole step (all four entry points) as a CUDA graph; returns (graph, launches per step)."""
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        l0 = N.fgs4d_launch_count()
        with torch.cuda.graph(g):
            step()
        torch.cuda.synchronize()
        return g, N.fgs4d_launch_count() - l0

    def time_graph(g, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    frame = sized_frame(views, opts, p)
    npix = frame.total_pixels
    dL = torch.randn(3 * npix, device="cuda", generator=gen) * (1.0 / npix)
    counters = frame.last_counters

    # per-stage breakdown: eager launches bracketed by events (untimed for the headline)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)] for _ in range(max(3, args.steps))]
    for _ in range(max(3, args.warmup)):
        make_step(frame, p, dL)()
    for e in ev:
        make_step(frame, p, dL, e)()
    torch.cuda.synchronize()
    stage_ms = {s: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in ev) for i, s in enumerate(stages)}

    # headline: K whole steps, replayed as one CUDA graph each (or launched eagerly with --no-graph).
    # With groups > 1 the step runs the views as contiguous groups on as many streams, so that one
    # group's latency-bound stages overlap another's compositing kernels (same images; gradients
    # summed group after group)
    if args.groups > 1:
        sframe = R.SplitFrame(n, views, opts, groups=args.groups)
        sframe.forward(p, check=True)
        for fr_ in sframe.frames:
            c_ = fr_.last_counters
            if c_.n_pairs * 1.1 > fr_.pair_capacity:
                fr_._alloc(int(c_.n_pairs * 1.15) + 4096)
        sframe.forward(p, check=True)
        run_frame = sframe

        def step():
            sframe.step(p, dL, grads)
    else:
        run_frame = frame
        step = make_step(frame, p, dL)
    graph, per_step = (None, 0) if args.no_graph else capture(step)
    run = step if graph is None else graph.replay
    for _ in range(max(3, args.warmup)):
        run()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = N.fgs4d_launch_count()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e_start.record(stream)
    for k in range(args.steps):
        run()
    e_end.record(stream)
    torch.cuda.synchronize()
    launches = N.fgs4d_launch_count() - launches0 + per_step * args.steps * (graph is not None)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = e_start.elapsed_time(e_end)
    value, total_ms = job_throughput(npix, args.steps, total_ms, dist, device="cuda")
    ms_step = total_ms / args.steps
    fwd_ms = stage_ms["slice_project"] + stage_ms["bin_sort"] + stage_ms["render"]  # per step, eager
    fwd_mpix = npix / (fwd_ms * 1e-3) / 1e6
    # the forward alone (slice/project, binning, compositing) as a CUDA graph step, like the headline
    fwd_graph = None
    if graph is not None:
        def fwd_step():
            run_frame.forward(p, check=False)
        for _ in range(2):
            fwd_step()
        torch.cuda.synchronize()
        gf = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gf):
            fwd_step()
        ms_f = time_graph(gf, max(3, args.steps))
        del gf
        fwd_graph = dict(mpix_s=round(npix / (ms_f * 1e-3) / 1e6, 3), ms_per_step=round(ms_f, 4),
                         what="forward only (slice/project, binning, compositing), one CUDA graph per step, "
                              "the headline's view groups")

    # ---- roofline of the dominant kernel (algorithmic bytes per launch / time)
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    L, K = G["sh_degree"], G["n_freq"]
    C = 3 * (L + 1) ** 2 * (K + 1)
    shs_b = 2 if mixed else 4
    rec_b = 32 if mixed else 48   # splat record written per visible splat
    rd_b = 32 if mixed else 36    # record bytes a tile stages per list entry
    V = len(views)
    nvis, npairs = counters.n_visible, counters.n_pairs
    binsz = opts.get("bin_size") or opts["tile_size"]
    view_tiles = [-(-v["width"] // binsz) * -(-v["height"] // binsz) for v in views]
    if max(view_tiles) <= 4096:
        # counting-sort path: compaction (read tile counts + depth keys, write 8 B per visible splat), depth
        # sort (4 passes x 20 B), view keys (8 B) and view pass (20 B), histogram walk (id, record, count
        # written) and scatter walk (id, count, record) per visible splat, the (tile, chunk) counts written,
        # scanned (read twice, written once) and read back, and 4 B per pair written
        entries = sum(t * -(-nvis // (V * 256)) for t in view_tiles)
        bin_bytes = (V * n * 8 + nvis * (8 + 4 * 20 + 8 + 20 + (4 + rec_b + 4) + (8 + rec_b))
                     + entries * (4 + 12 + 4) + npairs * 4)
    else:
        # radix path: compaction, depth sort, offsets scan (8 B), emission (8 B per pair), pair sort (passes x
        # 20 B per pair), ranges (4 B per pair)
        bin_bytes = (V * n * 8 + nvis * (8 + 4 * 20 + 8) + npairs * (8 + 4)
                     + npairs * 20 * ((_bits(frame.layout().total_tiles) + 7) // 8))
    alg = {
        # parameters read once + records/tile counts/depth keys written
        "slice_project": n * (17 * 4 + C * shs_b) + nvis * rec_b + V * n * 8,
        "bin_sort": bin_bytes,
        # list ids + gathered records per pair, 20 B written per pixel
        "render": npairs * (4 + rd_b) + npix * 20,
        # same gathers + dL/dimage, T, n_last per pixel + 48 B gradient record per splat (zeroed) and per
        # visible splat (atomics)
        "render_backward_2d": npairs * (4 + rd_b) + npix * 20 + V * n * 48 + nvis * 48,
        # visible-splat list and its 2D gradients + per-Gaussian parameters read and gradients written
        "project_backward": nvis * (4 + 48) + n * (17 * 4 + C * shs_b) + n * (17 * 4 + C * 4),
    }
    # compositing and its adjoint are bound by FP32 arithmetic, not bytes: their
    # algorithmic work is FLOPs per blended (pixel, splat) pair (Eq. 6 forward:
    # 23, adjoint: 51; FMA = 2, exp = 1), counted by fgs4d_render_stats, against
    # the FP32 peak 152 SMs x 128 lanes x 2 x SM clock
    work = frame.render_stats()
    torch.cuda.synchronize()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    flops = {"render": 23 * work["blended"], "render_backward_2d": 51 * work["blended"]}
    stage_roof = {}
    for st_name, ms in stage_ms.items():
        if st_name in flops:
            a_ = flops[st_name] / (ms * 1e-3) / 1e12
            stage_roof[st_name] = dict(bound="alu", achieved=round(a_, 3), peak=round(fp32_peak, 1), unit="TFLOP/s",
                                       frac=round(a_ / fp32_peak, 4))
        else:
            a_ = alg[st_name] / (ms * 1e-3) / 1e9
            stage_roof[st_name] = dict(bound="hbm", achieved=round(a_, 1), peak=hbm, unit="GB/s",
                                       frac=round(a_ / hbm, 4))
    dom = max(stage_ms, key=stage_ms.get)
    full_workload = (args.n is None and args.views is None and args.scale == 1.0 and mixed
                     and all(opts[k] == v for k, v in PROFILED_SHAPE.items()))
    traffic, traffic_note = profiled_traffic(dom) if full_workload else (None, "not the profiled workload")
    kernel_of = {"render_backward_2d": "render_bwd_kernel (stage: 2D-gradient memset + kernel)",
                 "render": "render_fwd_kernel", "project_backward": "project_backward_kernel + sh_backward_kernel",
                 "bin_sort": "bin_sort pipeline", "slice_project": "slice_project_kernel"}
    roofline = dict(stage_roof[dom], traffic=traffic, traffic_source=traffic_note, kernel=kernel_of.get(dom, dom),
                    peak_source=("FP32: 152 SMs x 128 lanes x 2 FLOP x max SM clock" if stage_roof[dom]["bound"] == "alu"
                                 else f"{peak_kind} hbm_gbs"))

    # ---- plain FP32 paths on the same GPU: the whole batch, and one view per call
    single = batched_fp32 = None
    if rank == 0:
        if mixed:
            fr = sized_frame(views, opts_fp32, p32)
            g32, _ = capture(make_step(fr, p32, dL))
            ms32 = time_graph(g32, 3)
            batched_fp32 = dict(mpix_s=round(npix / (ms32 * 1e-3) / 1e6, 3), ms_per_step=round(ms32, 4))
            del g32, fr
        fr1 = sized_frame(views[:1], opts_fp32, p32)
        dL1 = torch.randn(3 * fr1.total_pixels, device="cuda", generator=gen) * (1.0 / fr1.total_pixels)
        step1 = make_step(fr1, p32, dL1)
        for _ in range(3):
            step1()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            step1()
        e1.record(stream)
        torch.cuda.synchronize()
        ms1 = e0.elapsed_time(e1) / reps
        single = dict(mpix_s=round(fr1.total_pixels / (ms1 * 1e-3) / 1e6, 3), ms_per_view=round(ms1, 4),
                      path="plain FP32 records and coefficients, one view per call, eager launches")
        del fr1

    # ---- e2e through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        host_p = {k: p[k].cpu().pin_memory() for k in R.PARAM_KEYS}
        host_dL = dL.cpu().pin_memory()
        host_img = torch.empty(3 * npix, dtype=torch.float32).pin_memory()
        host_g = {k: torch.empty(p[k].shape, dtype=torch.float32).pin_memory() for k in R.PARAM_KEYS}
        h2d = sum(t.numel() * t.element_size() for t in host_p.values()) + host_dL.numel() * 4
        d2h = host_img.numel() * 4 + sum(t.numel() * 4 for t in host_g.values())

        # pipelined across steps (HostPipeline): the inputs of step k + 1 go in and the outputs of
        # step k - 1 come out on copy streams while step k computes
        from paper_2310_10642_gb300.pipeline import HostPipeline
        pipe = HostPipeline(run_frame, p)
        pipe.run([(host_p, host_dL)] * 4, [(host_img, host_g)] * 4)  # both slots captured before timing
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ks = max(3, min(args.steps, 10))
        clocks_e2e = ClockSampler(torch.cuda.current_device())
        clocks_e2e.start()
        time.sleep(0.3)
        e0.record(stream)
        t_host = time.perf_counter()
        pipe.run([(host_p, host_dL)] * ks, [(host_img, host_g)] * ks)
        t_host = time.perf_counter() - t_host
        e1.record(stream)
        torch.cuda.synchronize()
        clk_e2e = clocks_e2e.stop()
        ms_e2e = e0.elapsed_time(e1) / ks
        # the same pipeline with the copies left out (compute through its graphs and event waits only), and
        # with the copies of each direction alone: how much of the gap to the device step the copies make
        def pipe_pieces(do_in, do_out, k_steps):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pipe.s_in.wait_stream(stream)
            if do_in:
                pipe._copy_in(pipe.slots[0], host_p, host_dL)
            for k_ in range(k_steps):
                if do_in and k_ + 1 < k_steps:
                    pipe._copy_in(pipe.slots[(k_ + 1) % 2], host_p, host_dL)
                pipe._compute(pipe.slots[k_ % 2])
                if do_out:
                    pipe._copy_out(pipe.slots[k_ % 2], host_img, host_g)
            stream.wait_stream(pipe.s_out)
            stream.wait_stream(pipe.s_in)
            b.record(stream)
            torch.cuda.synchronize()
            return round(a.elapsed_time(b) / k_steps, 3)
        pieces_ms = dict(compute_only=pipe_pieces(False, False, ks), with_copies_in=pipe_pieces(True, False, ks),
                         with_copies_out=pipe_pieces(False, True, ks), all=pipe_pieces(True, True, ks))

        # the copies alone on this machine (same buffers, the pipeline's copy streams): in, out, both at once
        def copies(kind):
            s_in, s_out = pipe.s_in, pipe.s_out
            sl = pipe.slots[0]
            torch.cuda.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            s_in.wait_stream(stream)
            s_out.wait_stream(stream)
            for _ in range(3):
                if kind in ("in", "both"):
                    with torch.cuda.stream(s_in):
                        for k_ in R.PARAM_KEYS:
                            sl["p"][k_].copy_(host_p[k_], non_blocking=True)
                        sl["dL"].copy_(host_dL, non_blocking=True)
                if kind in ("out", "both"):
                    with torch.cuda.stream(s_out):
                        host_img.copy_(sl["img"], non_blocking=True)
                        for k_ in R.PARAM_KEYS:
                            host_g[k_].copy_(sl["g"][k_], non_blocking=True)
            stream.wait_stream(s_in)
            stream.wait_stream(s_out)
            c1.record(stream)
            torch.cuda.synchronize()
            return round(c0.elapsed_time(c1) / 3, 3)

        copy_ms = {k_: copies(k_) for k_ in ("in", "out", "both")}
        e2e = dict(value=npix * world / (ms_e2e * 1e-3) / 1e6, unit="Mpix/s", h2d_bytes_per_step=int(h2d),
                   d2h_bytes_per_step=int(d2h), ms_per_step=ms_e2e, copies_alone_ms=copy_ms,
                   host_enqueue_ms_per_step=round(t_host * 1e3 / ks, 3), pipeline_pieces_ms=pieces_ms,
                   clocks=clk_e2e,
                   pipeline="inputs of step k+1 in and outputs of step k-1 out on copy streams while step k "
                            "computes (each buffer set's step replayed as a CUDA graph)")

    # ---- rotation variants on the same Gaussians and views: the No-4DRot fast path (spatial rotation
    # from q_left, block-diagonal Sigma: no Schur complement, no velocity term) and static 3DGS (no time
    # axis, plain SH colour: the first (L+1)^2 coefficient rows); eager stage times as for the 4D path
    variants = None
    if rank == 0 and not args.no_variants:
        def stage_times(params):
            fr = sized_frame(views, opts, params)
            gr = {k: torch.empty(params[k].shape, device="cuda", dtype=torch.float32) for k in R.PARAM_KEYS}
            evv = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)] for _ in range(3)]
            for _ in range(2):
                make_step(fr, params, dL, gr=gr)()
            for e in evv:
                make_step(fr, params, dL, e, gr)()
            torch.cuda.synchronize()
            st = {s_: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evv) for i, s_ in enumerate(stages)}
            st = {k: round(v, 4) for k, v in st.items()}
            total = sum(st.values())
            out_ = dict(stage_ms=st, ms_per_step=round(total, 4), mpix_s=round(npix / (total * 1e-3) / 1e6, 3),
                        visible_splats=fr.last_counters.n_visible, pairs=fr.last_counters.n_pairs)
            del fr, gr
            return out_

        nb3 = 3 * (G["sh_degree"] + 1) ** 2
        ql_eq, qr_eq = block_diagonal_pair(G["ql"])
        p_eq = dict(p, ql=torch.as_tensor(ql_eq, dtype=torch.float32).cuda(),
                    qr=torch.as_tensor(qr_eq, dtype=torch.float32).cuda(), rotation=N.ROT_4D)
        fast = stage_times(dict(p, rotation=N.ROT_SPATIAL))
        general = stage_times(p_eq)
        per_g = ("slice_project", "project_backward")
        variants = {
            "4d": dict(stage_ms={k: round(v, 4) for k, v in stage_ms.items()},
                       ms_per_step=round(sum(stage_ms.values()), 4),
                       mpix_s=round(npix / (sum(stage_ms.values()) * 1e-3) / 1e6, 3), visible_splats=nvis,
                       pairs=npairs),
            "no_4drot": fast,
            "no_4drot_through_4d_kernels": general,
            "no_4drot_saved_ms": dict({k: round(general["stage_ms"][k] - fast["stage_ms"][k], 4) for k in per_g},
                                      step=round(general["ms_per_step"] - fast["ms_per_step"], 4)),
            "static_3dgs": stage_times(dict(p, shs=p["shs"][:nb3].contiguous(), n_freq=0,
                                            rotation=N.ROT_STATIC)),
            "note": "eager stage times, same Gaussians, views and launch shape.  no_4drot: q_left as the spatial "
                    "rotation (block-diagonal Sigma), rendered by the fast path and, as the same scene, by the 4D "
                    "kernels through the equivalent quaternion pair of Eq. 8 (identical splats and pairs); "
                    "static_3dgs: no time axis, SH degree 3 colour without Fourier orders",
        }

    # ---- batching on the workload shaped for it (config 2: 300k Gaussians, 80 views at 1352x1014 from
    # 20 arc cameras x 4 times plus 20 views at 676x507): the whole batch as one graph step (two view
    # groups) against the same views one call each (eager), both mixed precision, forward + backward
    batching = None
    if rank == 0 and not args.no_batching:
        from paper_2310_10642_gb300 import inputs as I2
        c2 = I2.config(2, n=(args.n // 3 if args.n else None), scale=args.scale)
        G2, views2 = c2["gaussians"], c2["views"]
        n2 = G2["logit"].shape[0]
        p2 = R.params_to_device(G2, shs_dtype=torch.bfloat16 if mixed else torch.float32)
        o2 = dict(c2["options"], record_fp16=int(mixed), **{k: opts[k] for k in ("tile_size", "bin_size",
                                                                                 "batch_depth")})
        g2 = {k: torch.empty(p2[k].shape, device="cuda", dtype=torch.float32) for k in R.PARAM_KEYS}
        sf2 = R.SplitFrame(n2, views2, o2, groups=max(1, args.groups))
        sf2.forward(p2, check=True)
        for fr_ in sf2.frames:
            fr_._alloc(int(fr_.last_counters.n_pairs * 1.15) + 4096)
        sf2.forward(p2, check=True)
        dL2 = torch.randn(3 * sf2.total_pixels, device="cuda", generator=gen) * (1.0 / sf2.total_pixels)
        for _ in range(2):
            sf2.step(p2, dL2, g2)
        torch.cuda.synchronize()
        gb = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gb):
            sf2.step(p2, dL2, g2)
        ms_b = time_graph(gb, 3)
        del gb
        ones = [R.Frame(n2, [v], o2) for v in views2]
        for f1 in ones:
            f1.forward(p2, check=True)
        offs = sf2.pix_offsets + [sf2.total_pixels]

        def one_by_one():
            for i, f1 in enumerate(ones):
                f1.step(p2, dL2[3 * offs[i]: 3 * offs[i + 1]], g2)

        one_by_one()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_by_one()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_1 = e0.elapsed_time(e1)
        npix2 = sf2.total_pixels
        batching = dict(views=len(views2), sizes=sorted({f"{v['width']}x{v['height']}" for v in views2}),
                        gaussians=n2, pixels=npix2, batched_ms=round(ms_b, 3),
                        batched_mpix_s=round(npix2 / (ms_b * 1e-3) / 1e6, 3), one_by_one_ms=round(ms_1, 3),
                        one_by_one_mpix_s=round(npix2 / (ms_1 * 1e-3) / 1e6, 3), speedup=round(ms_1 / ms_b, 3),
                        what="forward + backward of all views: one CUDA graph step (views in two groups) vs one "
                             "eager call sequence per view (its gradients overwritten per view)")
        del sf2, ones, p2, g2
        torch.cuda.empty_cache()

    # ---- depth and optical-flow maps (f2) through the same lists: eager stage times
    aux = None
    if rank == 0 and not args.no_aux:
        fra = sized_frame(views, dict(opts, aux_channels=1), p)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for _ in range(2):
            fra.slice_project(p)
            fra.bin_sort()
            fra.render()
            fra.render_aux()
        reps, t_sp, t_r, t_a = 5, 0.0, 0.0, 0.0
        for _ in range(reps):
            evs[0].record(stream)
            fra.slice_project(p)
            evs[1].record(stream)
            fra.bin_sort()
            fra.render()
            evs[2].record(stream)
            fra.render_aux()
            evs[3].record(stream)
            torch.cuda.synchronize()
            t_sp += evs[0].elapsed_time(evs[1])
            t_r += evs[1].elapsed_time(evs[2])
            t_a += evs[2].elapsed_time(evs[3])
        aux = dict(render_aux_ms=round(t_a / reps, 4), mpix_s=round(npix / (t_a / reps * 1e-3) / 1e6, 3),
                   slice_project_ms_with_aux=round(t_sp / reps, 4), bin_sort_plus_render_ms=round(t_r / reps, 4),
                   what="fgs4d_render_aux: accumulated depth and the flow of the projected conditional means "
                        "over one frame (flow_dt 1/300), composited through the image's sorted lists")
        del fra

    # ---- training step (config 4: 3M Gaussians, 8 views), one CUDA graph per step
    train = None
    if rank == 0 and world == 1 and not args.no_train:
        r = measure_train(args, steps=5, per_view=True, e2e=False)
        train = {k: r[k] for k in ("value", "ms_per_step", "steps_per_s", "pixels_per_step", "per_view_fp32",
                                   "train_vs_per_view_fp32", "final_loss", "status", "clocks", "gpu_launches")}
        train["unit"] = "Mpix/s"
        train["config"] = r["config"]

    # ---- CPU baseline (oracle on the host cores, bounded sample)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_both(G, views)

    if rank == 0:
        out = dict(metric="Mpix/s fwd+bwd (4DGS render, 1M Gaussians, 1352x1014)", value=round(value, 3),
                   unit="Mpix/s", n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=round(ms_step, 4),
                   higher_is_better=True, scaling="weak", vs_baseline=None,
                   dtype="f32", data="synthetic",
                   config=dict(WORKLOAD, n=n, views=V, tile=opts["tile_size"], bin=opts["bin_size"],
                               batch_depth=opts["batch_depth"],
                               view_groups=[list(g) for g in run_frame.parts] if args.groups > 1 else [[0, V]],
                               view_groups_tuned=groups_table,
                               autotune=tune_table, precision=(
                       "BF16 4DSH coefficients, 16-bit Cholesky conics; FP32 arithmetic" if mixed else "FP32"),
                       cuda_graph=graph is not None,
                       l2="inputs larger than L2 (356 MB mixed / 644 MB FP32 parameters)",
                               parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                               pixels_per_step=npix, visible_splats=nvis, pairs=npairs),
                   fwd_mpix_s=round(fwd_mpix, 3), fwd_graph=fwd_graph,
                   stage_ms={k: round(v, 4) for k, v in stage_ms.items()},
                   single_view=single, batched_fp32=batched_fp32,
                   batched_vs_single_fp32=round(value / world / single["mpix_s"], 3) if single else None,
                   roofline=roofline, stage_roofline=stage_roof, work=work, cpu_baseline=cpu, e2e=e2e, clocks=clk,
                   rotation_variants=variants, uneven_batch=batching, depth_flow_maps=aux, train_step=train,
                   gpu_launches=int(launches))
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


def _bits(total_tiles: int) -> int:
    b = 1
    while b < 32 and (1 << b) < total_tiles:
        b += 1
    return b


if __name__ == "__main__":
    sys.exit(main())
