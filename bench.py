"""Throughput of the GLU hot path on one (or N replica) GB300 GPUs.

One step = the whole 3840x2160 x8 pipeline on a seeded synthetic guide already resident in HBM:
glu_joint_optimize (grid downsample, Algorithm 1, Algorithm 2 with a 5x5 window and 5
iterations), the LR operator (3x3 box blur then saturation x1.3), glu_apply (Eq. 1, float32 HR
output). Metric: HR Mpixel/s (higher is better). L2 is flushed (a 2 x L2 buffer is written)
between timed steps; every step is timed with CUDA events on the stream it runs on.

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload on the
host cores (the reference arm of this comparison).
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H4K, W4K, SCALE, WIN, NITER = 2160, 3840, 8, 5, 5
BATCH_NITER = 3
EXACT_OPS_PER_PAIR = 21   # GLU*: d (3), v (3), v.d (3), |d|^2 + eps (4), w (1), e (3), |e|^2 (3), compare (1)
VIDEO_FRAMES = 120
METRIC = "HR Mpix/s for GLU optimise+apply at 4K x8; batched/bwd vs plain; % of roofline"
WORKLOAD = "joint-optimise+LRop+apply 3840x2160 x8, 5x5 window, 5 Alg.2 iterations, STRICT"
# canonical FP32 lane operations of Algorithm 1 per window candidate (a-step 7, b-step 20)
OPS_PER_CANDIDATE = 27
# DRAM bytes (read + write) of the trial kernel over one call (its 5 launches) on this workload,
# from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum of every k_trials launch of
# `bench.py --kernel-case trials --case-reps 1`), and the digest of the kernel sources it was
# taken on: once the sources differ, the figure no longer describes the kernel and is not reported
TRIALS_DRAM = dict(bytes_per_call=(94.638 + 40.750) * 1e6,
                   sources_sha256="3c1d5a11502900f4f4e9afad9d17359e5752f039ba097eb9930f6f462f79699f")
TRIALS_SOURCES = ("k_joint.cu", "search.cuh", "common.cuh")


def trials_sources_digest() -> str:
    h = hashlib.sha256()
    for name in TRIALS_SOURCES:
        with open(os.path.join(ROOT, "paper_2307_09582_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)),
                    src="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, src="fallback")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms (with nvidia-smi's own
    timestamps) from before an untimed pre-roll of the workload until after the timed region,
    so that the load window holds many samples even when the timed region is short."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _when(ts: str):
        try:
            return datetime.datetime.strptime(ts.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self, t0=None, t1=None, timed=None):
        """Samples taken in [t0, t1] (host wall-clock seconds; the load window): median SM clock,
        max clock, the throttle reasons seen; `timed` = (start, end) of the timed region, whose
        own samples are counted and summarised beside."""
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((self._when(f[0]), float(f[1]), float(f[2]),
                             {n for n, v in zip(names, f[5:9]) if v.lower() == "active"}))
            except ValueError:
                continue

        def within(a, b):
            return [r for r in rows if r[0] is None or (a is None or r[0] >= a - 0.05)
                    and (b is None or r[0] <= b + 0.05)]
        sel = within(t0, t1)
        if not sel:
            return None
        out = dict(sm_mhz=statistics.median(r[1] for r in sel), sm_max_mhz=max(r[2] for r in sel),
                   reasons=sorted(set().union(*(r[3] for r in sel))), samples=len(sel),
                   period_ms=self.PERIOD_MS,
                   window="untimed pre-roll of the same step, the timed region, the e2e leg")
        if timed is not None:
            tr = within(*timed)
            out["samples_timed_region"] = len(tr)
            if tr:
                out["sm_mhz_timed_region"] = statistics.median(r[1] for r in tr)
                out["reasons_timed_region"] = sorted(set().union(*(r[3] for r in tr)))
        return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------- CPU oracle arm

def oracle_pipeline_sample(img, rows: int):
    """The oracle's pipeline on the top `rows` rows of the guide (a bounded sample): Algorithm 2,
    the LR operator, Eq. 1. Returns (pixels, seconds)."""
    from oracle import oracle as O
    crop = img[:rows]
    t0 = time.perf_counter()
    j = O.joint(crop, SCALE, WIN, N=NITER, strict=True)
    T = O.op_saturation(O.op_box3(O.to_unit(j["L"])), 1.3)
    _ = O.apply(j["ka"], j["kb"], j["omega"], SCALE, WIN, T)
    return crop.shape[0] * crop.shape[1], time.perf_counter() - t0


def cpu_baseline(img):
    """The oracle's whole pipeline on the whole 3840x2160 guide, once (no crop: Algorithm 2's
    cost follows the components, not the area, so a crop would not give the image's rate)."""
    px, sec = oracle_pipeline_sample(img, img.shape[0])
    return dict(value=px / sec / 1e6, unit="HR Mpix/s", cores=os.cpu_count(), kind="oracle",
                seconds=sec,
                sample=f"FP64 oracle pipeline (Alg.2 N={NITER} STRICT, LR op, Eq.1) on the whole "
                       f"3840x2160 guide ({px} px, {sec:.2f} s, one run)")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2307_09582_gb300.inputs import joint_4k_scene, render_u8
    img = render_u8(joint_4k_scene())
    # a step is the whole guide when K steps of it take at most ~150 s, else the top rows
    # (a multiple of the scale) that fit that
    _, t_full = oracle_pipeline_sample(img, img.shape[0])   # the first warm-up step
    rows = img.shape[0]
    if args.steps * t_full > 150.0:
        rows = max(SCALE * 8, int(img.shape[0] * 150.0 / (args.steps * t_full)) // SCALE * SCALE)
    for _ in range(args.warmup - 1):
        oracle_pipeline_sample(img, rows)
    times, px = [], 0
    for _ in range(args.steps):
        px, sec = oracle_pipeline_sample(img, rows)
        times.append(sec)
    tot = sum(times)
    value = px * args.steps / tot / 1e6
    sample = (f"FP64 oracle pipeline on the whole 3840x2160 guide per step ({px} px)"
              if rows == img.shape[0] else
              f"FP64 oracle pipeline on the top {rows} rows of the 3840x2160 guide per step "
              f"({px} px; the whole guide takes {t_full:.1f} s)")
    line = dict(metric=METRIC, value=value, unit="HR Mpix/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * tot / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, H=2160, W=3840, scale=SCALE, window=WIN,
                            iterations=NITER, joint="STRICT", sample=sample),
                cpu_baseline=dict(value=value, unit="HR Mpix/s", cores=os.cpu_count(),
                                  kind="oracle", sample=sample),
                e2e=dict(value=value, unit="HR Mpix/s", h2d_bytes_per_step=0,
                         d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------ GPU arm

def run_glu(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as g
    g.build()
    from paper_2307_09582_gb300 import api
    from paper_2307_09582_gb300.inputs import joint_4k_scene, render_u8

    img = render_u8(joint_4k_scene())
    H, W = img.shape[:2]
    h, w = api.lr_dims(H, W, SCALE)
    npx = H * W
    stream = torch.cuda.current_stream()
    hr = torch.from_numpy(img).to(dev)
    params = api.glu_params(S=WIN, N=NITER)
    lr = torch.empty((h, w, 3), dtype=torch.uint8, device=dev)
    theta = api.Theta.empty(H, W, SCALE, WIN, api.GLU_W_UNORM16, dev)
    err = torch.empty((H, W), dtype=torch.float32, device=dev)
    wsz = api.glu_joint_workspace_size(H, W, SCALE, params)
    wsbuf = torch.empty(wsz + 256, dtype=torch.uint8, device=dev)
    T2 = torch.empty((h, w, 3), dtype=torch.float32, device=dev)
    out = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20), dtype=torch.uint8, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    ev = {k: [] for k in ("s", "j", "e")}

    def step(record):
        if record:
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
        api.glu_joint_optimize(hr, SCALE, params, lr_out=lr, theta=theta, err_map=err,
                               stats=False, workspace=wsbuf)
        if record:
            e[1].record(stream)
        # the LR operator on the optimised LR image (3x3 box on x / 255, saturation 1.3), then
        # Eq. 1: one issue, the apply launched as the operator's programmatic dependent
        api.glu_apply_lrop(theta, lr, filter=0, sat=1.3, gamma=1.0, target=T2, out=out)
        if record:
            e[2].record(stream)
            for k, x in zip(("s", "j", "e"), e):
                ev[k].append(x)

    # the autotuner picks the search and apply variants during the first warm-up step; the
    # phase events are on from the start, so the warm-up also records the call's CUDA graph
    # with them (the library replays a repeated call as a graph)
    api.tune_mode(True)
    api.glu_joint_profile(True)
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step(False)
    torch.cuda.synchronize()
    # one checked run with statistics (outside the timed region)
    _, _, _, st = api.glu_joint_optimize(hr, SCALE, params, lr_out=lr, theta=theta, err_map=err,
                                         stats=True, workspace=wsbuf)
    searched = sum(it["searched"] for it in st["iters"])
    status = api.glu_device_status()
    if status != 0:
        raise RuntimeError(f"device status {status} after the warm-up run")

    clk = ClockSampler(local).__enter__()
    t_load0 = time.time()
    # untimed pre-roll of the same step (about a second) so that the clock record under load has
    # many samples however short the timed region is
    while time.time() - t_load0 < 1.0:
        flush.zero_()
        step(False)
        torch.cuda.synchronize()
    api.glu_joint_profile_read()   # forget the warm-up and pre-roll calls
    barrier(ws)
    torch.cuda.synchronize()
    t_timed0 = time.time()
    for _ in range(args.steps):
        flush.zero_()
        step(True)
    torch.cuda.synchronize()
    t_timed1 = time.time()
    barrier(ws)
    api.glu_joint_profile(False)
    prof = api.glu_joint_profile_read()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev["s"], ev["e"])]
    joint_ms = [a.elapsed_time(b) for a, b in zip(ev["s"], ev["j"])]
    apply_ms = [a.elapsed_time(b) for a, b in zip(ev["j"], ev["e"])]
    tot = max_over_ranks(sum(step_ms), ws, dev)
    ms_per_step = tot / args.steps
    value = ws * npx * args.steps / (tot / 1e3) / 1e6

    # roofline of the dominant kernel (per-launch times from events on the launching stream)
    pk = peaks()
    K = WIN * WIN
    alu_peak = sms * 128 * pk["sm_max_mhz"] * 1e6 / 1e12   # FP32 lane ops, T/s
    calls = max(prof["calls"], 1)
    cand = {
        "glu_search (Alg.1, k_search)": dict(ms=prof["search_ms"] / calls, bound="alu",
                                             work=OPS_PER_CANDIDATE * K * npx / 1e12,
                                             peak=alu_peak, unit="TFLOP/s"),
        "glu_joint trials (Alg.2, k_trials)": dict(ms=prof["trials_ms"] / calls, bound="alu",
                                                   work=OPS_PER_CANDIDATE * K * searched / 1e12,
                                                   peak=alu_peak, unit="TFLOP/s"),
        # the step's tail: LR u8 in, T out and back in, codes + unorm16 weights in, f32 out
        "glu_apply_lrop (LR operator + Eq.1)": dict(
            ms=statistics.mean(apply_ms), bound="hbm",
            work=(npx * (2 + 2 + 12) + h * w * (3 + 12 + 12)) / 1e9,
            peak=pk["hbm_gbs"], unit="GB/s"),
    }
    dom_name, dom = max(cand.items(), key=lambda kv: kv[1]["ms"])
    achieved = dom["work"] / (dom["ms"] / 1e3)
    traffic, traffic_note = None, None
    if "k_trials" in dom_name:
        if trials_sources_digest() == TRIALS_DRAM["sources_sha256"]:
            traffic = TRIALS_DRAM["bytes_per_call"]
            traffic_note = ("DRAM bytes per call (all trial launches of one call) from an ncu "
                            "capture of these kernel sources")
        else:
            traffic_note = "no ncu capture of the current kernel sources"
    roofline = dict(kernel=dom_name, bound=dom["bound"], achieved=achieved, peak=dom["peak"],
                    unit=dom["unit"], frac=achieved / dom["peak"], traffic=traffic,
                    traffic_note=traffic_note,
                    peak_source=pk["src"], launch_ms=dom["ms"],
                    others={k: dict(ms=v["ms"], frac=(v["work"] / (v["ms"] / 1e3)) / v["peak"])
                            for k, v in cand.items()})

    # end to end through the C ABI with host buffers: one glu_pipeline_host call per step copies
    # the guide in, runs the same pipeline and copies the result out (pinned host memory)
    hr_host = torch.from_numpy(img).pin_memory()
    out_host = torch.empty((H, W, 3), dtype=torch.float32).pin_memory()
    pws = torch.empty(api.glu_pipeline_host_workspace_size(H, W, SCALE, params) + 256,
                      dtype=torch.uint8, device=dev)
    def host_step():
        api.glu_pipeline_host(hr_host, SCALE, params, 0, 1.3, 1.0, out_host, pws)
    for _ in range(3):   # the library records the call's CUDA graph on its second sighting
        host_step()
    e2e_ms = []
    for i in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        host_step()
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    del pws
    t_load1 = time.time()
    clk.__exit__(None, None, None)
    e2e_tot = max_over_ranks(sum(e2e_ms), ws, dev)
    e2e_val = ws * npx * len(e2e_ms) / (e2e_tot / 1e3) / 1e6

    names = {k: api.tune_variants(k) for k in (api.GLU_TUNE_SEARCH, api.GLU_TUNE_APPLY)}
    tuned = [dict(kernel=("search", "apply")[int(f[0])], key=[int(x) for x in f[1:6]],
                  variant=names[int(f[0])][int(f[6])], ms=float(f[7]))
             for f in (l.split() for l in api.tune_export().splitlines())]
    extras = {}
    if args.extras and rank == 0:
        extras = measure_extras(api, torch, img, dev, flush, stream)

    line = None
    if rank == 0:
        line = dict(metric=METRIC, value=value, unit="HR Mpix/s", n_gpus=ws, steps=args.steps,
                    warmup=args.warmup, ms_per_step=ms_per_step, higher_is_better=True,
                    scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                    config=dict(workload=WORKLOAD, H=H, W=W, scale=SCALE, window=WIN,
                                iterations=NITER, joint="STRICT", weights="unorm16",
                                l2="flushed between steps (write of a 2xL2 buffer)",
                                parallelism=f"replicas x{ws}"),
                    roofline=roofline,
                    e2e=dict(value=e2e_val, unit="HR Mpix/s", h2d_bytes_per_step=img.nbytes,
                             d2h_bytes_per_step=out_host.numel() * 4),
                    gpu_launches=args.steps * (api.joint_launches(
                        NITER, graph=True, multi_kernel_lists=st["multi_kernel_lists"]) + 3),
                    clocks=clk.summary(t_load0, t_load1, timed=(t_timed0, t_timed1)),
                    autotune=tuned,
                    breakdown=dict(joint_ms=statistics.mean(joint_ms),
                                   lrop_apply_ms=statistics.mean(apply_ms),
                                   joint_phases_ms={k: v / calls for k, v in prof.items()
                                                    if k.endswith("_ms")},
                                   joint_stats=dict(R0=st["R0"], iters=st["iters"])),
                    extras=extras)
        if args.cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(img)
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def measure_extras(api, torch, img, dev, flush, stream):
    """Secondary numbers (not the headline): plain GLU (no joint) and the adjoint."""
    H, W = img.shape[:2]
    h, w = api.lr_dims(H, W, SCALE)
    hr = torch.from_numpy(img).to(dev)
    res = {}

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    lr = api.glu_downsample(hr, SCALE, api.GLU_DOWN_GRID)
    p = api.glu_params(S=WIN)
    theta = api.Theta.empty(H, W, SCALE, WIN, api.GLU_W_UNORM16, dev)
    T = torch.rand((h, w, 3), device=dev)
    out = torch.empty((H, W, 3), dtype=torch.float32, device=dev)

    def plain():
        api.glu_downsample(hr, SCALE, api.GLU_DOWN_GRID, lr=lr)
        api.glu_optimize(hr, lr, p, SCALE, theta=theta)
        api.glu_apply(theta, T, out=out)

    ms = timed(plain)
    res["plain_glu_minus_mpix_s"] = H * W / ms / 1e3
    ms_s = timed(lambda: api.glu_optimize(hr, lr, p, SCALE, theta=theta))
    res["search_ms"] = ms_s
    ms_a = timed(lambda: api.glu_apply(theta, T, out=out))
    res["apply_ms"] = ms_a
    G = torch.randn((H, W, 3), device=dev)
    gT = torch.empty((h, w, 3), device=dev)
    gw = torch.empty((H, W), device=dev)
    # the adjoint for one Theta and many calls (a fit through the upsampler): the plan (inverse
    # pixel-to-LR map) is built once; also the workspace form without a plan
    ms_plan = timed(lambda: api.glu_apply_backward_plan(theta), reps=3)
    plan = api.glu_apply_backward_plan(theta)
    ms_b = timed(lambda: api.glu_apply_backward(theta, T, G, grad_lr=gT, grad_w=gw, plan=plan))
    ms_bw = timed(lambda: api.glu_apply_backward(theta, T, G, grad_lr=gT, grad_w=gw))
    res["backward_ms"] = ms_b
    res["backward_vs_apply"] = ms_b / ms_a
    res["backward_plan_build_ms"] = ms_plan
    res["backward_workspace_form_ms"] = ms_bw
    # GLU* (Eq. 4, every pair of window pixels) on the same guide and LR image
    pe = api.glu_params(S=WIN, mode=api.GLU_MODE_EXACT)
    th_e = api.Theta.empty(H, W, SCALE, WIN, api.GLU_W_F32, dev)
    ms_e = timed(lambda: api.glu_optimize(hr, lr, pe, SCALE, theta=th_e), reps=5)
    pairs = WIN * WIN * (WIN * WIN - 1) // 2
    res["exact_ms"] = ms_e
    res["exact_alu_frac"] = (H * W * pairs * EXACT_OPS_PER_PAIR / (ms_e / 1e3)) / (
        torch.cuda.get_device_properties(dev).multi_processor_count * 128 * 2.07e9)
    # the least-squares LR update alternated with Algorithm 1 (not the paper's method) beside
    # Algorithm 2 on the same guide, window and iteration count: time and final residual
    pl = api.glu_params(S=WIN, N=NITER)
    wl = torch.empty(api.glu_ls_joint_workspace_size(H, W, SCALE, pl) + 256, dtype=torch.uint8,
                     device=dev)
    lr_l = torch.empty((h, w, 3), dtype=torch.float32, device=dev)
    th_l = api.Theta.empty(H, W, SCALE, WIN, api.GLU_W_F32, dev)
    ms_l = timed(lambda: api.glu_ls_joint_optimize(hr, SCALE, pl, lr_out=lr_l, theta=th_l,
                                                   err_map=False, stats=False, workspace=wl),
                 reps=5)
    _, _, _, st_l = api.glu_ls_joint_optimize(hr, SCALE, pl, lr_out=lr_l, theta=th_l,
                                              err_map=False, workspace=wl)
    _, _, _, st_j = api.glu_joint_optimize(hr, SCALE, pl, err_map=False)
    res["ls_joint"] = dict(ms=ms_l, R0=st_l["R0"], kept=st_l["kept"],
                           residual=([st_l["R0"]] + st_l["residuals"])[st_l["kept"]],
                           alg2_residual=st_j["iters"][-1]["residual"] if st_j["iters"]
                           else st_j["R0"])
    res["batch16"] = measure_batch(api, torch, dev, timed)
    if VIDEO_FRAMES > 0:
        res["video"] = measure_video(api, torch, dev, VIDEO_FRAMES)
    return res


def measure_video(api, torch, dev, n_frames):
    """The video workload: n 3840x2160 float16 frames (cells moving 2 px/frame, 5% of dots
    re-drawn per frame), BOX x8 -> 3x3 Gaussian + gamma 0.8 on the LR image -> Algorithm 1
    (5x5) -> Eq. 1 into float16 frames. Every frame is a different resident buffer (5.97 GB in
    all for 120 frames), so no frame's input is in L2 when it starts. Three ways of issuing the
    same kernels: one CUDA graph per frame slot (LR operator forked beside Algorithm 1), the
    same launches issued directly, and the separate Python-level calls one after another.
    Per-frame latency = device time between the events around that frame's launches."""
    import time
    from paper_2307_09582_gb300.inputs import render_u8
    from paper_2307_09582_gb300.inputs.workloads import video_scene
    sc = video_scene()
    H, W, s, S = sc.height, sc.width, 8, 5
    t0 = time.time()
    frames = torch.empty((n_frames, H, W, 3), dtype=torch.float16, device=dev)
    for f in range(n_frames):
        u8 = torch.from_numpy(render_u8(sc, frame=f)).to(dev)
        frames[f] = (u8.to(torch.float32) / 255).to(torch.float16)
    render_s = time.time() - t0
    outs = torch.empty_like(frames)
    p = api.glu_params(S=S)
    st = torch.cuda.current_stream()

    def timeline(issue):
        for f in range(min(3, n_frames)):
            issue(f)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_frames + 1)]
        ev[0].record(st)
        for f in range(n_frames):
            issue(f)
            ev[f + 1].record(st)
        ev[-1].synchronize()
        lat = sorted(ev[f].elapsed_time(ev[f + 1]) for f in range(n_frames))
        tot = ev[0].elapsed_time(ev[-1])
        pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
        return dict(fps=n_frames / (tot / 1e3), ms_total=tot, p50_ms=pct(0.5), p99_ms=pct(0.99))

    res = dict(frames=n_frames, H=H, W=W, scale=s, window=S, render_s=render_s)
    v = api.Video(H, W, s, p, out_dtype=torch.float16, overlap=True)
    v.run(frames[0], outs[0])   # a direct frame first, so the tuner has chosen before capture
    torch.cuda.synchronize()
    for f in range(n_frames):
        v.bind(f, frames[f], outs[f])
    res["graph"] = timeline(lambda f: v.launch(f))
    res["direct"] = timeline(lambda f: v.run(frames[f], outs[f]))
    v.close()
    vs = api.Video(H, W, s, p, out_dtype=torch.float16, overlap=False)
    for f in range(n_frames):
        vs.bind(f, frames[f], outs[f])
    res["graph_no_fork"] = timeline(lambda f: vs.launch(f))
    vs.close()
    # Theta reused by two operators (Gaussian + gamma 0.8; box + saturation 1.3): one pipeline
    # with both operators (one Algorithm 1 per frame, each operator's branch forked beside it)
    # against two single-operator pipelines per frame
    ops2 = [(1, 1.0, 0.8), (0, 1.3, 1.0)]
    outs2 = torch.empty((n_frames, H, W, 3), dtype=torch.float16, device=dev)
    vm = api.Video(H, W, s, p, out_dtype=torch.float16, overlap=True, ops=ops2)
    for f in range(n_frames):
        vm.bind(f, frames[f], [outs[f], outs2[f]])
    va = api.Video(H, W, s, p, out_dtype=torch.float16, overlap=True, ops=ops2[:1])
    vb = api.Video(H, W, s, p, out_dtype=torch.float16, overlap=True, ops=ops2[1:])
    for f in range(n_frames):
        va.bind(f, frames[f], outs[f])
        vb.bind(f, frames[f], outs2[f])
    res["two_operators"] = dict(
        shared_theta_graph=timeline(lambda f: vm.launch(f)),
        two_pipelines=timeline(lambda f: (va.launch(f), vb.launch(f))))
    res["two_operators"]["speedup"] = (res["two_operators"]["shared_theta_graph"]["fps"] /
                                       res["two_operators"]["two_pipelines"]["fps"])
    vm.close()
    va.close()
    vb.close()
    del outs2
    h, w = api.lr_dims(H, W, s)
    lr = torch.empty((h, w, 3), dtype=torch.float32, device=dev)
    t1, T = torch.empty_like(lr), torch.empty_like(lr)
    theta = api.Theta.empty(H, W, s, S, api.GLU_W_UNORM16, dev)

    def separate(f):
        api.glu_downsample(frames[f], s, api.GLU_DOWN_BOX, lr=lr)
        api.glu_fx_filter3(lr, 1, out=t1)
        api.glu_fx_point(t1, 1.0, 0.8, out=T)
        api.glu_optimize(frames[f], lr, p, s, theta=theta)
        api.glu_apply(theta, T, out=outs[f])

    res["separate_calls"] = timeline(separate)
    res["graph_vs_separate"] = res["graph"]["fps"] / res["separate_calls"]["fps"]
    res["gpu_launches_per_frame"] = 5
    del frames, outs
    torch.cuda.empty_cache()
    return res


def measure_batch(api, torch, dev, timed):
    """The 16-image batch (uneven sizes, scales {4, 8, 16}, windows {3, 5}, 3 iterations of
    Algorithm 2): all of them in one batched call against 16 single-image calls, same outputs
    and workspace."""
    from paper_2307_09582_gb300.inputs import render_u8
    from paper_2307_09582_gb300.inputs.workloads import batch_scenes
    items = [(render_u8(sc), s, S) for sc, s, S in batch_scenes()]
    hrs = [torch.from_numpy(i).to(dev) for i, _, _ in items]
    scales = [s for _, s, _ in items]
    Ss = [S for _, _, S in items]
    p = api.glu_params(N=BATCH_NITER)
    ps = [api.glu_params(S=S, N=BATCH_NITER) for S in Ss]
    lrs = [torch.empty((*api.lr_dims(h.shape[0], h.shape[1], s), 3), dtype=torch.uint8,
                       device=dev) for h, s in zip(hrs, scales)]
    thetas = [api.Theta.empty(h.shape[0], h.shape[1], s, S, api.GLU_W_UNORM16, dev)
              for h, s, S in zip(hrs, scales, Ss)]
    need = api.glu_joint_batched_workspace_size([h.shape[:2] for h in hrs], scales, Ss, p)
    wsb = torch.empty(need + 256, dtype=torch.uint8, device=dev)

    def batched():
        api.glu_joint_optimize_batched(hrs, scales, p, Ss, lrs=lrs, thetas=thetas,
                                       err_maps=False, stats=False, workspace=wsb)

    def sequential():
        for k in range(len(hrs)):
            api.glu_joint_optimize(hrs[k], scales[k], ps[k], lr_out=lrs[k], theta=thetas[k],
                                   err_map=False, stats=False, workspace=wsb)

    npx = sum(h.shape[0] * h.shape[1] for h in hrs)
    mb = timed(batched, reps=5)
    msq = timed(sequential, reps=5)
    return dict(images=len(hrs), mpix=npx / 1e6, batched_ms=mb, sequential_ms=msq,
                batched_mpix_s=npx / mb / 1e3, sequential_mpix_s=npx / msq / 1e3,
                speedup=msq / mb)


def run_kernel_case(args):
    """One kernel on an input larger than L2, a few launches (the target of an ncu capture):
    search / apply / backward / exact (GLU*, float32 weights) on a 7680x4320 guide at scale 8,
    window 5; trials = the joint 4K workload (its first trial launch is iteration 1); tail = the
    bench step's LR operator + Eq. 1 after the 4K joint call."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2307_09582_gb300 import api
    from paper_2307_09582_gb300.inputs import Scene, joint_4k_scene, render_u8
    dev = torch.device("cuda", 0)
    if args.variant is not None and args.kernel_case in ("search", "apply", "tail"):
        api.tune_force(api.GLU_TUNE_SEARCH if args.kernel_case == "search" else api.GLU_TUNE_APPLY,
                       args.variant)
    if args.kernel_case == "trials":
        img = render_u8(joint_4k_scene())
        hr = torch.from_numpy(img).to(dev)
        for _ in range(args.case_reps):
            api.glu_joint_optimize(hr, SCALE, api.glu_params(S=WIN, N=NITER), stats=False)
        torch.cuda.synchronize()
        return 0
    if args.kernel_case == "tail":
        # the bench step's tail on its own inputs: the 4K joint result, then per rep an L2 flush
        # (a 256 MB write) and the LR operator + Eq. 1 (glu_apply_lrop)
        img = render_u8(joint_4k_scene())
        hr = torch.from_numpy(img).to(dev)
        H, W = img.shape[:2]
        h, w = api.lr_dims(H, W, SCALE)
        lr = torch.empty((h, w, 3), dtype=torch.uint8, device=dev)
        theta = api.Theta.empty(H, W, SCALE, WIN, api.GLU_W_UNORM16, dev)
        api.glu_joint_optimize(hr, SCALE, api.glu_params(S=WIN, N=NITER), lr_out=lr,
                               theta=theta, stats=False)
        T = torch.empty((h, w, 3), dtype=torch.float32, device=dev)
        out = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        for _ in range(args.case_reps):
            flush.zero_()
            api.glu_apply_lrop(theta, lr, filter=0, sat=1.3, gamma=1.0, target=T, out=out)
        torch.cuda.synchronize()
        return 0
    H, W = 4320, 7680
    img = render_u8(Scene(width=W, height=H, n_cells=1600, n_dots=8000, n_lines=400, seed=7))
    hr = torch.from_numpy(img).to(dev)
    lr = api.glu_downsample(hr, SCALE, api.GLU_DOWN_GRID)
    p = api.glu_params(S=WIN)
    theta = api.Theta.empty(H, W, SCALE, WIN, api.GLU_W_UNORM16, dev)
    err = torch.empty((H, W), dtype=torch.float32, device=dev)
    h, w = api.lr_dims(H, W, SCALE)
    T = torch.rand((h, w, 3), device=dev)
    out = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    api.glu_optimize(hr, lr, p, SCALE, theta=theta, err_map=err)
    if args.kernel_case == "exact":
        pe = api.glu_params(S=WIN, mode=api.GLU_MODE_EXACT)
        th_e = api.Theta.empty(H, W, SCALE, WIN, api.GLU_W_F32, dev)
        for _ in range(args.case_reps):
            api.glu_optimize(hr, lr, pe, SCALE, theta=th_e, err_map=err)
        torch.cuda.synchronize()
        return 0
    if args.kernel_case == "backward":
        # the plan is built once; each rep runs the planned adjoint, then the workspace form
        plan = api.glu_apply_backward_plan(theta)
        G = torch.randn((H, W, 3), device=dev)
        for _ in range(args.case_reps):
            api.glu_apply_backward(theta, T, G, plan=plan)
            api.glu_apply_backward(theta, T, G)
        torch.cuda.synchronize()
        return 0
    for _ in range(args.case_reps):
        if args.kernel_case == "search":
            api.glu_optimize(hr, lr, p, SCALE, theta=theta, err_map=err)
        elif args.kernel_case == "apply":
            api.glu_apply(theta, T, out=out)
    torch.cuda.synchronize()
    return 0


def run_quality_sweep(args):
    """Self-upsampling quality over scaling ratios and window sizes on the 3840x2160 guide, after
    the paper's large-ratio experiment and its window-size table (Sec. 5): PSNR of Eq. 1 applied
    to the LR image itself against the guide, for GLU- (Algorithm 1 on the grid-downsampled LR),
    GLU (Algorithm 2, N = 3, STRICT), GLU* (all pairs, Eq. 4) and GNU (weight 1), with the time
    of each call. One JSON line (not a throughput measurement)."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2307_09582_gb300 import api
    from paper_2307_09582_gb300.inputs import joint_4k_scene, render_u8
    dev = torch.device("cuda", 0)
    img = render_u8(joint_4k_scene())
    hr = torch.from_numpy(img).to(dev)
    ref = hr.to(torch.float32) / 255.0

    def psnr(th, lr):
        out = api.glu_apply(th, lr.to(torch.float32) / 255.0)
        mse = ((out - ref).double() ** 2).mean()
        return float(10 * torch.log10(1.0 / mse))

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        return r, a.elapsed_time(b)

    rows = []
    for s_ in (8, 16, 32, 64, 128):
        lr = api.glu_downsample(hr, s_, api.GLU_DOWN_GRID)
        for S in (3, 5, 7, 9):
            row = dict(scale=s_, window=S)
            for name, mode, wfmt in (("glu_minus", api.GLU_MODE_FAST, api.GLU_W_F32),
                                     ("glu_star", api.GLU_MODE_EXACT, api.GLU_W_F32),
                                     ("gnu", api.GLU_MODE_GNU, api.GLU_W_F32)):
                p = api.glu_params(S=S, mode=mode)
                api.glu_optimize(hr, lr, p, s_, wfmt=wfmt)   # warm-up (and tuning)
                (th, _), ms = timed(lambda: api.glu_optimize(hr, lr, p, s_, wfmt=wfmt))
                row[name] = dict(psnr=psnr(th, lr), ms=ms)
            # Algorithm 2 where a trial's re-searched area (S^2 blocks of s^2 pixels) stays
            # moderate: its trials at the largest windows and ratios run for seconds
            if s_ * S <= 384:
                pj = api.glu_params(S=S, N=3)
                try:
                    (lj, tj, _, st), ms = timed(lambda: api.glu_joint_optimize(hr, s_, pj))
                    row["glu"] = dict(psnr=psnr(tj, lj), ms=ms,
                                      iterations=len(st["iters"]) if st else None)
                except Exception as e:   # noqa: BLE001 - recorded, the sweep goes on
                    row["glu"] = dict(error=str(e).splitlines()[0])
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps(dict(sweep="self-upsampling PSNR (dB) vs scale and window, 3840x2160 "
                                "synthetic guide", rows=rows,
                          status=api.glu_device_status())))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="glu", choices=["glu", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    ap.add_argument("--kernel-case",
                    choices=["search", "apply", "backward", "trials", "exact", "tail"],
                    help="run one kernel on a profiling case and exit (no JSON line)")
    ap.add_argument("--case-reps", type=int, default=3)
    ap.add_argument("--quality-sweep", action="store_true",
                    help="self-upsampling PSNR over scales 8-128 and windows 3-9, then exit")
    ap.add_argument("--video-frames", type=int, default=VIDEO_FRAMES)
    ap.add_argument("--variant", type=int, default=None,
                    help="with --kernel-case search/apply: the kernel variant to run")
    args = ap.parse_args()
    globals()["VIDEO_FRAMES"] = args.video_frames
    if args.kernel_case:
        return run_kernel_case(args)
    if args.quality_sweep:
        return run_quality_sweep(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_glu(args)


if __name__ == "__main__":
    sys.exit(main())
