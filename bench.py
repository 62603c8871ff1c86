"""Throughput of one GO-Surf optimisation step on GB300 (rays/s per full step).

One step = gs_sample_rays + gs_forward_backward (fused fwd+bwd incl. the smoothness
second-order path) + gs_adam_step over every grid and decoder parameter, on the room
workload (8x6x3 m, 1000 poses at 640x480, 8192 rays x (64 + 32) samples, 4096 smoothness
points, 75.7 M parameters).  Frames are rendered once on the host and stay resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The plain sampler reads no parameters, so each step's batch is sampled on a side stream
during the step before (double-buffered; --no-pipeline samples in line); the work per step
is the same.

--impl reference times the FP64 CPU oracle (the only baseline this method has here) on
the host cores, each step a bounded sample of the same workload.  Under torchrun each rank
runs an independent replica (rays are independent; no collective) and rank 0 prints the
aggregate.  Prints ONE JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/s per fwd+bwd step (samples/ray stated); gather/scatter HBM GB/s vs peak"
WORKLOAD = "room-8192x96"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        """Starts sampling every 50 ms and returns once the first sample is in (nvidia-smi takes
        a moment to start), so that the timed region that follows is covered."""
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.f.name) == 0:
                time.sleep(0.02)
        except Exception:
            self.p = None
        self.t_start = time.time()

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t_stop = time.time()
        time.sleep(0.06)  # one more sample at the end of the region
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",")[1:] + [r.split(",")[0]] for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)

        def stamp(r):
            try:
                import datetime
                return datetime.datetime.strptime(r[-1].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except Exception:
                return None
        inside = [r for r in rows if stamp(r) is not None and self.t_start - 0.06 <= stamp(r) <= t_stop + 0.06]
        rows = inside or rows
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def replica_seed(rank: int) -> int:
    """Each replica samples its own rays: the seed of rank r (rays are independent, so the
    replicas share nothing and exchange nothing)."""
    return 3 + 1000 * rank


def max_over_ranks(values, world: int, device: str = "cuda"):
    """Element-wise maximum of per-rank timings over all ranks (the slowest replica sets the
    whole job's time); the identity on one rank."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def aggregate_rays_per_s(rays_per_replica_step: int, steps: int, world: int, ms: float) -> float:
    """Whole-job throughput: the rays every replica processed over the slowest replica's time."""
    return rays_per_replica_step * steps * world / (ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def step_config(w, args, world, n_frames):
    """The workload and the form of the timed step, as both arms print it (no measured values)."""
    if w.prop_samples > 0:
        return {"workload": w.name, "rays": w.rays, "samples_per_ray": w.prop_samples,
                "guided_of_those": w.prop_guided, "lr_prop": w.lr_prop,
                "fallback_samples_per_ray": w.n_samples, "pretrain_steps": args.prop_pretrain,
                "parallelism": f"replicas{world}"}
    paper = w.arch == "paper"
    recompute = args.recompute
    pipelined = w.imp_coarse == 0 and not args.no_pipeline and not args.poses
    return {"workload": w.name, "rays": w.rays, "samples_per_ray": w.n_samples, "smooth_points": w.n_smooth,
            "params": w.layout()[2], "grid_params": w.layout()[1], "frames": n_frames,
            "resolution": [w.width, w.height], "parallelism": f"replicas{world}",
            "model": ("paper: colour grid (6 features, finest level) + view direction, decoders with "
                      "2 hidden layers of 32" if paper else "compact: decoders 16-32-16 and 15-32-3"),
            "activations": "recomputed" if recompute else f"stored ({624 if paper else 400} B/sample)",
            "sampler": (f"importance: {w.imp_coarse} coarse + {w.imp_steps} x {w.imp_per_step}"
                        if w.imp_coarse > 0 else f"stratified {w.n_strat} + depth-guided {w.n_guided}"),
            "pipeline": ("the next step's batch sampled on a side stream during this step (double-buffered)"
                         if pipelined else "in line"),
            "calls": ("gs_eikonal (grid part deferred to the render call) + " if args.eikonal else "") +
                     ("gs_forward + gs_backward" if args.split else "gs_forward_backward"),
            "loss_terms": "rgb, depth, sdf, fs, smooth" + (", eikonal (lam 1, free-space samples)"
                                                           if args.eikonal else ""),
            "poses": ("refined: per-frame (dt, nu), gs_pose_apply + gs_pose_backward" +
                      (" + gs_eikonal_pose_backward" if args.eikonal else "") + " + Adam 5e-4 in every step"
                      if args.poses else "fixed"),
            "l2": "inputs larger than L2: 1.2 GB of parameter/gradient/moment state streamed per step"}


def run_ours(args):
    import numpy as np
    import torch

    import paper_2206_14735_gb300 as gs
    import scenegen as sg
    from paper_2206_14735_gb300 import build as gbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    gbuild.build()
    w = sg.WORKLOADS[args.workload]
    t0 = time.time()
    fr = sg.make_frames(w, n_frames=args.frames, with_gt=args.sampler_report > 0)
    t_frames = time.time() - t0
    paper = w.arch == "paper"
    recompute = args.recompute
    ctx = gs.Context(w, store_activations=not recompute)
    dfr = gs.DeviceFrames(fr.rgb, fr.depth, fr.c2w, fr.fx, fr.fy, fr.cx, fr.cy)
    theta0 = sg.init_params(w)
    theta = torch.zeros((len(theta0) + 3) // 4 * 4, device="cuda")  # Adam works on 4-float vectors
    theta[:len(theta0)] = torch.from_numpy(theta0).cuda()
    grad, m, v = torch.zeros_like(theta), torch.zeros_like(theta), torch.zeros_like(theta)
    n_grid_ = w.layout()[1]
    # BF16 form: the grid copy the gathers read, refreshed by every Adam step
    mirror = theta[:n_grid_].to(torch.bfloat16).view(torch.int16).contiguous() if ctx.bf16 else None
    # the Eikonal term leaves its grid part to the render kernel's scatter (deferred records in
    # the batch), so its call comes before the render call
    defer_eik = args.eikonal
    batch = gs.Batch.allocate(w.rays, w.n_samples, w.n_smooth, dz=args.poses, dz_width=32 if paper else 16,
                              eik=defer_eik)
    loss = torch.empty(6, device="cuda")
    eik = torch.zeros(1, device="cuda")  # L_eik when --eikonal (Sec. 3.3, lam_eik = 1)
    stream = torch.cuda.current_stream()
    seed = replica_seed(rank)
    b1, b2 = w.betas

    # camera-pose refinement (--poses): per-frame corrections xi = (dt, nu), the corrected
    # poses applied before sampling, their gradient after the render call, Adam at 5e-4
    if args.poses:
        n_fr = dfr.c2w.shape[0]
        xi = torch.zeros((6 * n_fr + 3) // 4 * 4, device="cuda")
        xi_m, xi_v, xi_g = torch.zeros_like(xi), torch.zeros_like(xi), torch.zeros_like(xi)
        c2w_cur = torch.empty_like(dfr.c2w)
        dfr_pose = dfr.with_poses(c2w_cur)

    def frames_now():
        if not args.poses:
            return dfr
        ctx.pose_apply(dfr.c2w, xi[:6 * n_fr].view(n_fr, 6), c2w_cur)
        return dfr_pose

    def sample(k, b=batch):
        fr_k = frames_now()
        if w.imp_coarse > 0:  # the paper's hierarchical importance sampler (reads theta)
            ctx.sample_importance(fr_k, theta, seed, k, b)
        else:
            ctx.sample_rays(fr_k, seed, k, b)

    # The plain sampler does not read theta: the batch of step k + 1 is sampled on a side
    # stream (its own context, a second batch buffer) while step k renders and updates, and
    # lands on the SMs that the render kernel's last round leaves idle.  The importance
    # sampler reads theta, so it stays in line.
    pipelined = w.imp_coarse == 0 and not args.no_pipeline and not args.poses
    if pipelined:
        ctx_s = gs.Context(w)
        side = torch.cuda.Stream()
        batches = [batch, gs.Batch.allocate(w.rays, w.n_samples, w.n_smooth, eik=defer_eik)]
        ev_ready = [torch.cuda.Event(), torch.cuda.Event()]  # batch j sampled
        ev_free = [torch.cuda.Event(), torch.cuda.Event()]   # batch j no longer read
        sample_ev = {}

        def issue_sample(k):
            j = k % 2
            side.wait_event(ev_free[j])
            e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            e[0].record(side)
            with torch.cuda.stream(side):
                ctx_s.sample_rays(dfr, seed, k, batches[j])
            e[1].record(side)
            ev_ready[j].record(side)
            sample_ev[k] = e
    else:
        batches = [batch, batch]

    def step(k, ev=None, io=None):
        """One step; io = (dloss on the device, pinned loss and counts buffers) for the
        end-to-end loop: the upstream seed comes from the host and the results go back."""
        b = batches[k % 2]
        dl = io[0] if io is not None else None
        if ev is not None:
            ev[0].record(stream)
        if pipelined:
            stream.wait_event(ev_ready[k % 2])
        else:
            sample(k, b)
        if ev is not None:
            ev[1].record(stream)
        if defer_eik:  # before the render call, which adds the Eikonal term's grid part
            ctx.eikonal(theta, b, loss=eik, grad=grad)
        if ev is not None:
            ev[5].record(stream)
        if args.split:
            ctx.forward(theta, b, loss, theta_bf16=mirror)
            ctx.backward(theta, b, dl, grad, theta_bf16=mirror)
        else:
            ctx.forward_backward(theta, b, dl, loss, grad, theta_bf16=mirror)
        if ev is not None:
            ev[2].record(stream)
        if args.eikonal and not defer_eik:
            ctx.eikonal(theta, b, loss=eik, grad=grad)
        if args.poses:
            ctx.pose_backward(theta, dfr_pose, xi[:6 * n_fr].view(n_fr, 6), b, xi_g[:6 * n_fr].view(n_fr, 6))
            if args.eikonal:  # the Eikonal term moves with the poses too (x-Hessian of phi)
                ctx.eikonal_pose_backward(theta, dfr_pose, xi[:6 * n_fr].view(n_fr, 6), b,
                                          xi_g[:6 * n_fr].view(n_fr, 6))
            ctx.adam_step(xi, xi_g, xi_m, xi_v, k + 1, 0.0, 5e-4, n_grid=0)
        if ev is not None:
            ev[3].record(stream)
        if io is not None:  # before the batch is handed back to the sampler
            io[1].copy_(loss, non_blocking=True)
            io[2].copy_(b.counts, non_blocking=True)
        if pipelined:
            ev_free[k % 2].record(stream)
            issue_sample(k + 1)
        ctx.adam_step(theta, grad, m, v, k + 1, w.lr_grid, w.lr_mlp, b1, b2, w.adam_eps, theta_bf16=mirror)
        if ev is not None:
            ev[4].record(stream)

    if pipelined:
        issue_sample(0)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    ctx.sync_status()

    # ---- device-timed region: K full steps, inputs resident in HBM ----
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    start.record(stream)
    for k in range(args.steps):
        step(args.warmup + k, evs[k])
    stop.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = start.elapsed_time(stop)
    per = {"sample": [], "render": [], "adam": []}
    # after the render call: the Eikonal call (paper architecture) and / or the pose calls
    extra = ("eikonal" if args.eikonal and not defer_eik else ("poses" if args.poses else None))
    if extra:
        per[extra] = []
    if defer_eik:
        per["eikonal"] = []  # the Eikonal call before the render call
    for k, e in enumerate(evs):
        if pipelined:  # the sampler's own time on the side stream (overlapped with the step before)
            se = sample_ev[args.warmup + k]
            per["sample"].append(se[0].elapsed_time(se[1]))
        else:
            per["sample"].append(e[0].elapsed_time(e[1]))
        per["render"].append(e[5].elapsed_time(e[2]))
        if defer_eik:
            per["eikonal"].append(e[1].elapsed_time(e[5]))
        if extra:
            per[extra].append(e[2].elapsed_time(e[3]))
        per["adam"].append(e[3].elapsed_time(e[4]))
    avg = {k: sum(vv) / len(vv) for k, vv in per.items()}
    ctx.sync_status()
    lossv = loss.cpu().numpy().tolist() + (eik.cpu().numpy().tolist() if args.eikonal else [])

    # ---- end-to-end region: the same steps through the public API with host round trips ----
    # Every step copies its upstream seed in from pinned host memory and its six losses and
    # four counts out to a pinned double buffer; the host reads step k's results while step
    # k + 1 runs (no idle GPU between steps).
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    dl_host = torch.tensor([0, 0, 0, 0, 0, 1.0], dtype=torch.float32).pin_memory()
    outs = [(torch.empty(6, dtype=torch.float32).pin_memory(), torch.empty(4, dtype=torch.int32).pin_memory(),
             torch.cuda.Event()) for _ in range(2)]
    dl_dev = torch.empty(6, device="cuda")
    seen = []
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    base = args.warmup + args.steps
    for k in range(e2e_steps):
        dl_dev.copy_(dl_host, non_blocking=True)
        o = outs[k % 2]
        step(base + k, io=(dl_dev, o[0], o[1]))
        o[2].record(stream)
        if k >= 1:
            p = outs[(k - 1) % 2]
            p[2].synchronize()
            seen.append((float(p[0][5]), int(p[1][0])))
    p = outs[(e2e_steps - 1) % 2]
    p[2].synchronize()
    seen.append((float(p[0][5]), int(p[1][0])))
    e2e_s = time.perf_counter() - t1
    assert len(seen) == e2e_steps and all(math.isfinite(x) for x, _ in seen)

    ms, e2e_s = max_over_ranks([ms, e2e_s], world)
    if rank != 0:
        return None

    value = aggregate_rays_per_s(w.rays, args.steps, world, ms)
    peaks, kind = _peaks()
    S = w.rays * w.n_samples
    n_grid = w.layout()[1]
    # algorithmic bytes: gather 4 levels x 8 corners x 16 B (8 B from the BF16 copy) and 512 B
    # of FP32 gradient scattered per sample; Adam 32 B per parameter (+2 B per grid entry copied)
    # (paper architecture: + the colour grid's 8 corners x 24 B gathered and scattered)
    render_bytes = S * (2 * (512 + 192) if paper else (256 if ctx.bf16 else 512) + 512)
    adam_bytes = w.layout()[2] * 32 + (2 * n_grid_ if ctx.bf16 else 0)
    dom = max(("render", "adam"), key=lambda k: avg[k])
    dom_bytes = render_bytes if dom == "render" else adam_bytes
    achieved = dom_bytes / (avg[dom] / 1e3) / 1e9
    peak = peaks["hbm_gbs"]
    traffic = args.traffic_render if dom == "render" else args.traffic_adam
    default_step = (w.name == WORKLOAD and not recompute and not args.split and not args.eikonal and
                    not args.poses and args.frames in (None, 50))
    if traffic is None and dom == "render" and default_step:
        traffic = _profiled_traffic("render_tc_kernel_room-8192x96.md",
                                    ("gs_render_tc.cuh", "gs_tc.cuh", "gs_device.cuh"))
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "rays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if ctx.bf16 else "f32", "data": "synthetic",
        "config": step_config(w, args, world, fr.depth.shape[0]),
        "samples_per_s": round(value * w.n_samples, 1), "frame_render_s": round(t_frames, 1),
        "kernels_ms": {k: round(vv, 4) for k, vv in avg.items()},
        "roofline": {"kernel": ("render call: paper_tc_kernel (fused gathers / tcgen05 decoders / compositing "
                                "/ backward / scatter) + paper_smooth_kernel + paper_combine_kernel" if paper else
                                "render call: render_tc_kernel (fused gather / tcgen05 decoders / compositing / "
                                "backward / scatter, 90 % of the call) + smooth_kernel + finalize_kernel")
                     if dom == "render" else "adam_kernel", "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_kind": f"{kind} hbm_gbs (copy)",
                     "algorithmic_bytes_per_launch": dom_bytes},
        "adam": {"achieved_gbs": round(adam_bytes / (avg['adam'] / 1e3) / 1e9, 1),
                 "frac_of_peak": round(adam_bytes / (avg['adam'] / 1e3) / 1e9 / peak, 4)},
        "e2e": {"value": round(w.rays * e2e_steps * world / e2e_s, 1), "unit": "rays/s",
                "h2d_bytes_per_step": 24, "d2h_bytes_per_step": 40, "steps": e2e_steps,
                "what": "per step: H2D dloss seed (pinned), the C-ABI calls of the step, D2H loss and counts into a "
                        "pinned double buffer that the host reads one step later; frames resident on the device"},
        "gpu_launches": ((9 if args.split else 6) + ((2 if paper else 1) if args.eikonal else 0) +
                         (3 if args.poses else 0) + (1 if args.poses and args.eikonal else 0)) * args.steps,
        "clocks": clk,
        "loss_last": [round(x, 6) for x in lossv],
    }
    if args.diff_report:
        line["differentiation"] = differentiation_report(w, dfr, theta, mirror)
    if args.mesh_report > 0:
        line["mesh_report"] = mesh_report(w, ctx, args.mesh_report)
    if args.sampler_report > 0 and w.imp_coarse > 0:
        line["sampler_report"] = sampler_report(w, fr, dfr, args.sampler_report)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, fr, args.cpu_rays)
    if rank == 0 and world == 1 and w.name == WORKLOAD and args.target_steps > 0:
        line["target_pair"] = target_pair(args)
    return line


def target_pair(args):
    """The pair of forms the method's target compares, measured in the same run: the plain
    FP32 form at 65536 rays x (64 + 32) samples and the BF16 + learned-proposal form at 65536
    rays x 32 samples (plain 96 as its fallback), both trained for the same number of steps
    from the same initial parameters on the room scene with 30 % of every depth frame dropped
    in discs; rays/s of each over those steps and the final rendered-depth L1 against the
    noise-free depth."""
    import scenegen as sg
    import paper_2206_14735_gb300 as gs
    wp = sg.WORKLOADS["room-prop-bf16-65536x32"]
    frp = sg.make_frames(wp, n_frames=args.frames, with_gt=True)
    dfrp = gs.DeviceFrames(frp.rgb, frp.depth, frp.c2w, frp.fx, frp.fy, frp.cx, frp.cy)
    tail = max(1, args.target_steps // 8)
    rep = proposal_report(wp, frp, dfrp, args.target_steps, tail=tail)
    plain, prop = rep["plain"], rep["proposal"]
    l1_plain, l1_prop = plain["depth_l1_gt_m"], prop["with_proposal"]["depth_l1_gt_m"]
    speed = prop["tail_rays_per_s"] / plain["tail_rays_per_s"]
    keys = ("rays_per_s", "tail_rays_per_s", "samples_per_ray")
    return {"workload": wp.name, "steps_each": args.target_steps,
            "plain_fp32": {**{k: plain[k] for k in keys}, "depth_l1_gt_m": l1_plain,
                           "depth_l1_gt_dropped_m": plain["depth_l1_gt_dropped_m"]},
            "bf16_proposal": {**{k: prop[k] for k in keys}, "steps_on_proposal": prop["proposal_steps"],
                              "tail_steps_on_proposal": prop["tail_steps_on_proposal"], "depth_l1_gt_m": l1_prop,
                              "depth_l1_gt_dropped_m": prop["with_proposal"]["depth_l1_gt_dropped_m"]},
            "rays_per_s_ratio": round(speed, 4), "depth_l1_ratio": round(l1_prop / l1_plain, 4),
            "target_met": bool(speed > 1.0 and l1_prop <= 1.05 * l1_plain),
            "what": (f"{rep['what']}; the rays/s ratio compares the last {tail} steps of each (the trained "
                     f"regime, where the controller may use the proposal)")}


def _eval_depth(ctx, w, dfr, gt, theta, sampler, q=None, R=65536, seed=99, mirror=None):
    """Rendered depth of R fresh rays against the noise-free depth: mean |d_hat - D_gt| over
    rays with D_gt > 0, and over those whose observed depth was dropped (D = 0)."""
    import numpy as np
    import torch

    import paper_2206_14735_gb300 as gs
    R = min(R, w.rays)
    if sampler == "plain":
        b = gs.Batch.allocate(R, w.n_strat + w.n_guided, 0)
        ctx.sample_rays(dfr, seed, 0, b)
    elif sampler == "importance":
        b = gs.Batch.allocate(R, w.n_samples, 0)
        ctx.sample_importance(dfr, theta, seed, 0, b)
    else:
        b = gs.Batch.allocate(R, w.prop_samples, 0)
        ctx.proposal_sample(dfr, seed, 0, b, theta=theta, prop=q)
    loss = torch.empty(6, device="cuda")
    dh = torch.empty(R, device="cuda")
    ctx.forward(theta, b, loss, d_hat=dh, theta_bf16=mirror)
    d_hat = dh.cpu().numpy().astype(np.float64)
    pix = b.pix.cpu().numpy()
    D = b.depth.cpu().numpy()
    g = gt.reshape(-1)[pix].astype(np.float64)
    ok = g > 0
    drop = ok & (D <= 0)
    return {"depth_l1_gt_m": round(float(np.abs(d_hat - g)[ok].mean()), 5),
            "depth_l1_gt_dropped_m": round(float(np.abs(d_hat - g)[drop].mean()), 5) if drop.any() else None,
            "rays": int(R), "dropped_rays": int(drop.sum())}


def sampler_report(w, fr, dfr, steps):
    """Trains the workload's plain form (stratified + depth-guided samples) and the paper's
    hierarchical importance form from the same initial parameters for `steps` steps each;
    reports the host wall clock per step and the rendered-depth error against the noise-free
    depth on fresh rays, each model with its own sampler and both with the plain one."""
    import torch

    import paper_2206_14735_gb300 as gs
    import scenegen as sg
    out = {}
    for form in ("plain", "importance"):
        wf = w if form == "importance" else w.with_(imp_coarse=0, imp_steps=0, imp_per_step=0)
        ctx = gs.Context(wf, store_activations=True)
        theta = torch.from_numpy(sg.init_params(wf)).cuda()
        grad, m, v = torch.zeros_like(theta), torch.zeros_like(theta), torch.zeros_like(theta)
        loss = torch.empty(6, device="cuda")
        batch = gs.Batch.allocate(wf.rays, wf.n_samples, wf.n_smooth)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            if form == "importance":
                ctx.sample_importance(dfr, theta, 5, k, batch)
            else:
                ctx.sample_rays(dfr, 5, k, batch)
            ctx.forward_backward(theta, batch, None, loss, grad)
            ctx.adam_step(theta, grad, m, v, k + 1, wf.lr_grid, wf.lr_mlp, wf.betas[0], wf.betas[1], wf.adam_eps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ctx.sync_status()
        res = {"steps": steps, "ms_per_step": round(1e3 * dt / steps, 3), "rays_per_s": round(wf.rays * steps / dt, 1),
               "samples_per_ray": wf.n_samples, "with_own_sampler": _eval_depth(ctx, wf, dfr, fr.gt_depth, theta, form)}
        if form == "importance":
            res["with_plain_sampler"] = _eval_depth(ctx, wf, dfr, fr.gt_depth, theta, "plain")
        out[form] = res
        ctx.close()
    out["what"] = ("both forms trained from the same initial parameters on the same frames; depth error of the "
                   "rendered depth against the noise-free depth on fresh rays (host wall clock per step)")
    return out


def mesh_report(w, ctx, step_m, reps=3):
    """Mesh extraction of the workload's scene (its exact SDF baked into the finest level) on a
    lattice of step_m metres over the whole grid box: lattice points, triangles, CUDA-event
    time of gs_extract_mesh (lattice SDF + isosurface), after one untimed call."""
    import torch

    import scenegen as sg
    scene = sg.room_scene() if w.scene == "room" else sg.cube_scene()
    th = torch.from_numpy(sg.sdf_params(w, scene, seed=31)).cuda()
    lo = [a + 0.5 * step_m for a in w.extent_min]
    dims = [int((b - a) / step_m) for a, b in zip(w.extent_min, w.extent_max)]
    phi = torch.empty((dims[2], dims[1], dims[0]), device="cuda")
    _, n = ctx.extract_mesh(th, lo, step_m, dims, phi=phi)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, n = ctx.extract_mesh(th, lo, step_m, dims, max_tris=n, phi=phi)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = sorted(times)[len(times) // 2]
    pts = dims[0] * dims[1] * dims[2]
    return {"step_m": step_m, "lattice": dims, "points": pts, "triangles": n, "ms": round(ms, 3),
            "points_per_s": round(pts / (ms / 1e3), 1),
            "what": "gs_extract_mesh on the scene's SDF baked into the finest level; the count comes back to the host "
                    "inside the timed call"}


def proposal_report(w, fr, dfr, steps, tail=0):
    """Trains the plain form (n_strat + n_guided samples) and the learned-proposal form
    (prop_samples, plain as the fallback) from the same initial parameters for `steps`
    steps; reports rays/s of each and the final rendered-depth error against the
    noise-free depth (overall and on rays whose observed depth was dropped).  With tail > 0
    also the rays/s of the last `tail` steps alone (the trained regime)."""
    import numpy as np
    import torch

    import paper_2206_14735_gb300 as gs
    import scenegen as sg
    from paper_2206_14735_gb300.proposal import ProposalTrainer
    out = {}
    for form in ("plain", "proposal"):
        # the plain form is always the FP32 one; the proposal form takes the workload's precision
        wf = w.with_(precision="fp32") if form == "plain" else w
        ctx = gs.Context(wf, store_activations=True)
        theta = torch.from_numpy(sg.init_params(w)).cuda()
        grad, m, v = torch.zeros_like(theta), torch.zeros_like(theta), torch.zeros_like(theta)
        mirror = theta[:w.layout()[1]].to(torch.bfloat16).view(torch.int16).contiguous() if ctx.bf16 else None
        loss = torch.empty(6, device="cuda")
        trainer = ProposalTrainer(ctx, w, dfr, seed=5, mirror=mirror) if form == "proposal" else None
        batch = gs.Batch.allocate(w.rays, w.n_samples, w.n_smooth) if form == "plain" else None
        n_prop = n_prop_tail = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t_tail = None
        for k in range(steps):
            if tail > 0 and k == steps - tail:
                torch.cuda.synchronize()
                t_tail = time.perf_counter()
            if trainer is None:
                ctx.sample_rays(dfr, 5, k, batch)
                ctx.forward_backward(theta, batch, None, loss, grad)
                ctx.adam_step(theta, grad, m, v, k + 1, w.lr_grid, w.lr_mlp, w.betas[0], w.betas[1], w.adam_eps)
            else:
                on = int(trainer.controller.use_proposal)
                n_prop += on
                n_prop_tail += on if t_tail is not None else 0
                trainer.step(k, theta, grad, m, v, loss)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        dt = t1 - t0
        ctx.sync_status()
        res = {"steps": steps, "ms_per_step": round(1e3 * dt / steps, 3), "rays_per_s": round(w.rays * steps / dt, 1)}
        if t_tail is not None:
            res["tail_steps"] = tail
            res["tail_rays_per_s"] = round(w.rays * tail / (t1 - t_tail), 1)
            if trainer is not None:
                res["tail_steps_on_proposal"] = n_prop_tail
        if trainer is None:
            res.update(_eval_depth(ctx, w, dfr, fr.gt_depth, theta, "plain"))
            res["samples_per_ray"] = w.n_samples
        else:
            res["proposal_steps"] = n_prop
            hist = trainer.controller.history
            res["controller_trace"] = [[round(a, 4), round(b, 4), c] for a, b, c in hist[::max(1, len(hist) // 12)]]
            res["ce_last"] = round(float(trainer.ce[0].item()), 5)
            res["with_proposal"] = _eval_depth(ctx, w, dfr, fr.gt_depth, theta, "proposal", q=trainer.q,
                                               mirror=mirror)
            res["with_plain"] = _eval_depth(ctx, w, dfr, fr.gt_depth, theta, "plain", mirror=mirror)
            res["samples_per_ray"] = w.prop_samples
            res["precision"] = w.precision
        out[form] = res
        ctx.close()
    out["what"] = ("both forms trained from the same initial parameters on the same frames; depth error of the "
                   "rendered depth against the noise-free depth on 65536 fresh rays; rays_per_s includes the "
                   "proposal's training step and its held-out fallback checks (host wall clock)")
    return out


def run_proposal(args):
    """The learned-proposal form as the timed step: sampler (proposal, or the plain
    fallback), fused forward/backward, proposal training, Adam on both, periodic fallback
    check."""
    import torch

    import paper_2206_14735_gb300 as gs
    import scenegen as sg
    from paper_2206_14735_gb300 import build as gbuild
    from paper_2206_14735_gb300.proposal import ProposalTrainer

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    gbuild.build()
    w = sg.WORKLOADS[args.workload]
    if args.prop_guided is not None:
        w = w.with_(prop_guided=args.prop_guided)
    if args.lr_prop is not None:
        w = w.with_(lr_prop=args.lr_prop)
    fr = sg.make_frames(w, n_frames=args.frames, with_gt=args.prop_report > 0)
    dfr = gs.DeviceFrames(fr.rgb, fr.depth, fr.c2w, fr.fx, fr.fy, fr.cx, fr.cy)
    ctx = gs.Context(w, store_activations=not args.recompute)
    theta = torch.from_numpy(sg.init_params(w)).cuda()
    grad, m, v = torch.zeros_like(theta), torch.zeros_like(theta), torch.zeros_like(theta)
    mirror = theta[:w.layout()[1]].to(torch.bfloat16).view(torch.int16).contiguous() if ctx.bf16 else None
    loss = torch.empty(6, device="cuda")
    trainer = ProposalTrainer(ctx, w, dfr, seed=3 + 1000 * rank, mirror=mirror)
    for k in range(args.warmup + args.prop_pretrain):
        trainer.step(k, theta, grad, m, v, loss)
    torch.cuda.synchronize()
    ctx.sync_status()
    stream = torch.cuda.current_stream()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    base = args.warmup + args.prop_pretrain
    n_prop = 0
    start.record(stream)
    for k in range(args.steps):
        n_prop += int(trainer.controller.use_proposal)
        trainer.step(base + k, theta, grad, m, v, loss)
    stop.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = start.elapsed_time(stop)
    ctx.sync_status()
    ms = max_over_ranks([ms], world)[0]
    if rank != 0:
        return None
    value = aggregate_rays_per_s(w.rays, args.steps, world, ms)
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "rays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if ctx.bf16 else "f32", "data": "synthetic",
        "config": step_config(w, args, world, fr.depth.shape[0]),
        "proposal": {"timed_steps_on_proposal": n_prop, "controller_last": trainer.controller.history[-3:],
                     "ce_last": round(float(trainer.ce[0].item()), 5)},
        "clocks": clk,
        "loss_last": [round(x, 6) for x in loss.cpu().numpy().tolist()],
    }
    if args.prop_report > 0:
        line["proposal_report"] = proposal_report(w, fr, dfr, args.prop_report)
    return line


def differentiation_report(w, dfr, theta, mirror, reps=20):
    """Forward + backward of one sampled batch with the decoder activations recomputed in the
    backward pass versus stored by the forward pass: device time per call (CUDA events) for
    the split calls (gs_forward then gs_backward, as the autograd Function runs them) and the
    fused call, and the memory the store takes."""
    import torch

    import paper_2206_14735_gb300 as gs
    out = {}
    stream = torch.cuda.current_stream()
    for name, store in (("recompute", False), ("store", True)):
        c = gs.Context(w, store_activations=store)
        b = gs.Batch.allocate(w.rays, w.n_samples, w.n_smooth)
        c.sample_rays(dfr, 11, 0, b)
        loss = torch.empty(6, device="cuda")
        grad = torch.zeros_like(theta)
        ms = {"forward": 0.0, "backward": 0.0, "fused": 0.0}
        for it in range(reps + 3):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            c.forward(theta, b, loss, theta_bf16=mirror)
            ev[1].record(stream)
            c.backward(theta, b, None, grad, theta_bf16=mirror)
            ev[2].record(stream)
            c.forward_backward(theta, b, None, loss, grad, theta_bf16=mirror)
            ev[3].record(stream)
            torch.cuda.synchronize()
            if it >= 3:
                ms["forward"] += ev[0].elapsed_time(ev[1]) / reps
                ms["backward"] += ev[1].elapsed_time(ev[2]) / reps
                ms["fused"] += ev[2].elapsed_time(ev[3]) / reps
        c.sync_status()
        extra = w.rays * w.n_samples * 99 * 4 if store else 0
        out[name] = {"forward_ms": round(ms["forward"], 4), "backward_ms": round(ms["backward"], 4),
                     "split_ms": round(ms["forward"] + ms["backward"], 4), "fused_ms": round(ms["fused"], 4),
                     "extra_device_bytes": extra}
        c.close()
    out["what"] = (f"{w.rays} rays x {w.n_samples} samples + {w.n_smooth} smoothness points; "
                   f"store keeps 100 floats per sample (z, both ReLU layers, SDF and geometric feature, colour, one pad); "
                   f"mean of {reps} calls each")
    return out


def _profiled_traffic(profile: str, sources) -> float | None:
    """DRAM bytes per launch recorded by an ncu capture under profiles/, or None when the
    kernel's sources no longer hash as they did when it was captured."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        want = re.search(r"kernel_sources_sha256: ([0-9a-f]{64})", text).group(1)
        traffic = float(re.search(r"traffic_bytes_per_launch: (\d+)", text).group(1))
    except (OSError, AttributeError):
        return None
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2206_14735_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return traffic if h.hexdigest() == want else None


def _oracle_steps(w, fr, R, P, n_steps, time_cap_s=None, k0=0):
    """Run n_steps full oracle steps (sample R rays and P smoothness points, FP64 forward and
    backward, FP64 Adam over every parameter) and return their durations.  With time_cap_s,
    stop early once that much time has passed (at least one step runs)."""
    import numpy as np

    import oracle as oc
    import scenegen as sg

    cfg = oc.make_config(w)
    ofr = oc.OcFramesHolder(fr)
    theta = sg.init_params(w).astype(np.float64)
    n = w.layout()[2]
    mom, vel = np.zeros(n), np.zeros(n)
    times = []
    t_all = time.perf_counter()
    for k in range(k0, k0 + n_steps):
        t0 = time.perf_counter()
        if w.imp_coarse > 0:
            bt = oc.sample_importance(cfg, ofr, theta, 3, k, R, w.imp_coarse, w.imp_steps, w.imp_per_step)
        else:
            bt = oc.sample_rays(cfg, ofr, 3, k, R)
        sm = oc.sample_smooth(cfg, ofr, 3, k, P)
        out = oc.step(cfg, theta, bt, sm)
        g = np.ascontiguousarray(out["grad"])
        oc.adam(theta, g, mom, vel, w.layout()[1], k + 1, w.lr_grid, w.lr_mlp)
        times.append(time.perf_counter() - t0)
        if time_cap_s is not None and time.perf_counter() - t_all > time_cap_s:
            break
    return times, oc.num_threads()


def cpu_baseline(w, fr, R):
    P = max(1, w.n_smooth * R // w.rays)
    times, cores = _oracle_steps(w, fr, R, P, 3, time_cap_s=10.0)
    t = statistics.median(times)
    return {"value": round(R / t, 2), "unit": "rays/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(times)} oracle step(s) of {R} rays x {w.n_samples} samples + "
                      f"{P} smoothness points + FP64 Adam over all "
                      f"{w.layout()[2]} parameters; value = rays / median step time"}


def run_reference(args):
    """The oracle as the reference arm: W untimed then exactly K timed full steps of the same
    workload (every ray, smoothness point and parameter of the GPU arm's step), on the host
    cores.  Rank 0 only; other ranks exit without work."""
    rank, world, local = dist_env()
    if rank != 0:
        return None
    import scenegen as sg
    w = sg.WORKLOADS[args.workload]
    if w.prop_samples > 0 or w.arch == "paper":
        return {"impl": "reference", "unavailable": "the oracle arm covers the plain compact-architecture workloads"}
    fr = sg.make_frames(w, n_frames=args.frames)
    _oracle_steps(w, fr, w.rays, w.n_smooth, args.warmup)
    t0 = time.perf_counter()
    times, cores = _oracle_steps(w, fr, w.rays, w.n_smooth, args.steps, k0=args.warmup)
    total = time.perf_counter() - t0
    assert len(times) == args.steps
    value = w.rays * args.steps / total
    sample = (f"every step in full: {w.rays} rays x {w.n_samples} samples, {w.n_smooth} smoothness points, "
              f"FP64 forward + backward and FP64 Adam over all {w.layout()[2]} parameters; "
              f"{args.warmup} untimed + {args.steps} timed steps")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": step_config(w, args, world, fr.depth.shape[0]),
            "cpu_baseline": {"value": round(value, 2), "unit": "rays/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 2), "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--frames", type=int, default=None, help="render only the first F poses (default: all)")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-rays", type=int, default=8192)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic-render", type=float, default=None)
    ap.add_argument("--traffic-adam", type=float, default=None)
    ap.add_argument("--diff-report", action="store_true",
                    help="also time forward/backward with stored versus recomputed decoder activations")
    ap.add_argument("--recompute", action="store_true",
                    help="recompute the decoder activations in the backward pass instead of storing them")
    ap.add_argument("--split", action="store_true", help="gs_forward then gs_backward instead of the fused call")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="sample each step's batch in line instead of during the previous step")
    ap.add_argument("--poses", action="store_true",
                    help="refine the camera poses in every step (gs_pose_apply, gs_pose_backward, Adam at 5e-4)")
    ap.add_argument("--eikonal", action="store_true",
                    help="add the Eikonal term on the free-space samples (gs_eikonal, lam_eik = 1) to every step")
    ap.add_argument("--prop-pretrain", type=int, default=300,
                    help="proposal workloads: untimed steps before the timed region (controller settles)")
    ap.add_argument("--prop-guided", type=int, default=None, help="proposal workloads: override prop_guided")
    ap.add_argument("--lr-prop", type=float, default=None, help="proposal workloads: override the proposal's lr")
    ap.add_argument("--prop-report", type=int, default=0,
                    help="proposal workloads: train plain and proposal forms this many steps and compare depth")
    ap.add_argument("--target-steps", type=int, default=8000,
                    help="default workload: also train the plain FP32 and the BF16 + proposal forms this many "
                         "steps each at 65536 rays and report the pair (0: skip)")
    ap.add_argument("--mesh-report", type=float, default=0.0,
                    help="also time mesh extraction of the scene at this lattice step (metres; the paper uses 0.01)")
    ap.add_argument("--sampler-report", type=int, default=0,
                    help="importance workloads: train the plain and the importance form this many steps and compare "
                         "depth")
    args = ap.parse_args()
    if args.impl == "reference":
        line = run_reference(args)
    else:
        import scenegen as sg
        line = run_proposal(args) if sg.WORKLOADS[args.workload].prop_samples > 0 else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
