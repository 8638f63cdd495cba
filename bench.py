"""Benchmark: fwd+bwd mapping iterations/s at 300k Gaussians, 1200 x 680.

One step = one whole photorealistic-mapping iteration of Photo-SLAM
(arXiv 2311.16728, Sec. 3.3): EWA preprocess, tile binning + radix sort,
forward blend (Eq. 3), L1 + D-SSIM loss and its gradient (Eq. 4, lambda 0.2),
backward blend + chain rule, fused Adam, on one view of a 50-pose trajectory.
Inputs are seeded synthetic scenes shaped like the paper's Replica frames (the
dataset itself is not available).  The path does not shard: with --gpus N
every rank runs an independent replica (weak scaling, no collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--mode mapping|window|mlp|ttp|densify|stereo|gp_ablation|pose]

--impl reference times the FP64 CPU oracle (the only other implementation of
this path) on the host cores, on a bounded band of image rows per step.
--mode window times the batched Gaussian-pyramid window (500k Gaussians,
8 keyframes of 640 x 480 x 3 levels, one persistent launch per iteration,
whole iteration in one CUDA graph); --mode mlp times the learned
initialiser's tensor-core forward and training step at 2k and 20k rows;
--mode ttp runs the time-to-PSNR experiment (plain single-view path with
default initialisation against the batched window with the learned
initialiser, and with the default one); --mode densify runs mapping on a
1M-Gaussian 1920 x 1080 scene with densification and pruning every 100
iterations (uneven Gaussian counts); --mode stereo maps 752 x 480 grayscale
stereo pairs (0.11 m baseline, luminance loss); --mode gp_ablation compares
the final PSNR of the plain path with 1 to 4 pyramid levels (Sec. 4.4,
Tab. 4); --mode pose times the camera pose gradient pass and a photometric
pose refinement.  The default (mapping) line is the headline.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GAUSS = 300_000
WIDTH, HEIGHT, FOCAL = 1200, 680, 600.0
N_POSES = 50
METRIC = "fwd+bwd iters/s @300k Gaussians 1200x680"
WORKLOAD = ("single-view mapping step (Replica-shaped): 300k Gaussians in a 6x3x4 m room, 1200x680, fx=fy=600, "
            "50-pose seeded trajectory, 16x16 tiles, L1+D-SSIM (lambda 0.2), Adam, FP32")


def _config(extra=None):
    c = {"workload": WORKLOAD, "gaussians": N_GAUSS, "width": WIDTH, "height": HEIGHT, "tile": "16x16",
         "poses": N_POSES, "sh_degree": 3,
         "l2": "inputs larger than L2: params + grads + Adam moments (4 x 72 MB) stream through HBM every step",
         "parallelism": "replicas (no data-path collective)"}
    if extra:
        c.update(extra)
    return c


WORKLOAD_WALLS = WORKLOAD.replace("300k Gaussians in a 6x3x4 m room",
                                  "300k Gaussians on the six walls of a 6x3x4 m room (surface-like; sensitivity variant)")


def _scene(poses: int = N_POSES, kind: str = "room"):
    import synthetic as S
    target = S.room_scene(N_GAUSS, seed=0) if kind == "room" else S.wall_scene(N_GAUSS, seed=0)
    start = S.perturb(target, 0.05, seed=1)
    cams = [S.replica_camera(k) for k in range(poses)]
    return target, start, cams


def _ordered(gsr, params, args):
    """The map store in the order --order names (setup, untimed): Morton
    order of the means over the room box, or the generator's order."""
    if args.order == "input":
        return params
    import synthetic as S
    return gsr.permuted(params, gsr.spatial_order(params, S.ROOM_LO, S.ROOM_HI))


def max_over_ranks(x: float, device) -> float:
    """The slowest rank's value of a per-rank time (replicas: the job ends
    when the last replica does); x itself without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ms_per_step: float, world: int) -> float:
    """Whole-job iterations/s of `world` replicas that each ran one iteration
    per ms_per_step (the max over ranks)."""
    return world * 1000.0 / ms_per_step


# ---------------------------------------------------------------- CPU oracle sample
def oracle_sample(start, target_imgs_rows, cams, pose: int, rows: int, row0: int):
    """Time the oracle over one iteration restricted to `rows` image rows and
    extrapolate to the full frame.  Returns (seconds per full iteration, detail)."""
    import oracle
    cam = cams[pose]
    ca = cam.as_array()
    band = (row0, row0 + rows)
    t0 = time.perf_counter()
    dec = oracle.decide(start.mean_op, start.quat, start.logscale, ca, cam.width, cam.height)
    sc = oracle.Scene64(start.mean_op, start.quat, start.logscale, start.sh)
    t1 = time.perf_counter()
    oracle.render(sc, ca, cam.width, cam.height, dec, rows=(0, 0))  # per-call fixed cost (projection, depth sort)
    t2 = time.perf_counter()
    img, _, _, _ = oracle.render(sc, ca, cam.width, cam.height, dec, rows=band)
    t3 = time.perf_counter()
    L, d = oracle.loss(img[:, band[0]:band[1]], target_imgs_rows, 0.2)
    t4 = time.perf_counter()
    dimg = np.zeros((3, cam.height, cam.width))
    dimg[:, band[0]:band[1]] = d
    oracle.render_bwd(sc, ca, cam.width, cam.height, dec, np.zeros_like(dimg), rows=(0, 0))
    t5 = time.perf_counter()
    g, _ = oracle.render_bwd(sc, ca, cam.width, cam.height, dec, dimg, rows=band)
    t6 = time.perf_counter()
    n = start.n
    lr = np.full((n, 60), 1e-3)
    p = np.zeros((n, 60))
    oracle.adam(p, g, np.zeros_like(p), np.zeros_like(p), lr, 1)
    t7 = time.perf_counter()
    # the band calls repeat their per-call fixed part (projection, depth
    # sort): only the remainder scales with the number of rows
    fixed = (t1 - t0) + (t2 - t1) + (t5 - t4) + (t7 - t6)
    per_band = max(0.0, (t3 - t2) - (t2 - t1)) + (t4 - t3) + max(0.0, (t6 - t5) - (t5 - t4))
    full = fixed + per_band * (cam.height / rows)
    return full, {"measured_s": t7 - t0, "fixed_s": fixed, "band_s": per_band}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synthetic as S
    target, start, cams = _scene()
    rows = args.ref_rows
    # target band: the oracle renders the unperturbed set on the same rows
    per_step = []
    detail = None
    tgt_cache = {}
    # bounded: at most 3 timed steps after 1 warm-up (a full-frame oracle
    # step takes seconds), each on a band of `rows` rows extrapolated to the
    # frame; the mean of the timed steps is the per-step time
    n_warm, n_timed = min(args.warmup, 1), max(1, min(args.steps, 3))
    for k in range(n_warm + n_timed):
        pose = k % N_POSES
        row0 = (97 * k) % (HEIGHT - rows)
        key = (pose, row0)
        if key not in tgt_cache:
            cam = cams[pose]
            dt = oracle.decide(target.mean_op, target.quat, target.logscale, cam.as_array(), WIDTH, HEIGHT)
            st = oracle.Scene64(target.mean_op, target.quat, target.logscale, target.sh)
            im, _, _, _ = oracle.render(st, cam.as_array(), WIDTH, HEIGHT, dt, rows=(row0, row0 + rows))
            tgt_cache = {key: im[:, row0:row0 + rows].copy()}
        full, detail = oracle_sample(start, tgt_cache[key], cams, pose, rows, row0)
        if k >= n_warm:
            per_step.append(full)
    sec = statistics.mean(per_step)
    cores = oracle.num_threads()
    sample = (f"oracle (FP64, OpenMP), {n_timed} timed step(s) after {n_warm} warm-up: decide+Adam over all "
              f"{N_GAUSS} Gaussians, render+loss+backward on a {rows}-row band of the 1200x680 frame, extrapolated "
              f"to the full frame")
    line = {"impl": "reference", "metric": METRIC, "value": 1.0 / sec, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _config(),
            "cpu_baseline": {"value": 1.0 / sec, "unit": "iters/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": 1.0 / sec, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
class ClockSampler:
    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms",
                                       "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self, gpu_index: int):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != gpu_index:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def count_kernel_nodes(graphs) -> int:
    """Kernel nodes in the captured graphs of one iteration."""
    from cuda.bindings import runtime as rt
    total = 0
    for g in graphs:
        raw = rt.cudaGraph_t(init_value=g.raw_cuda_graph())
        err, _, num = rt.cudaGraphGetNodes(raw, 0)
        err, nodes, num = rt.cudaGraphGetNodes(raw, num)
        for nd in nodes[:num]:
            err, ty = rt.cudaGraphNodeGetType(nd)
            if ty == rt.cudaGraphNodeType.cudaGraphNodeTypeKernel:
                total += 1
    return total


# ---------------------------------------------------------------- batched window (pattern 2)
WIN_N = 500_000
WIN_KF = 8
WIN_LEVELS = 3


def _profile_steps(step, k):
    import torch
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for _ in range(k):
        step()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profiled_steps": k}), flush=True)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def run_window(args):
    import torch
    import synthetic as S
    import paper_2311_16728_b300 as gsr
    from paper_2311_16728_b300.autotune import autotune_window
    from paper_2311_16728_b300.batched import BatchedWindow
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    target = S.room_scene(WIN_N, seed=0)
    start = S.perturb(target, 0.05, seed=1)
    cams = [S.tum_camera(k * N_POSES // WIN_KF) for k in range(WIN_KF)]
    g_tgt = gsr.Gaussians.from_arrays(target.mean_op, target.quat, target.logscale, target.sh)
    vb = gsr.ViewBuffers(WIN_N, gsr.camera_from(cams[0]), gsr.tiling_struct(16, 16), 1024)
    kf = []
    for cam in cams:
        vb.cam = gsr.camera_from(cam)
        gsr.ensure_capacity(vb, g_tgt)
        vb.forward(g_tgt)
        kf.append((cam, vb.img.clone()))
    del vb, g_tgt
    params = _ordered(gsr, gsr.Gaussians.from_arrays(start.mean_op, start.quat, start.logscale, start.sh), args)
    if args.tile == "auto":
        tile, report = autotune_window(params, kf, levels=WIN_LEVELS, steps=5, warmup=2)
    else:
        tile = tuple(int(x) for x in args.tile.split("x"))
        report = {"ms_per_step": {}}
    bw = BatchedWindow(params, kf, levels=WIN_LEVELS, tiling=gsr.tiling_struct(*tile))
    bw.capture()
    for _ in range(args.warmup):
        bw.step()
    torch.cuda.synchronize()
    if args.profile:
        _profile_steps(bw.step, args.steps)
        return
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler()
    clocks.start()
    torch.cuda.synchronize()
    t0.record()
    for _ in range(args.steps):
        bw.step()
    t1.record()
    torch.cuda.synchronize()
    clk = clocks.stop(int(os.environ.get("LOCAL_RANK", "0")))
    if bw.status.item() != 0:
        raise RuntimeError(f"device status {bw.status.item():#x} during the timed region")
    ms_per_step = t0.elapsed_time(t1) / args.steps
    launches_per_iter = count_kernel_nodes([bw.graph])
    # end to end: every view's target image from pinned host memory in, the
    # per-view losses out, every step.  Two target sets and two graphs: step
    # k reads set k % 2 while set (k + 1) % 2 is refilled for the next step on
    # a second stream (it waits for step k - 1, the last reader of that set);
    # every copy lies inside the timed region.
    host_gts = [g.cpu().pin_memory() for g in bw.gts]
    host_loss = torch.empty(bw.V, dtype=torch.float32).pin_memory()
    sets = [bw.gts, [torch.empty_like(g) for g in bw.gts]]
    graph_a = bw.graph
    bw.set_targets(sets[1])
    bw.capture()
    graphs = [graph_a, bw.graph]
    main, copy = torch.cuda.current_stream(), torch.cuda.Stream()
    ready = [torch.cuda.Event() for _ in range(args.steps)]
    done = [torch.cuda.Event() for _ in range(args.steps)]

    def fetch(k):
        with torch.cuda.stream(copy):
            for d, h in zip(sets[k % 2], host_gts):
                d.copy_(h, non_blocking=True)
        ready[k].record(copy)

    torch.cuda.synchronize()
    t0.record()
    copy.wait_stream(main)
    fetch(0)
    for k in range(args.steps):
        main.wait_event(ready[k])
        if k + 1 < args.steps:
            if k >= 1:
                copy.wait_event(done[k - 1])
            fetch(k + 1)
        graphs[k % 2].replay()
        done[k].record(main)
        host_loss.copy_(bw.losses, non_blocking=True)
    t1.record()
    torch.cuda.synchronize()
    e2e_ms = t0.elapsed_time(t1) / args.steps
    bw.set_targets(sets[0])
    h2d = sum(g.numel() * 4 for g in bw.gts)
    # stage breakdown: the same iteration captured one graph per stage
    bw.capture(per_stage=True)
    nst = len(bw.STAGES)
    ksteps = min(args.steps, 200)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nst + 1)] for _ in range(ksteps)]
    for k in range(ksteps):
        bw.step(events=evs[k])
    torch.cuda.synchronize()
    stage_ms = {nm: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs) for i, nm in enumerate(bw.STAGES)}
    phases = bw.phase_ms()
    phases["bwd_blend"] = stage_ms["iterate"] - phases.pop("entry_to_bwd")
    # work counters (outside the timed region): blends of every view at the final parameters
    # and the same views through the one-view kernels, timed one by one
    blends = 0
    single = {"render_fwd": 0.0, "loss": 0.0, "blend_bwd": 0.0}
    per_level = {}
    for cam_v, gt_v, lvl, _ in bw.views:
        vbv = gsr.ViewBuffers(WIN_N, cam_v, bw.tiling, 1024)
        gsr.ensure_capacity(vbv, params)
        nblend = torch.zeros(cam_v.height, cam_v.width, dtype=torch.int32, device="cuda")
        vbv.preprocess(params)
        vbv.bin_sort()
        vbv.render_fwd(n_blended=nblend)
        nb = int(nblend.sum().item())
        blends += nb
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        vbv.render_fwd()
        ev[1].record()
        vbv.loss_fwd_bwd(gt_v, 0.2)
        ev[2].record()
        vbv.blend_bwd()
        ev[3].record()
        torch.cuda.synchronize()
        for j, nm in enumerate(("render_fwd", "loss", "blend_bwd")):
            single[nm] += ev[j].elapsed_time(ev[j + 1])
        pl = per_level.setdefault(str(lvl), {"views": 0, "blends": 0, "pairs": 0, "render_fwd_ms": 0.0,
                                             "blend_bwd_ms": 0.0})
        pl["views"] += 1
        pl["blends"] += nb
        pl["pairs"] += int(vbv.num_pairs.item())
        pl["render_fwd_ms"] += ev[0].elapsed_time(ev[1])
        pl["blend_bwd_ms"] += ev[2].elapsed_time(ev[3])
        del vbv
    peaks = _peaks()
    mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    fp32 = 148 * 128 * 2 * mhz * 1e6 / 1e12
    flops = (FLOPS_PER_BLEND_FWD + FLOPS_PER_BLEND_BWD) * blends
    it_s = stage_ms["iterate"] * 1e-3
    px = sum(c.width * c.height for c, _, _, _ in bw.views)
    line = {"metric": f"window iters/s @{WIN_N // 1000}k Gaussians, {WIN_KF} keyframes 640x480 x {WIN_LEVELS} levels",
            "value": 1000.0 / ms_per_step, "unit": "iters/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; TUM-shaped keyframes)",
            "views_per_s": bw.V * 1000.0 / ms_per_step,
            "config": {"workload": f"batched Gaussian-pyramid window: {WIN_N} Gaussians in a 6x3x4 m room, "
                                   f"{WIN_KF} keyframes 640x480 fx=fy=525 x {WIN_LEVELS} levels = {bw.V} views, "
                                   f"{bw.tiles} tiles, {px} px; one persistent launch per iteration; whole "
                                   "iteration (preprocess, binning, persistent fwd/loss/bwd, chain, Adam) in one "
                                   "CUDA graph", "tile": f"{tile[0]}x{tile[1]}" + (" (autotuned)" if args.tile == "auto" else " (given)"),
                       "autotune_ms": report["ms_per_step"], "pairs": int(bw.num_pairs.item()),
                       "map_order": args.order,
                       "l2": "inputs larger than L2 (4 x 120 MB of params, grads, moments per step)"},
            "roofline": {"kernel": "batched_iterate_kernel (fwd + bwd blends)", "bound": "alu",
                         "achieved": flops / it_s / 1e12, "peak": fp32, "unit": "TFLOP/s",
                         "frac": flops / it_s / 1e12 / fp32,
                         "traffic": NCU_TRAFFIC_WINDOW_ITERATE if (tile == (16, 16) and args.order == "morton") else None,
                         "alg_per_launch": flops,
                         "peak_source": f"FP32 148 SMs x 128 lanes x 2 x {mhz:.0f} MHz (sampled median clock)"},
            "stages_ms": stage_ms, "iterate_phases_ms": phases,
            "one_view_kernels_ms": single, "per_level": per_level, "work": {"blends": blends, "views": bw.V},
            "gpu_launches": launches_per_iter * args.steps, "clocks": clk,
            "e2e": {"value": 1000.0 / e2e_ms, "unit": "iters/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 4 * bw.V}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- learned initialiser (cfg5)
def run_mlp(args):
    import torch
    from paper_2311_16728_b300.learned_init import LearnedInit, init_weights, pad_rows, K_IN, H, N_OUT, N3
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    peaks = _peaks()
    out = []
    for M in ((20000,) if args.profile else (2048, 20000)):
        li = LearnedInit(init_weights(3), M, lr=1e-4)
        gen = torch.Generator(device="cuda").manual_seed(5)
        li.x[:M, :K_IN] = torch.rand(M, K_IN, device="cuda", generator=gen).to(torch.bfloat16)
        li.xT.copy_(li.x.t())
        tgt = torch.zeros(li.mpad, N3, device="cuda")
        tgt[:M, :N_OUT] = torch.randn(M, N_OUT, device="cuda", generator=gen)
        fwd_flop = 2.0 * M * (K_IN * H + H * H + H * N_OUT)
        res = {"rows": M, "padded_rows": li.mpad}
        for name, fn, flop in (("forward", lambda: li.forward(), fwd_flop),
                               ("train_step", lambda: li.train_step(tgt, M), 3 * fwd_flop)):
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                fn()
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                fn()
            for _ in range(max(args.warmup, 3)):
                g.replay()
            if args.profile and name == "train_step":
                _profile_steps(g.replay, args.steps)
                return
            reps = 200
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                g.replay()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            res[name] = {"ms": ms, "tflops": flop / ms / 1e9,
                         "frac_of_bf16_burst": flop / ms / 1e9 / peaks.get("bf16_tflops", 1800.0)}
        if li.status.item() != 0:
            raise RuntimeError(f"MLP device status {li.status.item():#x}")
        out.append(res)
    big = out[-1]["train_step"]
    line = {"metric": "learned-initialiser training step TFLOP/s @20k rows (2308-256-256-56, BF16 x BF16 -> FP32)",
            "value": big["tflops"], "unit": "TFLOP/s", "n_gpus": 1, "steps": 200, "warmup": max(args.warmup, 3),
            "ms_per_step": big["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic (seeded uniform patches, Gaussian targets)",
            "config": {"workload": "MLP forward / training step (5 tcgen05 GEMMs + fused epilogues + Adam) on "
                                   "2k and 20k rows", "results": out},
            "roofline": {"kernel": "training step (all GEMMs)", "bound": "tensor", "achieved": big["tflops"],
                         "peak": peaks.get("bf16_tflops", 1800.0), "unit": "TFLOP/s",
                         "frac": big["frac_of_bf16_burst"], "traffic": None,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst; of measured)"}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- time to PSNR
TTP_N = 200_000
TTP_KF = 8
TTP_NEW = 20_000         # at most this many new primitives per keyframe (all in-view centres, first keyframe first)
TTP_BUDGET = 3000        # plain-path iterations fixing the target PSNR
TTP_WINDOW_MAX = 1500    # window iterations at most
TTP_TRAIN_SEEDS = (10, 11)
TTP_HARVEST_ITERS = 400  # window iterations of the harvesting run
TTP_MLP_STEPS = 6000


def _ttp_setup(seed, gsr, torch):
    """Scene `seed`, its keyframes (images rendered from the true map) and the
    keypoints of the held-out primitives, with ORB-style angles."""
    import synthetic as S
    cams = [S.tum_camera(k * N_POSES // TTP_KF) for k in range(TTP_KF)]
    truth, offsets, kps = S.densify_scene(S.room_scene(TTP_N, seed=seed), cams, TTP_NEW, seed=seed + 1)
    g = gsr.Gaussians.from_arrays(truth.mean_op, truth.quat, truth.logscale, truth.sh)
    vb = gsr.ViewBuffers(TTP_N, gsr.camera_from(cams[0]), gsr.tiling_struct(16, 16), 1024)
    keyframes = []
    for cam, kp in zip(cams, kps):
        vb.cam = gsr.camera_from(cam)
        gsr.ensure_capacity(vb, g)
        vb.forward(g)
        img = vb.img.clone()
        host = img.cpu().numpy()
        kp[:, 4] = [S.orb_angle(host, u, v) for u, v in kp[:, :2]]
        keyframes.append((cam, img))
    del vb
    return truth, keyframes, [torch.tensor(k, device="cuda") for k in kps], offsets


def _ttp_run(kind, truth, keyframes, kps, offsets, init, li, budget, target, every, gsr, torch):
    """One arm: fresh map = truth with the held-out primitives initialised by
    `init`; iterate until `target` PSNR (if given) or `budget` iterations.
    Returns the PSNR curve [(iterations, training ms, PSNR)]."""
    from paper_2311_16728_b300.batched import BatchedWindow
    from paper_2311_16728_b300.mapping import Evaluator, PlainMapper, densify_default, densify_learned
    params = gsr.Gaussians.from_arrays(truth.mean_op, truth.quat, truth.logscale, truth.sh)
    if init == "learned":
        densify_learned(li, params, keyframes, kps, offsets)
    else:
        densify_default(params, keyframes, kps, offsets)
    ev = Evaluator(TTP_N, keyframes)
    mapper = PlainMapper(params, keyframes) if kind == "plain" else BatchedWindow(params, keyframes)
    mapper.capture()
    curve = [(0, 0.0, ev(params))]
    it, wall = 0, 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    while it < budget and not (target is not None and curve[-1][2] >= target):
        k = min(every, budget - it)
        e0.record()
        for _ in range(k):
            mapper.step()
        e1.record()
        torch.cuda.synchronize()
        it += k
        wall += e0.elapsed_time(e1)
        curve.append((it, wall, ev(params)))
    status = mapper.status() if kind == "plain" else int(mapper.status.item())
    if status != 0:
        raise RuntimeError(f"{kind} arm: device status {status:#x}")
    return curve


def _first_at(curve, target):
    for it, ms, ps in curve:
        if ps >= target:
            return it, ms
    return None, None


def run_ttp(args):
    import torch
    import paper_2311_16728_b300 as gsr
    from paper_2311_16728_b300.batched import BatchedWindow
    from paper_2311_16728_b300.learned_init import LearnedInit, init_weights
    from paper_2311_16728_b300.mapping import densify_default, harvest, train_initialiser
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.time()
    li = LearnedInit(init_weights(3), TTP_NEW, lr=1e-3)  # batches of up to one keyframe's new primitives
    # ---- harvest (patch, converged parameter) pairs from window runs on training scenes
    batches = []
    for seed in TTP_TRAIN_SEEDS:
        truth, keyframes, kps, offsets = _ttp_setup(seed, gsr, torch)
        params = gsr.Gaussians.from_arrays(truth.mean_op, truth.quat, truth.logscale, truth.sh)
        densify_default(params, keyframes, kps, offsets)
        initial = gsr.Gaussians(*(t.clone() for t in params.tensors()), params.sh_degree)
        bw = BatchedWindow(params, keyframes)
        bw.capture()
        for _ in range(TTP_HARVEST_ITERS):
            bw.step()
        torch.cuda.synchronize()
        batches += harvest(li, params, initial, keyframes, kps, offsets)
        del bw, params, initial
    losses = train_initialiser(li, batches, TTP_MLP_STEPS)
    t_train = time.time() - t0
    # ---- held-out scenes: plain + default init fixes the target, then the window arms race to it
    seeds = [int(x) for x in args.ttp_seeds.split(",") if x]
    per_seed = []
    for seed in seeds:
        truth, keyframes, kps, offsets = _ttp_setup(seed, gsr, torch)
        plain = _ttp_run("plain", truth, keyframes, kps, offsets, "default", li, TTP_BUDGET, None, 100, gsr, torch)
        target = plain[-1][2]
        res = {"seed": seed, "target_psnr": target, "plain": {"curve": plain},
               "new": sum(int(k.shape[0]) for k in kps)}
        res["plain"]["iters"], res["plain"]["ms"] = _first_at(plain, target)
        for name, init in (("window_learned", "learned"), ("window_default", "default")):
            c = _ttp_run("window", truth, keyframes, kps, offsets, init, li, TTP_WINDOW_MAX, target, 10, gsr, torch)
            it, ms = _first_at(c, target)
            res[name] = {"curve": c, "iters": it, "ms": ms, "psnr0": c[0][2]}
        res["plain"]["psnr0"] = plain[0][2]
        per_seed.append(res)
    speed = [r["plain"]["ms"] / r["window_learned"]["ms"] for r in per_seed if r["window_learned"]["ms"]]
    speed_def = [r["plain"]["ms"] / r["window_default"]["ms"] for r in per_seed if r["window_default"]["ms"]]
    summary = [{"seed": r["seed"], "new_primitives": r["new"], "target_psnr": r["target_psnr"],
                "plain_ms": r["plain"]["ms"], "plain_iters": r["plain"]["iters"],
                "learned_window_ms": r["window_learned"]["ms"], "learned_window_iters": r["window_learned"]["iters"],
                "default_window_ms": r["window_default"]["ms"], "default_window_iters": r["window_default"]["iters"],
                "psnr0": {"default": r["plain"]["psnr0"], "learned": r["window_learned"]["psnr0"]}}
               for r in per_seed]
    line = {"metric": "time-to-PSNR speed-up, learned initialiser + batched window vs plain single-view path",
            "value": statistics.mean(speed) if speed else None, "unit": "x (plain ms / learned+batched ms)",
            "n_gpus": 1, "higher_is_better": True, "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded; held-out scenes)",
            "config": {"workload": f"{TTP_N} Gaussians in a 6x3x4 m room, {TTP_KF} keyframes 640x480 fx=fy=525, "
                                   "every Gaussian whose centre a keyframe sees (at most "
                                   f"{TTP_NEW} per keyframe) re-created at its keypoint (known depth, unknown shape, "
                                   "opacity and colour); target = PSNR of the plain path (default init, sequential "
                                   f"pyramid, tau_u 30) after {TTP_BUDGET} iterations; wall time = CUDA-event time "
                                   "of the training iterations (evaluation excluded)",
                       "train_seeds": list(TTP_TRAIN_SEEDS), "eval_seeds": seeds,
                       "harvest": f"{TTP_HARVEST_ITERS} window iterations per training scene, "
                                  f"{sum(b.M for b in batches)} pairs", "mlp_steps": TTP_MLP_STEPS,
                       "mlp_loss_first_last": [losses[0], losses[-1]] if losses else None,
                       "setup_s": round(t_train, 1)},
            "speedup_default_window": statistics.mean(speed_def) if speed_def else None,
            "per_seed": summary, "curves": {str(r["seed"]): {k: r[k]["curve"] for k in
                                                            ("plain", "window_learned", "window_default")}
                                           for r in per_seed}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- densify / prune (uneven counts)
DENS_N = 1_000_000
DENS_W, DENS_H, DENS_F = 1920, 1080, 1000.0
DENS_EVERY = 100


def run_densify(args):
    import torch
    import synthetic as S
    import paper_2311_16728_b300 as gsr
    from paper_2311_16728_b300.mapping import Densifier
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    target = S.room_scene(DENS_N, seed=0)
    start = S.perturb(target, 0.05, seed=1)
    cams = []
    for k in range(N_POSES):
        pos, yaw = S.trajectory(k)
        cams.append(S.pose_camera(pos, yaw, DENS_F, DENS_F, DENS_W, DENS_H))
    g_tgt = gsr.Gaussians.from_arrays(target.mean_op, target.quat, target.logscale, target.sh)
    vb = gsr.ViewBuffers(DENS_N, gsr.camera_from(cams[0]), gsr.tiling_struct(16, 16), 1024)
    gts = []
    for cam in cams:
        vb.cam = gsr.camera_from(cam)
        gsr.ensure_capacity(vb, g_tgt)
        vb.forward(g_tgt)
        gts.append(vb.img.clone())
    del vb, g_tgt
    cap = int(DENS_N * 1.25)
    params = gsr.Gaussians.zeros(cap)
    first = _ordered(gsr, gsr.Gaussians.from_arrays(start.mean_op, start.quat, start.logscale, start.sh), args)
    for dst, src in zip(params.tensors()[:3], first.tensors()[:3]):
        dst[:DENS_N] = src
    params.sh[:, :DENS_N] = first.sh
    del first
    adam = gsr.Adam(params)
    dens = Densifier(params, adam, DENS_N)
    views = list(zip(cams, gts))

    def build():
        ms = gsr.MappingStep(dens.params, views, adam=dens.adam, densify_stat=dens.stat,
                             densify_count=dens.count)
        ms.capture()
        return ms

    t_build = time.time()
    ms = build()
    sized_for = DENS_N
    build_s = [time.time() - t_build]
    for _ in range(args.warmup):
        ms.step()
    torch.cuda.synchronize()
    dens.stat.zero_()
    dens.count.zero_()
    segments = max(1, args.steps // DENS_EVERY)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, dens_ms, counts, rebuilds = 0.0, 0.0, [dens.n_live], 0
    clocks = ClockSampler()
    clocks.start()
    for seg in range(segments):
        e0.record()
        for _ in range(DENS_EVERY):
            ms.step()
        e1.record()
        torch.cuda.synchronize()
        if ms.status() != 0:
            raise RuntimeError(f"device status {ms.status():#x} in segment {seg} (pair capacity)")
        step_ms += e0.elapsed_time(e1)
        if seg == segments - 1:
            break
        t0 = time.time()
        n_live, grown = dens.step()
        counts.append(n_live)
        # a new store, or a map grown by 30 % since the pair capacity was sized
        # (it carries a 50 % margin), is captured again; a segment that still
        # overflowed would stop the run above
        if grown or n_live > 1.3 * sized_for:
            ms = build()
            sized_for = n_live
            rebuilds += 1
        torch.cuda.synchronize()
        dens_ms += (time.time() - t0) * 1e3
    clk = clocks.stop(int(os.environ.get("LOCAL_RANK", "0")))
    iters = segments * DENS_EVERY
    total_ms = step_ms + dens_ms
    line = {"metric": f"mapping iters/s with densify / prune every {DENS_EVERY} @{DENS_N // 1000}k starting "
                      f"Gaussians {DENS_W}x{DENS_H}",
            "value": iters * 1000.0 / total_ms, "unit": "iters/s", "n_gpus": 1, "steps": iters,
            "warmup": args.warmup, "ms_per_step": total_ms / iters, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; 1920x1080 frames)",
            "config": {"workload": f"{DENS_N} Gaussians (perturbed room scene), {DENS_W}x{DENS_H} fx=fy={DENS_F:.0f}, "
                                   f"{N_POSES}-pose trajectory; every {DENS_EVERY} iterations clone / split where the "
                                   "mean NDC gradient norm >= 2e-4 (split above scale 0.03 m), prune opacity < 0.005; "
                                   "store with 25 % spare capacity, re-captured when it overflows or the map grew "
                                   "30 % since the pair capacity was sized", "gaussians_after_each_densify": counts,
                       "rebuilds": rebuilds, "first_build_s": round(build_s[0], 1), "map_order": args.order},
            "iteration_ms": step_ms / iters, "densify_ms_per_step": dens_ms / max(1, segments - 1),
            "clocks": clk}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- stereo grayscale views
STEREO_N = 300_000


def run_stereo(args):
    import torch
    import synthetic as S
    import paper_2311_16728_b300 as gsr
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    target = S.room_scene(STEREO_N, seed=0)
    start = S.perturb(target, 0.05, seed=1)
    cams = [c for k in range(N_POSES) for c in S.stereo_pair(k)]
    g_tgt = gsr.Gaussians.from_arrays(target.mean_op, target.quat, target.logscale, target.sh)
    vb = gsr.ViewBuffers(STEREO_N, gsr.camera_from(cams[0]), gsr.tiling_struct(16, 16), 1024)
    views = []
    for cam in cams:
        vb.cam = gsr.camera_from(cam)
        gsr.ensure_capacity(vb, g_tgt)
        vb.forward(g_tgt)
        # monochrome target: the luminance of the true render
        views.append((cam, (0.299 * vb.img[0] + 0.587 * vb.img[1] + 0.114 * vb.img[2])[None].contiguous()))
    del vb, g_tgt
    params = _ordered(gsr, gsr.Gaussians.from_arrays(start.mean_op, start.quat, start.logscale, start.sh), args)
    ms = gsr.MappingStep(params, views)
    ms.capture()
    for _ in range(args.warmup):
        ms.step()
    torch.cuda.synchronize()
    nst = len(gsr.STAGES)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nst + 1)] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler()
    clocks.start()
    torch.cuda.synchronize()
    t0.record()
    for k in range(args.steps):
        ms.step(events=evs[k])
    t1.record()
    torch.cuda.synchronize()
    clk = clocks.stop(int(os.environ.get("LOCAL_RANK", "0")))
    if ms.status() != 0:
        raise RuntimeError(f"device status {ms.status():#x}")
    ms_per = t0.elapsed_time(t1) / args.steps
    stage_ms = {nm: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs) for i, nm in enumerate(gsr.STAGES)}
    line = {"metric": f"stereo grayscale mapping iters/s @{STEREO_N // 1000}k Gaussians 752x480",
            "value": 1000.0 / ms_per, "unit": "iters/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded; EuRoC-shaped monochrome stereo)",
            "config": {"workload": f"{STEREO_N} Gaussians in a 6x3x4 m room; {N_POSES} poses x 2 cameras "
                                   "(0.11 m baseline) of 752x480 fx=fy=376, one view per iteration, Eq. 4 on the "
                                   "luminance 0.299 R + 0.587 G + 0.114 B against monochrome targets, Adam",
                       "map_order": args.order},
            "stages_ms": stage_ms, "clocks": clk}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- camera pose gradient
def run_pose(args):
    """Pose-gradient passes on the mapping workload: one pass = preprocess,
    binning, forward blend, Eq. 4 loss and gradient, backward blend and the
    camera pose chain (gsr_pose_bwd), captured as one CUDA graph for a fixed
    pose; plus an eager photometric refinement (host pose update, one sync
    per step) from a pose 1 degree and 3 cm off."""
    import torch
    import synthetic as S
    import paper_2311_16728_b300 as gsr
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    target, _, cams = _scene(1)
    true_cam = cams[0]
    g = _ordered(gsr, gsr.Gaussians.from_arrays(target.mean_op, target.quat, target.logscale, target.sh), args)
    vb = gsr.ViewBuffers(N_GAUSS, gsr.camera_from(true_cam), gsr.tiling_struct(16, 16), 1024)
    gsr.ensure_capacity(vb, g)
    vb.forward(g)
    gt = vb.img.clone()
    R0 = gsr.so3_exp([0.01, -0.012, 0.006]) @ true_cam.R
    t0 = true_cam.t + np.array([0.02, -0.015, 0.012])
    start = S.Camera(R0, t0, true_cam.fx, true_cam.fy, true_cam.cx, true_cam.cy, true_cam.width, true_cam.height)
    vb.cam = gsr.camera_from(start)
    gsr.ensure_capacity(vb, g)
    vb.set_pair_capacity(int(vb.pairs_needed() * 1.3) + 4096)
    d_pose = torch.zeros(15, dtype=torch.float32, device="cuda")

    def grad_pass(stream):
        vb.forward(g, stream=stream)
        vb.loss_fwd_bwd(gt, stream=stream)
        vb.blend_bwd(stream=stream)
        d_pose.zero_()
        vb.pose_bwd(g, d_pose, stream=stream)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        grad_pass(s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    whole = torch.cuda.CUDAGraph()
    with torch.cuda.graph(whole):
        grad_pass(torch.cuda.current_stream())
    chain = torch.cuda.CUDAGraph()
    with torch.cuda.graph(chain):
        vb.pose_bwd(g, d_pose, stream=torch.cuda.current_stream())
    for _ in range(args.warmup):
        whole.replay()
    torch.cuda.synchronize()
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler()
    clocks.start()
    torch.cuda.synchronize()
    t0e.record()
    for _ in range(args.steps):
        whole.replay()
    t1e.record()
    torch.cuda.synchronize()
    ms_pass = t0e.elapsed_time(t1e) / args.steps
    # the pose chain alone (inputs: params 240 B + screen-space gradients 48 B per visible Gaussian, the
    # visibility word of every Gaussian), timed the same way
    t0e.record()
    for _ in range(args.steps):
        chain.replay()
    t1e.record()
    torch.cuda.synchronize()
    clk = clocks.stop(int(os.environ.get("LOCAL_RANK", "0")))
    ms_chain = t0e.elapsed_time(t1e) / args.steps
    if vb.read_status() != 0:
        raise RuntimeError(f"device status {vb.read_status():#x}")
    nv = int((vb.ntiles > 0).sum().item())
    alg = 4 * N_GAUSS + (240 + 48) * nv
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6400.0)
    achieved = alg / (ms_chain * 1e-3) / 1e9
    # refinement: eager, host update and read-back every step
    ref = gsr.PoseRefiner(g, start, gt)

    def err(R, t):
        ang = float(np.degrees(np.arccos(np.clip((np.trace(R @ true_cam.R.T) - 1) / 2, -1, 1))))
        return ang, float(np.linalg.norm(t - true_cam.t))

    e0 = err(ref.R, ref.t)
    n_ref = 60
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    losses = []
    for k in range(n_ref):
        if k == 40:
            ref.lr = ref.lr * 0.1
        losses.append(ref.step())
    w1 = time.perf_counter()
    e1 = err(ref.R, ref.t)
    line = {"metric": "pose-gradient passes/s @300k Gaussians 1200x680", "value": 1000.0 / ms_pass,
            "unit": "passes/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_pass,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded; Replica-shaped)",
            "config": {"workload": "camera pose gradient of Eq. 4 through the Eq. 3 render: 300k Gaussians in a "
                                   "6x3x4 m room, 1200x680 fx=fy=600, frame rendered from the true pose, camera "
                                   "1 degree / 3 cm off; preprocess, binning, forward blend, loss, backward blend "
                                   "and pose chain in one CUDA graph (fixed pose)",
                       "visible": nv, "pairs": vb.pairs_needed(), "map_order": args.order},
            "roofline": {"kernel": "pose_bwd_kernel", "bound": "hbm", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": NCU_TRAFFIC_POSE if args.order == "morton" else None, "alg_bytes": alg,
                         "ms": ms_chain, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
            "refinement": {"steps": n_ref, "steps_per_s": n_ref / (w1 - w0), "rot_err_deg": [e0[0], e1[0]],
                           "trans_err_m": [e0[1], e1[1]], "loss": [losses[0], losses[-1]],
                           "note": "eager: camera updated on the host, one read-back per step"},
            "clocks": clk}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- Gaussian-pyramid ablation
def run_gp_ablation(args):
    """Plain path with n + 1 = 1 .. 4 pyramid levels on the held-out
    time-to-PSNR scenes, same iteration budget: final PSNR and time (the
    paper's ablation of GP learning, Sec. 4.4, Tab. 4, and its remark that
    more levels stop helping)."""
    import torch
    import paper_2311_16728_b300 as gsr
    from paper_2311_16728_b300.mapping import Evaluator, PlainMapper, densify_default
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    seeds = [int(x) for x in args.ttp_seeds.split(",") if x][:3]
    budget = TTP_BUDGET
    rows = {}
    for seed in seeds:
        truth, keyframes, kps, offsets = _ttp_setup(seed, gsr, torch)
        ev = Evaluator(TTP_N, keyframes)
        for levels in (1, 2, 3, 4):
            params = gsr.Gaussians.from_arrays(truth.mean_op, truth.quat, truth.logscale, truth.sh)
            densify_default(params, keyframes, kps, offsets)
            pm = PlainMapper(params, keyframes, levels=levels)
            pm.capture()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(budget):
                pm.step()
            e1.record()
            torch.cuda.synchronize()
            if pm.status() != 0:
                raise RuntimeError(f"device status {pm.status():#x}")
            rows.setdefault(str(levels), []).append({"seed": seed, "psnr": ev(params), "ms": e0.elapsed_time(e1)})
            del pm, params
    summary = {k: {"psnr_mean": statistics.mean(r["psnr"] for r in v), "ms_mean": statistics.mean(r["ms"] for r in v)}
               for k, v in rows.items()}
    best = max(summary, key=lambda k: summary[k]["psnr_mean"])
    line = {"metric": "Gaussian-pyramid ablation: final PSNR of the plain path with 1-4 levels",
            "value": summary["3"]["psnr_mean"] - summary["1"]["psnr_mean"], "unit": "dB (3 levels minus 1)",
            "n_gpus": 1, "higher_is_better": True, "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded; held-out scenes)",
            "config": {"workload": f"time-to-PSNR scenes {seeds}, default initialisation, {budget} iterations of the "
                                   "plain path (one view per iteration, tau_u 30) with n + 1 pyramid levels",
                       "best_levels": int(best)},
            "levels": summary, "per_seed": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-rows", type=int, default=64, help="image rows per oracle step (reference arm)")
    ap.add_argument("--cpu-rows", type=int, default=680, help="image rows of the cpu_baseline sample")
    ap.add_argument("--mode", default="mapping",
                    choices=["mapping", "window", "mlp", "ttp", "densify", "stereo", "gp_ablation", "pose"])
    ap.add_argument("--ttp-seeds", default="100,101,102,103,104", help="ttp mode: held-out evaluation scenes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", default="auto", help="window mode: WxH tile shape instead of the autotuner's choice")
    ap.add_argument("--profile", action="store_true",
                    help="run --steps iterations between cudaProfilerStart/Stop after the warm-up and exit "
                         "(for ncu --profile-from-start off); prints no bench line")
    ap.add_argument("--poses", type=int, default=N_POSES, help="trajectory poses trained on (profiling uses fewer)")
    ap.add_argument("--scene", default="room", choices=["room", "walls"],
                    help="mapping mode: Gaussians filling the room (headline) or on its six walls (sensitivity variant)")
    ap.add_argument("--order", default="morton", choices=["morton", "input"],
                    help="map store in Morton order of the means (setup) or in generator order")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.mode == "window":
        run_window(args)
        return
    if args.mode == "mlp":
        run_mlp(args)
        return
    if args.mode == "ttp":
        run_ttp(args)
        return
    if args.mode == "densify":
        run_densify(args)
        return
    if args.mode == "stereo":
        run_stereo(args)
        return
    if args.mode == "gp_ablation":
        run_gp_ablation(args)
        return
    if args.mode == "pose":
        run_pose(args)
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2311_16728_b300 as gsr
    target, start, cams = _scene(args.poses, args.scene)

    # targets: renders of the unperturbed set at every pose (setup, untimed)
    g_tgt = gsr.Gaussians.from_arrays(target.mean_op, target.quat, target.logscale, target.sh)
    tiling = gsr.tiling_struct(16, 16)
    vb = gsr.ViewBuffers(N_GAUSS, gsr.camera_from(cams[0]), tiling, 1024)
    gts = []
    for cam in cams:
        vb.cam = gsr.camera_from(cam)
        gsr.ensure_capacity(vb, g_tgt)
        vb.forward(g_tgt)
        gts.append(vb.img.clone())
    del vb, g_tgt
    params = _ordered(gsr, gsr.Gaussians.from_arrays(start.mean_op, start.quat, start.logscale, start.sh), args)
    ms = gsr.MappingStep(params, list(zip(cams, gts)), tiling)
    ms.capture()
    for _ in range(args.warmup):
        ms.step()
    torch.cuda.synchronize()
    if args.profile:
        _profile_steps(ms.step, args.steps)
        return
    if world > 1:
        dist.barrier()

    # ---- timed region: K whole iterations, one graph replay each
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler()
    clocks.start()
    torch.cuda.synchronize()
    t_start.record()
    for k in range(args.steps):
        ms.step()
    t_end.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms_total = t_start.elapsed_time(t_end)
    # ---- stage times: the same iterations replayed one graph per stage,
    # events between the stages (live, on the launching stream)
    nst = len(gsr.STAGES)
    k_st = min(args.steps, 300)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nst + 1)] for _ in range(k_st)]
    for k in range(k_st):
        ms.step(events=evs[k])
    torch.cuda.synchronize()
    clk = clocks.stop(local)
    stage_ms = {name: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs) for i, name in enumerate(gsr.STAGES)}
    status = ms.status()
    pairs = int(ms.vb.num_pairs.item())
    if status != 0:
        raise RuntimeError(f"device status {status} during the timed region (pair capacity {ms.vb.pair_capacity})")
    ms_total = max_over_ranks(ms_total, "cuda")
    ms_per_step = ms_total / args.steps
    value = job_rate(ms_per_step, world)

    # ---- end to end: target image from pinned host memory in, loss out, every
    # step.  Each step's target is copied on a second stream one step ahead,
    # while the previous step computes (double buffering: each view has its
    # own device buffer, last read 50 steps earlier; the copy waits for the
    # step before the current one); every copy lies inside the timed region.
    host_gts = [g.cpu().pin_memory() for g in gts]
    host_loss = torch.empty(1, dtype=torch.float32).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    main, copy = torch.cuda.current_stream(), torch.cuda.Stream()
    nv, k0 = len(ms.views), ms.k
    ready = [torch.cuda.Event() for _ in range(args.steps)]
    done = [torch.cuda.Event() for _ in range(args.steps)]

    def fetch(k):  # the target of step k, on the copy stream
        j = (k0 + k) % nv
        with torch.cuda.stream(copy):
            ms.views[j][1].copy_(host_gts[j], non_blocking=True)
        ready[k].record(copy)

    torch.cuda.synchronize()
    e0.record()
    copy.wait_stream(main)
    fetch(0)
    for k in range(args.steps):
        main.wait_event(ready[k])
        if k + 1 < args.steps:
            if k >= 1:
                copy.wait_event(done[k - 1])
            fetch(k + 1)
        ms.step()
        done[k].record(main)
        host_loss.copy_(ms.vb.loss, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    e2e_ms = max_over_ranks(e2e_ms, "cuda")

    # ---- kernels launched per iteration (kernel nodes of one view's graph)
    try:
        per_iter = count_kernel_nodes([ms.whole[0]])
    except Exception:  # introspection unavailable: count from the launch sequence
        per_iter = None
    launches = per_iter * args.steps if per_iter is not None else None

    # ---- work counters at the final state (outside the timed region): visible
    # Gaussians, pairs, and (pixel, Gaussian) blends over the first poses
    vb = ms.vb
    nblend = torch.zeros(HEIGHT, WIDTH, dtype=torch.int32, device="cuda")
    blends, nvis = [], []
    for k in range(min(5, len(ms.views))):
        vb.cam = ms.views[k][0]
        vb.preprocess(params)
        vb.bin_sort()
        vb.render_fwd(n_blended=nblend)
        blends.append(int(nblend.sum().item()))
        nvis.append(int((vb.ntiles > 0).sum().item()))
    work = {"blends": statistics.mean(blends), "visible": statistics.mean(nvis), "pairs": pairs}

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    # the captured DRAM traffic is the room scene's in the Morton-ordered
    # store; other scenes and orders report none
    traffic = NCU_TRAFFIC if (args.scene == "room" and args.order == "morton") else {}
    stages = stage_rooflines(stage_ms, work, peaks, clk, traffic)
    dom = max(stage_ms, key=stage_ms.get)
    roof = dict(stages[dom])

    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; Replica-shaped)",
            "config": _config({"pairs_last_step": pairs, "poses": len(cams), "scene": args.scene,
                               "map_order": args.order,
                               **({"workload": WORKLOAD_WALLS} if args.scene == "walls" else {})}),
            "roofline": roof, "stages_ms": stage_ms, "stage_rooflines": stages, "work": work,
            "gpu_launches": launches, "clocks": clk,
            "e2e": {"value": job_rate(e2e_ms, world), "unit": "iters/s",
                    "h2d_bytes_per_step": 3 * WIDTH * HEIGHT * 4, "d2h_bytes_per_step": 4}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        import synthetic as S
        rows = min(args.cpu_rows, HEIGHT)
        row0 = (HEIGHT - rows) // 2
        st = oracle.Scene64(target.mean_op, target.quat, target.logscale, target.sh)
        total, measured = 0.0, 0.0
        poses = (0, 1)
        for pose in poses:
            cam = cams[pose]
            dt = oracle.decide(target.mean_op, target.quat, target.logscale, cam.as_array(), WIDTH, HEIGHT)
            im, _, _, _ = oracle.render(st, cam.as_array(), WIDTH, HEIGHT, dt, rows=(row0, row0 + rows))
            full, det = oracle_sample(start, im[:, row0:row0 + rows].copy(), cams, pose, rows, row0)
            total += full
            measured += det["measured_s"]
        line["cpu_baseline"] = {"value": len(poses) / total, "unit": "iters/s", "cores": oracle.num_threads(),
                                "kind": "oracle",
                                "sample": f"{len(poses)} iterations (poses 0, 1): decide+Adam over all {N_GAUSS} "
                                          f"Gaussians, render+loss+backward on rows {row0}-{row0 + rows} of 680"
                                          + (", extrapolated to the full frame" if rows < HEIGHT else "")
                                          + f" ({measured:.1f} s measured)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# DRAM bytes (read + write) per launch from one ncu capture of this workload
# with the current kernels (profiles/mapping_kernels_300k_1200x680.md; the
# loss stage is its two SSIM passes, the binning stage its seven kernels).
NCU_TRAFFIC = {"preprocess": 15.454464e6, "bin_sort": 21.094912e6, "render_fwd": 4.217856e6, "loss": 69.083904e6,
               "blend_bwd": 20.793600e6, "preprocess_bwd": 12.432640e6, "adam": 393.139456e6}
# the pose chain (profiles/pose_bwd_300k_1200x680.md)
NCU_TRAFFIC_POSE = 15.037952e6
# the persistent window kernel (profiles/window_kernels_500k_8x640x480x3.md)
NCU_TRAFFIC_WINDOW_ITERATE = 604.692224e6

# FP32 work per blended (pixel, Gaussian) pair and algorithmic bytes per unit.
FLOPS_PER_BLEND_FWD = 20
FLOPS_PER_BLEND_BWD = 60


def stage_rooflines(stage_ms, work, peaks, clk, traffic):
    """Roofline entry of each stage's dominant kernel: algorithmic work per
    launch / measured stage time against the measured HBM copy bandwidth or
    the FP32 peak (148 SMs x 128 lanes x 2 flops x median SM clock)."""
    hbm = peaks.get("hbm_gbs", 6400.0)
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6400 GB/s (of fallback)"
    mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    fp32 = 148 * 128 * 2 * mhz * 1e6 / 1e12
    n, nv, K, E = N_GAUSS, work["visible"], work["pairs"], work["blends"]
    px = 3 * WIDTH * HEIGHT

    def hbm_entry(kernel, alg):
        sec = stage_ms[st] * 1e-3
        return {"kernel": kernel, "bound": "hbm", "achieved": alg / sec / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": alg / sec / 1e9 / hbm, "traffic": traffic.get(st), "alg_per_launch": alg,
                "peak_source": hbm_src}

    def alu_entry(kernel, flops):
        sec = stage_ms[st] * 1e-3
        return {"kernel": kernel, "bound": "alu", "achieved": flops / sec / 1e12, "peak": fp32, "unit": "TFLOP/s",
                "frac": flops / sec / 1e12 / fp32, "traffic": traffic.get(st), "alg_per_launch": flops,
                "peak_source": f"FP32 148 SMs x 128 lanes x 2 x {mhz:.0f} MHz (sampled median clock)"}

    out = {}
    for st in stage_ms:
        if st == "preprocess":
            # the frustum test reads the mean (16 B) and every Gaussian's tile
            # count is written (4 B); a visible Gaussian also reads rotation
            # and scale (32 B) and SH (192 B) and writes its record (48 B)
            out[st] = hbm_entry("preprocess_fwd_kernel", (16 + 4) * n + (32 + 192 + 48) * nv)
        elif st == "bin_sort":
            # depth passes 4 x 16 B per visible, tile passes 2 x 16 B per pair, keys + values out 12 B per pair
            out[st] = hbm_entry("binning + radix passes", 4 * 16 * nv + 2 * 16 * K + 12 * K)
        elif st == "render_fwd":
            out[st] = alu_entry("render_fwd_kernel", FLOPS_PER_BLEND_FWD * E)
        elif st == "loss":
            # x, y read twice, three maps written and read, dL/dx written
            out[st] = hbm_entry("ssim_pass1/2_kernel", 4 * px * (2 + 3 + 3 + 2 + 1))
        elif st == "blend_bwd":
            out[st] = alu_entry("render_bwd_q4_kernel", FLOPS_PER_BLEND_BWD * E)
        elif st == "preprocess_bwd":
            # per visible Gaussian: parameters 240 B and screen-space gradient
            # 48 B read, gradients 240 B stored (they are zero before the pass),
            # densify statistic and count 16 B; visibility word 4 B per Gaussian
            out[st] = hbm_entry("preprocess_bwd_kernel", (240 + 48 + 240 + 16) * nv + 4 * n)
        elif st == "adam":
            # 15 float4 planes: param, m, v read + written for every Gaussian, the
            # gradient read + zeroed only where the view flag (4 B) is set
            out[st] = hbm_entry("adam_kernel", (15 * 16 * 6 + 4) * n + 15 * 16 * 2 * nv)
    return out


if __name__ == "__main__":
    main()
