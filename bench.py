"""Benchmark: fwd+bwd mapping iterations/s at 300k Gaussians, 1200 x 680.

One step = one whole photorealistic-mapping iteration of Photo-SLAM
(arXiv 2311.16728, Sec. 3.3): EWA preprocess, tile binning + radix sort,
forward blend (Eq. 3), L1 + D-SSIM loss and its gradient (Eq. 4, lambda 0.2),
backward blend + chain rule, fused Adam, on one view of a 50-pose trajectory.
Inputs are seeded synthetic scenes shaped like the paper's Replica frames (the
dataset itself is not available).  The path does not shard: with --gpus N
every rank runs an independent replica (weak scaling, no collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only other implementation of
this path) on the host cores, on a bounded band of image rows per step.
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


def _scene(poses: int = N_POSES):
    import synthetic as S
    target = S.room_scene(N_GAUSS, seed=0)
    start = S.perturb(target, 0.05, seed=1)
    cams = [S.replica_camera(k) for k in range(poses)]
    return target, start, cams


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
    fixed = (t1 - t0) + (t2 - t1) + (t5 - t4) + (t7 - t6)
    per_band = (t3 - t2) + (t4 - t3) + (t6 - t5)
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
    for k in range(args.warmup + args.steps):
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
        if k >= args.warmup:
            per_step.append(full)
    sec = statistics.mean(per_step)
    cores = oracle.num_threads()
    sample = (f"oracle (FP64, OpenMP) per step: decide+Adam over all {N_GAUSS} Gaussians, render+loss+backward on a "
              f"{rows}-row band of the 1200x680 frame, extrapolated to the full frame")
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-rows", type=int, default=8, help="image rows per oracle step (reference arm)")
    ap.add_argument("--cpu-rows", type=int, default=160, help="image rows of the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--poses", type=int, default=N_POSES, help="trajectory poses trained on (profiling uses fewer)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
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
    target, start, cams = _scene(args.poses)

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
    params = gsr.Gaussians.from_arrays(start.mean_op, start.quat, start.logscale, start.sh)
    ms = gsr.MappingStep(params, list(zip(cams, gts)), tiling)
    ms.capture()
    for _ in range(args.warmup):
        ms.step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    # ---- timed region: K whole iterations, events between stages
    nst = len(gsr.STAGES)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nst + 1)] for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler()
    clocks.start()
    torch.cuda.synchronize()
    t_start.record()
    for k in range(args.steps):
        ms.step(events=evs[k])
    t_end.record()
    torch.cuda.synchronize()
    clk = clocks.stop(local)
    if world > 1:
        dist.barrier()
    ms_total = t_start.elapsed_time(t_end)
    stage_ms = {name: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs) for i, name in enumerate(gsr.STAGES)}
    status = ms.status()
    pairs = int(ms.vb.num_pairs.item())
    if status != 0:
        raise RuntimeError(f"device status {status} during the timed region (pair capacity {ms.vb.pair_capacity})")
    if world > 1:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_per_step = ms_total / args.steps
    value = world * 1000.0 / ms_per_step

    # ---- end to end: target image from pinned host memory in, loss out, every step
    host_gts = [g.cpu().pin_memory() for g in gts]
    host_loss = torch.empty(1, dtype=torch.float32).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for k in range(args.steps):
        i = ms.k % len(ms.views)
        ms.views[i][1].copy_(host_gts[i], non_blocking=True)
        ms.step()
        host_loss.copy_(ms.vb.loss, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())

    # ---- kernels launched per iteration (kernel nodes of one view's graphs)
    try:
        per_iter = count_kernel_nodes(ms.graphs[0])
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
    stages = stage_rooflines(stage_ms, work, peaks, clk)
    dom = max(stage_ms, key=stage_ms.get)
    roof = dict(stages[dom])

    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; Replica-shaped)",
            "config": _config({"pairs_last_step": pairs, "poses": len(cams)}),
            "roofline": roof, "stages_ms": stage_ms, "stage_rooflines": stages, "work": work,
            "gpu_launches": launches, "clocks": clk,
            "e2e": {"value": world * 1000.0 / e2e_ms, "unit": "iters/s",
                    "h2d_bytes_per_step": 3 * WIDTH * HEIGHT * 4, "d2h_bytes_per_step": 4}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        import synthetic as S
        rows = min(args.cpu_rows, HEIGHT)
        row0 = (HEIGHT - rows) // 2
        cam = cams[0]
        dt = oracle.decide(target.mean_op, target.quat, target.logscale, cam.as_array(), WIDTH, HEIGHT)
        st = oracle.Scene64(target.mean_op, target.quat, target.logscale, target.sh)
        im, _, _, _ = oracle.render(st, cam.as_array(), WIDTH, HEIGHT, dt, rows=(row0, row0 + rows))
        full, det = oracle_sample(start, im[:, row0:row0 + rows].copy(), cams, 0, rows, row0)
        line["cpu_baseline"] = {"value": 1.0 / full, "unit": "iters/s", "cores": oracle.num_threads(),
                                "kind": "oracle",
                                "sample": f"one iteration at pose 0: decide+Adam over all {N_GAUSS} Gaussians, "
                                          f"render+loss+backward on rows {row0}-{row0 + rows} of 680, "
                                          f"extrapolated to the full frame ({det['measured_s']:.1f} s measured)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# DRAM bytes per launch of a kernel from one ncu capture of this workload
# (profiles/blend_kernels_300k_1200x680.md); None when not captured for the
# current kernel version.
NCU_TRAFFIC = {"blend_bwd": 28.203264e6, "render_fwd": 11.310336e6}

# FP32 work per blended (pixel, Gaussian) pair and algorithmic bytes per unit.
FLOPS_PER_BLEND_FWD = 20
FLOPS_PER_BLEND_BWD = 60


def stage_rooflines(stage_ms, work, peaks, clk):
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
                "frac": alg / sec / 1e9 / hbm, "traffic": NCU_TRAFFIC.get(st), "alg_per_launch": alg,
                "peak_source": hbm_src}

    def alu_entry(kernel, flops):
        sec = stage_ms[st] * 1e-3
        return {"kernel": kernel, "bound": "alu", "achieved": flops / sec / 1e12, "peak": fp32, "unit": "TFLOP/s",
                "frac": flops / sec / 1e12 / fp32, "traffic": NCU_TRAFFIC.get(st), "alg_per_launch": flops,
                "peak_source": f"FP32 148 SMs x 128 lanes x 2 x {mhz:.0f} MHz (sampled median clock)"}

    out = {}
    for st in stage_ms:
        if st == "preprocess":
            out[st] = hbm_entry("preprocess_fwd_kernel", 48 * n + 4 * n + (192 + 48) * nv)
        elif st == "bin_sort":
            # depth passes 4 x 16 B per visible, tile passes 2 x 16 B per pair, keys + values out 12 B per pair
            out[st] = hbm_entry("binning + radix passes", 4 * 16 * nv + 2 * 16 * K + 12 * K)
        elif st == "render_fwd":
            out[st] = alu_entry("render_fwd_kernel", FLOPS_PER_BLEND_FWD * E)
        elif st == "loss":
            # x, y read twice, three maps written and read, dL/dx written
            out[st] = hbm_entry("ssim_pass1/2_kernel", 4 * px * (2 + 3 + 3 + 2 + 1))
        elif st == "blend_bwd":
            out[st] = alu_entry("render_bwd_kernel", FLOPS_PER_BLEND_BWD * E)
        elif st == "preprocess_bwd":
            out[st] = hbm_entry("preprocess_bwd_kernel", (240 + 48 + 480) * nv)
        elif st == "adam":
            # 15 float4 planes x (param r+w, grad r+w, m r+w, v r+w)
            out[st] = hbm_entry("adam_kernel", 15 * 16 * 8 * n)
    return out


if __name__ == "__main__":
    main()
