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
pose refinement.  The default (mapping) line is the headline; after its
throughput figure it also carries the batched window's rate (`window`) and a
bounded time-to-PSNR run (`ttp`: the learned initialiser trained on the GPU
inside the run, two held-out scenes), the two halves of the headline metric.
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
            "50-pose seeded trajectory, autotuned tiling, L1+D-SSIM (lambda 0.2), Adam, FP32")


def _config(extra=None):
    c = {"workload": WORKLOAD, "gaussians": N_GAUSS, "width": WIDTH, "height": HEIGHT,
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
    """The oracle on the host cores, every one of the K steps a bounded sample
    of one mapping iteration: decide + Adam over all Gaussians, render, loss
    and backward on a band of rows, the band's time scaled to the frame.
    ms_per_step is the measured time of a sampled step (so K x ms_per_step is
    the timed region); value is the full-frame rate that the samples
    extrapolate to."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synthetic as S
    target, start, cams = _scene()
    # bands of consecutive rows that tile the frame over the K timed steps
    # (image rows differ in cost, so the steps together sample every row)
    rows = args.ref_rows if args.ref_rows > 0 else min(HEIGHT, max(8, -(-HEIGHT // args.steps)))
    tgt_cache = {}
    n_warm = min(args.warmup, 1)
    full, measured = [], []
    t_region = None
    for k in range(n_warm + args.steps):
        if k == n_warm:
            t_region = time.perf_counter()
        pose = k % N_POSES
        row0 = min(((k - n_warm) % max(1, -(-HEIGHT // rows))) * rows, HEIGHT - rows)
        key = (pose, row0)
        if key not in tgt_cache:  # the target band (untimed): the oracle's render of the unperturbed set
            cam = cams[pose]
            dt = oracle.decide(target.mean_op, target.quat, target.logscale, cam.as_array(), WIDTH, HEIGHT)
            st = oracle.Scene64(target.mean_op, target.quat, target.logscale, target.sh)
            im, _, _, _ = oracle.render(st, cam.as_array(), WIDTH, HEIGHT, dt, rows=(row0, row0 + rows))
            tgt_cache = {key: im[:, row0:row0 + rows].copy()}
        f, det = oracle_sample(start, tgt_cache[key], cams, pose, rows, row0)
        if k >= n_warm:
            full.append(f)
            measured.append(det["measured_s"])
    timed_s = time.perf_counter() - t_region
    sec_full = statistics.mean(full)
    cores = oracle.num_threads()
    sample = (f"oracle (FP64, OpenMP), {args.steps} timed steps after {n_warm} warm-up, each a sample of one "
              f"iteration: decide + Adam over all {N_GAUSS} Gaussians, render + loss + backward on a {rows}-row band "
              f"of the 1200x680 frame, the steps' bands tiling the frame ({statistics.mean(measured):.2f} s measured "
              f"per step); value = the full-frame rate, each band's share scaled by {HEIGHT}/{rows} "
              f"({sec_full:.2f} s per full iteration, mean over the steps)")
    value = 1.0 / sec_full
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(measured) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(), "timed_steps": args.steps, "timed_s": timed_s, "extrapolated": True,
            "full_frame_ms_per_step": sec_full * 1e3,
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
class _NvmlCtypes:
    """The few read-only NVML queries the clock sampler makes, through ctypes
    on libnvidia-ml (for hosts without the pynvml module)."""
    NVML_CLOCK_SM = 1

    class NVMLError(Exception):
        pass

    def __init__(self):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")

    def _ok(self, rc):
        if rc != 0:
            raise self.NVMLError(f"NVML error {rc}")

    def nvmlInit(self):
        self._ok(self.lib.nvmlInit_v2())

    def nvmlDeviceGetCount(self):
        n = self.c.c_uint()
        self._ok(self.lib.nvmlDeviceGetCount_v2(self.c.byref(n)))
        return n.value

    def nvmlDeviceGetHandleByIndex(self, k):
        h = self.c.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByIndex_v2(self.c.c_uint(k), self.c.byref(h)))
        return h

    def nvmlDeviceGetUUID(self, h):
        buf = self.c.create_string_buffer(96)
        self._ok(self.lib.nvmlDeviceGetUUID(h, buf, self.c.c_uint(96)))
        return buf.value.decode()

    def nvmlDeviceGetPciInfo(self, h):
        raise self.NVMLError("PCI info not queried through ctypes")

    def _uint(self, fn, h, *args):
        v = self.c.c_uint()
        self._ok(fn(h, *args, self.c.byref(v)))
        return v.value

    def nvmlDeviceGetClockInfo(self, h, kind):
        return self._uint(self.lib.nvmlDeviceGetClockInfo, h, self.c.c_int(kind))

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        return self._uint(self.lib.nvmlDeviceGetMaxClockInfo, h, self.c.c_int(kind))

    def nvmlDeviceGetPowerUsage(self, h):
        return self._uint(self.lib.nvmlDeviceGetPowerUsage, h)

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.c.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self._ok(fn(h, self.c.byref(v)))
        return v.value


def _nvml_module():
    try:
        import pynvml
        return pynvml
    except ImportError:
        return _NvmlCtypes()


class ClockSampler:
    """SM clock, power and clock-event reasons of the benchmarked GPU, sampled
    every few milliseconds by a background thread through NVML's read-only
    queries (nvidia-smi's 100 ms loop as the fallback).  Started before the
    warm-up and stopped after the last measured loop, so it also covers timed
    regions far shorter than its period; `mark` records which samples fall
    inside the headline's timed region."""

    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
               ("sw_power_cap", 0x4))

    def __init__(self, device=None, period_s: float = 0.004):
        import threading
        self.device, self.period = device, period_s
        self.samples = []  # (t, sm_mhz, max_mhz, power_w, reason bits)
        self.marks = {}
        self.stop_ev = threading.Event()
        self.thread = None
        self.smi = None
        self.source = None
        self.nvml_error = None

    def _nvml_handle(self):
        """NVML handle of the CUDA device: NVML numbers every GPU of the node,
        so the device is found by its UUID (else its PCI bus id)."""
        import torch
        pynvml = _nvml_module()
        pynvml.nvmlInit()
        if self.device is None:
            self.device = torch.cuda.current_device()
        props = torch.cuda.get_device_properties(self.device)
        want = str(props.uuid).lower().replace("gpu-", "")
        bus = (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
        for k in range(pynvml.nvmlDeviceGetCount()):
            h = pynvml.nvmlDeviceGetHandleByIndex(k)
            uuid = pynvml.nvmlDeviceGetUUID(h)
            uuid = (uuid.decode() if isinstance(uuid, bytes) else str(uuid)).lower().replace("gpu-", "")
            if uuid == want:
                return pynvml, h
            try:
                pci = pynvml.nvmlDeviceGetPciInfo(h)
            except Exception:
                continue
            if (pci.domain, pci.bus, pci.device) == bus:
                return pynvml, h
        raise RuntimeError(f"no NVML device with UUID {want} or PCI {bus}")

    def start(self):
        import threading
        try:
            nv, h = self._nvml_handle()
        except Exception as e:  # recorded in the clock record; nvidia-smi is the fallback
            nv, self.nvml_error = None, f"{type(e).__name__}: {e}"[:200]
        if nv is None:
            self._start_smi()
            return
        self.source = "NVML (read-only queries, " + ("ctypes" if isinstance(nv, _NvmlCtypes) else "pynvml") + ")"

        def run():
            get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons",
                                  getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons", None))
            while not self.stop_ev.is_set():
                try:
                    self.samples.append((time.perf_counter(), float(nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM)),
                                         float(nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM)),
                                         nv.nvmlDeviceGetPowerUsage(h) / 1000.0, int(get_reasons(h))))
                except Exception:
                    pass
                self.stop_ev.wait(self.period)

        self.thread = threading.Thread(target=run, daemon=True)
        self.thread.start()

    def _start_smi(self):
        self.source = "nvidia-smi -lms 100"
        self.period = 0.1
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active")
        try:
            self.smi = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms",
                                         "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.smi = None

    def mark(self, name: str):
        self.marks[name] = time.perf_counter()

    def stop(self, gpu_index: int):
        if self.thread is not None:
            self.stop_ev.set()
            self.thread.join()
        elif self.smi is not None:
            self.smi.terminate()
            self.smi.wait()
            self.f.flush()
            self.f.seek(0)
            for line in self.f.read().splitlines():
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 5 or not parts[0].isdigit() or int(parts[0]) != gpu_index:
                    continue
                try:
                    self.samples.append((0.0, float(parts[1]), float(parts[2]), float(parts[3]), int(parts[4], 16)))
                except ValueError:
                    continue
            os.unlink(self.f.name)
        else:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock source"], "samples": 0}
        sm = [x[1] for x in self.samples]
        bits = 0
        for x in self.samples:
            bits |= x[4]
        t0, t1 = self.marks.get("timed_start"), self.marks.get("timed_end")
        inside = [x[1] for x in self.samples if t0 is not None and t1 is not None and t0 <= x[0] <= t1]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(x[2] for x in self.samples) if self.samples else None,
                "reasons": sorted(nm for nm, b in self.REASONS if bits & b),
                "samples": len(sm), "source": self.source, "period_ms": self.period * 1e3,
                "power_w_max": max(x[3] for x in self.samples) if self.samples else None,
                "samples_in_timed_region": len(inside),
                "sm_mhz_timed_region": statistics.median(inside) if inside else None,
                "window": "warm-up, the timed steps, the stage-timing and e2e loops",
                **({"nvml_error": self.nvml_error} if self.nvml_error else {})}


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


def parse_tiling(spec: str):
    """'WxH[/depth/bwd_threads]' -> (tile_w, tile_h, batch_depth, bwd_threads)."""
    parts = spec.split("/")
    tw, th = (int(x) for x in parts[0].split("x"))
    rest = [int(x) for x in parts[1:]] + [0, 0]
    return (tw, th, rest[0], rest[1])


def label(tile) -> str:
    from paper_2311_16728_b300.autotune import label as _label
    return _label(tuple(tile) + (0,) * (4 - len(tile)))


def _window_setup(args):
    """The window workload (setup, untimed): targets rendered from the true
    map, the perturbed map in the store order --order names, the tile shape
    chosen by the autotuner (or --tile), the window captured as one graph."""
    import torch
    import synthetic as S
    import paper_2311_16728_b300 as gsr
    from paper_2311_16728_b300.autotune import autotune_window
    from paper_2311_16728_b300.batched import BatchedWindow
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
        tile = parse_tiling(args.tile)
        report = {"ms_per_step": {}, "chosen": label(tile)}
    bw = BatchedWindow(params, kf, levels=WIN_LEVELS, tiling=gsr.tiling_struct(*tile))
    bw.capture()
    return bw, tile, report, kf, params


def window_figure(args, steps: int = 200):
    """The window's throughput for the headline line: `steps` whole-iteration
    graph replays timed by CUDA events after a warm-up."""
    import torch
    bw, tile, report, _, _ = _window_setup(args)
    for _ in range(max(args.warmup, 3)):
        bw.step()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    for _ in range(steps):
        bw.step()
    t1.record()
    torch.cuda.synchronize()
    if bw.status.item() != 0:
        raise RuntimeError(f"window: device status {bw.status.item():#x}")
    ms = t0.elapsed_time(t1) / steps
    return {"workload": f"{WIN_N // 1000}k Gaussians, {WIN_KF} keyframes 640x480 x {WIN_LEVELS} levels = {bw.V} "
                        "views, one persistent launch per iteration, whole iteration in one CUDA graph",
            "iters_per_s": 1000.0 / ms, "views_per_s": bw.V * 1000.0 / ms, "ms_per_step": ms, "steps": steps,
            "tiling": label(tile), "autotune": report.get("chosen"),
            "autotune_candidates": len(report.get("ms_per_step", {}))}


def run_window(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import paper_2311_16728_b300 as gsr
    bw, tile, report, kf, params = _window_setup(args)
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
    mhz, mhz_src = _fp32_clock(clk, peaks)
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
                                   "CUDA graph", "tiling": label(tile) + (" (autotuned)" if args.tile == "auto" else " (given)"),
                       "autotune_ms": report["ms_per_step"], "pairs": int(bw.num_pairs.item()),
                       "map_order": args.order,
                       "l2": "inputs larger than L2 (4 x 120 MB of params, grads, moments per step)"},
            "roofline": {"kernel": "batched_iterate_kernel (fwd + bwd blends)", "bound": "alu",
                         "achieved": flops / it_s / 1e12, "peak": fp32, "unit": "TFLOP/s",
                         "frac": flops / it_s / 1e12 / fp32,
                         "traffic": NCU_TRAFFIC_WINDOW_ITERATE if (tuple(tile) == (16, 16, 0, 0) and args.order == "morton") else None,
                         "alg_per_launch": flops,
                         "alg_rule": f"({FLOPS_PER_BLEND_FWD} + {FLOPS_PER_BLEND_BWD}) FP32 per (pixel, Gaussian) "
                                     "evaluation x blends over all views",
                         "peak_source": f"FP32 148 SMs x 128 lanes x 2 flops x {mhz:.0f} MHz, {mhz_src}"},
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


TTP_SMOOTH = 3  # evaluations in the running mean that decides a crossing


def _smoothed_reached(curve, target, k=TTP_SMOOTH):
    """Whether the mean PSNR of the last k evaluations (fewer at the start
    only once the run has ended) has reached `target`."""
    tail = [ps for _, _, ps in curve[-k:]]
    return len(tail) == k and statistics.mean(tail) >= target


def _ttp_run(kind, truth, keyframes, kps, offsets, init, li, budget, target, every, gsr, torch, levels=3):
    """One arm: fresh map = truth with the held-out primitives initialised by
    `init`; iterate until the running mean of the last TTP_SMOOTH evaluations
    reaches `target` PSNR (if given) or for `budget` iterations.  Returns the
    PSNR curve [(iterations, training ms, PSNR)]."""
    from paper_2311_16728_b300.batched import BatchedWindow
    from paper_2311_16728_b300.mapping import Evaluator, PlainMapper, densify_default, densify_learned
    params = gsr.Gaussians.from_arrays(truth.mean_op, truth.quat, truth.logscale, truth.sh)
    if init == "learned":
        densify_learned(li, params, keyframes, kps, offsets)
    else:
        densify_default(params, keyframes, kps, offsets)
    ev = Evaluator(TTP_N, keyframes)
    mapper = PlainMapper(params, keyframes, levels=levels) if kind == "plain" else BatchedWindow(params, keyframes)
    mapper.capture()
    curve = [(0, 0.0, ev(params))]
    it, wall = 0, 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    while it < budget and not (target is not None and _smoothed_reached(curve, target)):
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


def _first_at(curve, target, k=TTP_SMOOTH):
    """(iterations, training ms) at the first evaluation where the running
    mean of the last k evaluations reaches `target`, or (None, None)."""
    for i in range(k - 1, len(curve)):
        if statistics.mean(ps for _, _, ps in curve[i - k + 1:i + 1]) >= target:
            return curve[i][0], curve[i][1]
    return None, None


def ttp_experiment(eval_seeds, train_seeds=TTP_TRAIN_SEEDS, harvest_iters=TTP_HARVEST_ITERS,
                   mlp_steps=TTP_MLP_STEPS, budget=TTP_BUDGET, ablation_levels=()):
    """Time to PSNR (the second half of the headline metric).  The learned
    initialiser is trained inside the run, on the GPU, from (patch, converged
    parameter) pairs harvested from window runs on the training scenes; then
    on every held-out scene the plain path (single view, sequential pyramid
    schedule, default initialisation) runs `budget` iterations and fixes the
    target PSNR (the mean of its last TTP_SMOOTH evaluations), and the
    batched window with the learned and with the default initialisation run
    until the running mean of their evaluations reaches it.  With
    `ablation_levels`, the plain path also runs the same budget with each of
    those pyramid level counts (the 3-level run is the target's) on the same
    scenes: the Gaussian-pyramid ablation.  Returns (per-seed results,
    training summary)."""
    import torch
    import paper_2311_16728_b300 as gsr
    from paper_2311_16728_b300.batched import BatchedWindow
    from paper_2311_16728_b300.learned_init import LearnedInit, init_weights
    from paper_2311_16728_b300.mapping import densify_default, harvest, train_initialiser
    t0 = time.time()
    li = LearnedInit(init_weights(3), TTP_NEW, lr=1e-3)  # batches of up to one keyframe's new primitives
    batches = []
    for seed in train_seeds:
        truth, keyframes, kps, offsets = _ttp_setup(seed, gsr, torch)
        params = gsr.Gaussians.from_arrays(truth.mean_op, truth.quat, truth.logscale, truth.sh)
        densify_default(params, keyframes, kps, offsets)
        initial = gsr.Gaussians(*(t.clone() for t in params.tensors()), params.sh_degree)
        bw = BatchedWindow(params, keyframes)
        bw.capture()
        for _ in range(harvest_iters):
            bw.step()
        torch.cuda.synchronize()
        batches += harvest(li, params, initial, keyframes, kps, offsets)
        del bw, params, initial
    losses = train_initialiser(li, batches, mlp_steps)
    training = {"train_seeds": list(train_seeds), "harvest": f"{harvest_iters} window iterations per training "
                f"scene, {sum(b.M for b in batches)} pairs", "mlp_steps": mlp_steps,
                "mlp_loss_first_last": [losses[0], losses[-1]] if losses else None,
                "setup_s": round(time.time() - t0, 1)}
    per_seed = []
    for seed in eval_seeds:
        truth, keyframes, kps, offsets = _ttp_setup(seed, gsr, torch)
        plain = _ttp_run("plain", truth, keyframes, kps, offsets, "default", li, budget, None, 100, gsr, torch)
        target = statistics.mean(ps for _, _, ps in plain[-TTP_SMOOTH:])
        res = {"seed": seed, "target_psnr": target, "plain": {"curve": plain},
               "new": sum(int(k.shape[0]) for k in kps)}
        res["plain"]["iters"], res["plain"]["ms"] = _first_at(plain, target)
        for name, init in (("window_learned", "learned"), ("window_default", "default")):
            c = _ttp_run("window", truth, keyframes, kps, offsets, init, li, TTP_WINDOW_MAX, target, 10, gsr, torch)
            it, ms = _first_at(c, target)
            res[name] = {"curve": c, "iters": it, "ms": ms, "psnr0": c[0][2]}
        res["plain"]["psnr0"] = plain[0][2]
        res["levels"] = {3: plain}
        for L in ablation_levels:
            if L != 3:
                res["levels"][L] = _ttp_run("plain", truth, keyframes, kps, offsets, "default", li, budget, None, 100,
                                            gsr, torch, levels=L)
        per_seed.append(res)
    return per_seed, training


def gp_ablation_summary(per_seed, checkpoints=(400, TTP_BUDGET)) -> dict:
    """PSNR of the plain path after each checkpoint's iterations with n + 1
    pyramid levels (mean over the scenes, and per scene), and the training
    time to it: the replica of the paper's Tab. 4 rows."""
    out = {}
    levels = sorted(set().union(*(r["levels"].keys() for r in per_seed)))
    for L in levels:
        row = {}
        for c in checkpoints:
            pts = [next(pt for pt in r["levels"][L] if pt[0] >= c) for r in per_seed if L in r["levels"]]
            row[str(c)] = {"psnr_mean": statistics.mean(p[2] for p in pts), "psnr": [p[2] for p in pts],
                           "ms_mean": statistics.mean(p[1] for p in pts)}
        out[f"n={L - 1}"] = row
    return out


def ttp_summary(per_seed) -> dict:
    """Per-seed iterations and training time to the target PSNR, and the
    speed-ups (plain ms / window ms) with their spread across seeds."""
    def spread(xs):
        return {"mean": statistics.mean(xs), "min": min(xs), "max": max(xs)} if xs else None

    sp_l = [r["plain"]["ms"] / r["window_learned"]["ms"] for r in per_seed
            if r["window_learned"]["ms"] and r["plain"]["ms"]]
    sp_d = [r["plain"]["ms"] / r["window_default"]["ms"] for r in per_seed
            if r["window_default"]["ms"] and r["plain"]["ms"]]
    seeds = [{"seed": r["seed"], "new_primitives": r["new"], "target_psnr": r["target_psnr"],
              "plain": {"iters": r["plain"]["iters"], "ms": r["plain"]["ms"]},
              "learned_window": {"iters": r["window_learned"]["iters"], "ms": r["window_learned"]["ms"]},
              "default_window": {"iters": r["window_default"]["iters"], "ms": r["window_default"]["ms"]},
              "psnr0": {"default": r["plain"]["psnr0"], "learned": r["window_learned"]["psnr0"]}}
             for r in per_seed]
    return {"speedup_learned_window": spread(sp_l), "speedup_default_window": spread(sp_d), "per_seed": seeds}


TTP_WORKLOAD = (f"{TTP_N} Gaussians in a 6x3x4 m room, {TTP_KF} keyframes 640x480 fx=fy=525, every Gaussian whose "
                f"centre a keyframe sees (at most {TTP_NEW} per keyframe) re-created at its keypoint (known depth, "
                "unknown shape, opacity and colour); target = the plain path's PSNR (default init, sequential pyramid, "
                f"tau_u 30; mean of its last {TTP_SMOOTH} evaluations) after {TTP_BUDGET} iterations; an arm reaches "
                f"it when the mean of its last {TTP_SMOOTH} evaluations does; time = CUDA-event time of the training "
                "iterations (evaluation excluded)")


def run_ttp(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    seeds = [int(x) for x in args.ttp_seeds.split(",") if x]
    per_seed, training = ttp_experiment(seeds)
    summ = ttp_summary(per_seed)
    sl = summ["speedup_learned_window"]
    line = {"metric": "time-to-PSNR speed-up, learned initialiser + batched window vs plain single-view path",
            "value": sl["mean"] if sl else None, "unit": "x (plain ms / learned+batched ms)",
            "n_gpus": 1, "higher_is_better": True, "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded; held-out scenes)",
            "config": {"workload": TTP_WORKLOAD, "eval_seeds": seeds, **training},
            **summ, "curves": {str(r["seed"]): {k: r[k]["curve"] for k in ("plain", "window_learned",
                                                                         "window_default")}
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
    ap.add_argument("--ref-rows", type=int, default=0,
                    help="image rows per oracle step (reference arm; default: bands that tile the frame over --steps)")
    ap.add_argument("--cpu-rows", type=int, default=680, help="image rows of the cpu_baseline sample")
    ap.add_argument("--mode", default="mapping",
                    choices=["mapping", "window", "mlp", "ttp", "densify", "stereo", "gp_ablation", "pose"])
    ap.add_argument("--ttp-seeds", default="100,101,102,103,104", help="ttp mode: held-out evaluation scenes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="mapping mode: leave out the window figure and the bounded time-to-PSNR run")
    ap.add_argument("--headline-ttp-seeds", default="100,101",
                    help="mapping mode: held-out scenes of the bounded time-to-PSNR run in the headline line")
    ap.add_argument("--tile", default="auto",
                    help="mapping and window modes: WxH[/batch_depth/bwd_threads] instead of the autotuner's choice")
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
    tiling = gsr.tiling_struct(16, 16)  # the targets' renders (the image does not depend on the tiling)
    vb = gsr.ViewBuffers(N_GAUSS, gsr.camera_from(cams[0]), tiling, 1024)
    gts = []
    for cam in cams:
        vb.cam = gsr.camera_from(cam)
        gsr.ensure_capacity(vb, g_tgt)
        vb.forward(g_tgt)
        gts.append(vb.img.clone())
    del vb, g_tgt
    params = _ordered(gsr, gsr.Gaussians.from_arrays(start.mean_op, start.quat, start.logscale, start.sh), args)
    # tile shape, staging batch depth and backward threads per tile: the
    # autotuner's choice on the first poses (setup, untimed), or --tile
    if args.tile == "auto":
        from paper_2311_16728_b300.autotune import autotune
        tile, tune = autotune(params, list(zip(cams, gts))[:4], steps=8, warmup=2)
    else:
        tile, tune = parse_tiling(args.tile), None
    tiling = gsr.tiling_struct(*tile)
    ms = gsr.MappingStep(params, list(zip(cams, gts)), tiling)
    ms.capture()
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        ms.step()
    torch.cuda.synchronize()
    if args.profile:
        clocks.stop(local)
        _profile_steps(ms.step, args.steps)
        return
    if world > 1:
        dist.barrier()

    # ---- timed region: K whole iterations, one graph replay each
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clocks.mark("timed_start")
    t_start.record()
    for k in range(args.steps):
        ms.step()
    t_end.record()
    torch.cuda.synchronize()
    clocks.mark("timed_end")
    if world > 1:
        dist.barrier()
    ms_total = t_start.elapsed_time(t_end)
    # ---- stage times: the same iterations replayed one graph per stage,
    # events between the stages (live, on the launching stream)
    nst = len(gsr.STAGES)
    k_st = min(max(args.steps, 50), 300)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nst + 1)] for _ in range(k_st)]
    for k in range(k_st):
        ms.step(events=evs[k])
    torch.cuda.synchronize()
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
    clk = clocks.stop(local)
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
    # store with 16x16 tiles at the default staging (warp-private) and the
    # four-pixel backward; other configurations report none
    traffic = NCU_TRAFFIC if (args.scene == "room" and args.order == "morton" and
                              tuple(tile[:2]) == (16, 16) and tile[2] == 0 and tile[3] in (0, 64)) else {}
    stages = stage_rooflines(stage_ms, work, peaks, clk, traffic,
                             bwd_kernel=("render_bwd_warp_kernel" if tile[2] == 0 else "render_bwd_q4_kernel")
                             if (tuple(tile[:2]) == (16, 16) and tile[3] != 128) else "render_bwd_kernel",
                             fwd_kernel="render_fwd_warp_kernel" if (tuple(tile[:2]) == (16, 16) and tile[2] == 0)
                             else "render_fwd_kernel")
    dom = max(stage_ms, key=stage_ms.get)
    roof = dict(stages[dom])

    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; Replica-shaped)",
            "config": _config({"pairs_last_step": pairs, "poses": len(cams), "scene": args.scene,
                               "map_order": args.order,
                               "tile": label(tile) + (" (autotuned)" if tune else " (given)"),
                               **({"autotune": {"candidates": len(tune["ms_per_step"]),
                                                "ms_per_step_best": min(tune["ms_per_step"].values()),
                                                "ms_per_step_default": tune["ms_per_step"].get(
                                                    label((16, 16, 0, 0)))}} if tune else {}),
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
    if world == 1 and not args.no_extras and args.scene == "room":
        # the rest of the headline metric, after the throughput figure: the
        # batched window's rate and a bounded time-to-PSNR run (the learned
        # initialiser trained on the GPU inside this run, two held-out scenes)
        del ms, params
        torch.cuda.empty_cache()
        t_x = time.time()
        line["window"] = window_figure(args)
        seeds = [int(x) for x in args.headline_ttp_seeds.split(",") if x]
        per_seed, training = ttp_experiment(seeds, ablation_levels=(1, 2, 4))
        line["ttp"] = {"workload": TTP_WORKLOAD, "eval_seeds": seeds, **training, **ttp_summary(per_seed)}
        line["gp_ablation"] = {
            "workload": "the time-to-PSNR scenes above, default initialisation, plain path (one view per iteration, "
                        "tau_u 30) with n + 1 pyramid levels (n = 0: no pyramid); PSNR over the keyframes after 400 "
                        f"and {TTP_BUDGET} iterations (Tab. 4 replica)",
            "levels": gp_ablation_summary(per_seed)}
        line["extras_s"] = round(time.time() - t_x, 1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# DRAM bytes (read + write) per launch from one ncu capture of this workload
# with the current kernels (profiles/mapping_kernels_300k_1200x680.md; the
# loss stage is its two SSIM passes, the binning stage its seven kernels, the
# backward stage its tile reorder and blend, the Adam stage its step and
# counter kernels).
NCU_TRAFFIC = {"preprocess": 15.461e6, "bin_sort": 21.099e6, "render_fwd": 3.996e6, "loss": 69.038e6,
               "blend_bwd": 21.062e6, "preprocess_bwd": 12.438e6, "adam": 393.483e6}
# the pose chain (profiles/pose_bwd_300k_1200x680.md)
NCU_TRAFFIC_POSE = 15.037952e6
# the persistent window kernel (profiles/window_kernels_500k_8x640x480x3.md)
NCU_TRAFFIC_WINDOW_ITERATE = 597.588e6

# Algorithmic work per unit (the hot-path scope table's measurement figures;
# the implementation's own DRAM bytes are the ncu `traffic` above, never the
# algorithmic figure): FP32 operations per (pixel, Gaussian) evaluation in the
# forward and backward blends.
FLOPS_PER_BLEND_FWD = 16
FLOPS_PER_BLEND_BWD = 55


def _fp32_clock(clk, peaks):
    """SM clock for the FP32 peak and where it came from."""
    if clk.get("sm_mhz"):
        return clk["sm_mhz"], f"median SM clock sampled during the run ({clk.get('source')})"
    if "sm_max_mhz" in peaks:
        return peaks["sm_max_mhz"], "MEASURED_PEAKS.json sm_max_mhz (no clock samples)"
    return 2032.0, "nominal maximum 2032 MHz (no clock samples, no MEASURED_PEAKS.json)"


def sort_passes(tiles: int) -> int:
    """8-bit radix passes of a global LSD sort on 32 depth bits + ceil(log2 T) tile bits."""
    return -(-(32 + max(1, (tiles - 1).bit_length())) // 8)


def stage_rooflines(stage_ms, work, peaks, clk, traffic, tiles=None, bwd_kernel="render_bwd_warp_kernel",
                    fwd_kernel="render_fwd_warp_kernel"):
    """Roofline entry of each stage's dominant kernel: algorithmic work per
    launch (per-unit figure x the units of one launch) / measured stage time,
    against the measured HBM copy bandwidth or the FP32 peak (148 SMs x 128
    lanes x 2 flops x SM clock, the clock sampled during the run when there
    are samples, else MEASURED_PEAKS.json's maximum)."""
    hbm = peaks.get("hbm_gbs", 6400.0)
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6400 GB/s (of fallback)"
    mhz, mhz_src = _fp32_clock(clk, peaks)
    fp32 = 148 * 128 * 2 * mhz * 1e6 / 1e12
    n, nv, K, E = N_GAUSS, work["visible"], work["pairs"], work["blends"]
    T = tiles if tiles is not None else -(-WIDTH // 16) * -(-HEIGHT // 16)
    px = 3 * WIDTH * HEIGHT

    def hbm_entry(kernel, alg, rule):
        sec = stage_ms[st] * 1e-3
        return {"kernel": kernel, "bound": "hbm", "achieved": alg / sec / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": alg / sec / 1e9 / hbm, "traffic": traffic.get(st), "alg_per_launch": alg, "alg_rule": rule,
                "peak_source": hbm_src}

    def alu_entry(kernel, flops, rule):
        sec = stage_ms[st] * 1e-3
        return {"kernel": kernel, "bound": "alu", "achieved": flops / sec / 1e12, "peak": fp32, "unit": "TFLOP/s",
                "frac": flops / sec / 1e12 / fp32, "traffic": traffic.get(st), "alg_per_launch": flops,
                "alg_rule": rule, "peak_source": f"FP32 148 SMs x 128 lanes x 2 flops x {mhz:.0f} MHz, {mhz_src}"}

    out = {}
    for st in stage_ms:
        if st == "preprocess":
            out[st] = hbm_entry("preprocess_fwd_kernel", 12 * n + (228 + 48) * nv,
                                "12 B per Gaussian (cull read) + 228 B read + 48 B written per visible")
        elif st == "bin_sort":
            P = sort_passes(T)
            out[st] = hbm_entry("binning + per-tile sorts", 12 * K + 4 * n + 24 * P * K + 8 * K,
                                f"keys + values 12 B per pair + scan 4 B per Gaussian + {P} radix passes x 24 B per "
                                f"pair (32 depth + ceil(log2 {T}) tile bits) + ranges 8 B per pair")
        elif st == "render_fwd":
            out[st] = alu_entry(fwd_kernel, FLOPS_PER_BLEND_FWD * E,
                                f"{FLOPS_PER_BLEND_FWD} FP32 per (pixel, Gaussian) evaluation x blends")
        elif st == "loss":
            out[st] = hbm_entry("ssim kernels", 12 * px,
                                "rendered + target read (2 x 4 B) and dL/dI written (4 B) per pixel-channel")
        elif st == "blend_bwd":
            out[st] = alu_entry(bwd_kernel, FLOPS_PER_BLEND_BWD * E,
                                f"{FLOPS_PER_BLEND_BWD} FP32 per (pixel, Gaussian) evaluation x blends")
        elif st == "preprocess_bwd":
            out[st] = hbm_entry("preprocess_bwd_kernel", (236 + 236) * nv,
                                "236 B read + 236 B written per visible Gaussian")
        elif st == "adam":
            # 59 parameters: p, m, v read and written for every Gaussian; the
            # gradient read and zeroed only where a view flag (4 B) says the
            # view saw the Gaussian (an unseen Gaussian's gradient is zero)
            out[st] = hbm_entry("adam_kernel", 59 * 4 * 6 * n + 4 * n + 59 * 4 * 2 * nv,
                                "59 parameters x (p, m, v read + written) per Gaussian + view flag 4 B + gradient "
                                "read + zeroed per visible Gaussian (the dense step's 32 B per parameter less the "
                                "unseen Gaussians' zero gradients)")
    return out


if __name__ == "__main__":
    main()
