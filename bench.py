"""Benchmark of the neural path tracer's hot path on GB300.

A step is one full frame rendered through the C ABI: camera rays,
traversal, bounce sampling, NIF shading of every escape (BF16 tensor-core
kernel by default) and the sample reduction.  The default workload is the
spheres + HDR-NIF scene (256 spheres, 512x512 pixels, 64 samples per pixel,
depth 8: 16.8M paths per frame) whose environment NIF is first trained on the
procedural 2048x1024 sky with pt_train_nif.  The same line reports the
FP32-network frame rate and the relative RMSE between the BF16 and FP32
frames.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32|fp8]
                  [--workload C1|C2|C3|C4|C5]

Workload C5 (neural radiance cache on the heightfield scene): a step is one
frame of the online loop, i.e. one pt_train_cache step on 2^16 training
paths plus the 1024x1024, 4 spp render whose paths end in the cache at
vertex 2.  The line adds the plain full-depth FP32 and BF16 frame times and
the cache's bias against a plain 4096-spp FP32 reference.
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

Multi-GPU (torchrun, one rank per GPU): each rank renders its own disjoint
sample range of the frame (Philox counters first_sample = rank * spp), with
no data-path collective; value = all ranks' paths / max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2305_20061_gb300 import inputs as I  # noqa: E402
from paper_2305_20061_gb300 import replicas as R  # noqa: E402

METRIC = "Msamples/s & NIF evals/s at 1 GB300; BF16-TC vs FP32 at stated image RMSE"
UNIT = "Msamples/s"
FLOP_PER_EVAL = 2 * (3 * 128 * 128 + 128 * 3)   # 99,072: three 128x128 layers + 128->3 head
TC_FLOP_PER_EVAL = 2 * 3 * 128 * 128            # 98,304 in the three hidden layers
SM_COUNT = 152
FP32_LANES_PER_SM = 128
# Algorithmic FP32 FLOPs of the traversal's tests: a slab test of one child box is 12 (six plane distances,
# each a subtraction and a multiplication), a node fetch tests both children (24); a sphere test 20; an
# axis-aligned quad 10; the watertight triangle test 41 (9 vertex differences, 12 for the shear, 9 for the
# three edge functions, 2 for the determinant, 8 for the scaled distance, 1 division).
FLOP_NODE, FLOP_SPHERE, FLOP_QUAD, FLOP_TRI = 24, 20, 10, 41
# FP32 instructions per traversal step as implemented (node step of both children, sphere, quad and
# triangle tests), for the secondary issue-rate fraction
OPS_NODE, OPS_SPHERE, OPS_QUAD, OPS_TRI = 58, 36, 12, 46
# algorithmic bytes per traversal step (a node fetch reads both children's boxes and references) and per ray of
# the traversal kernel (origin and direction in, hit out)
BYTES_NODE, BYTES_SPHERE, BYTES_QUAD, BYTES_TRI, BYTES_RAY_TRACE = 48, 16, 32, 48, 40


def shade_bytes(counts, depth: int, emits: bool) -> int:
    """Queue bytes of the shading kernel over a frame, from the rays traced per vertex (counts[:depth]) and the
    escapes (counts[depth]): a camera ray's 8-byte hit; a later ray's origin, direction and throughput (48 B) and
    hit (8 B) read; every later ray was written once as a survivor (48 B), and with emitters its radiance (16 B)
    is written and read too; each escape a 24-byte record."""
    cam, later, esc = int(counts[0]), int(sum(counts[1:depth])), int(counts[depth])
    return 8 * cam + (56 + 48 + (32 if emits else 0)) * later + 24 * esc
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes (read + write) of the traversal kernel per traced ray, from one ncu capture of the workload's frame
# (or a smaller frame of it) (summaries and commands in profiles/), scaled to a frame by the rays it traces.  Valid only
# while the traversal source and the BVH builder are the ones captured (sha256 of trace.cu + device_common.cuh +
# bvh_build.cpp, first 16 hex digits): the bytes depend on the kernel and on the tree it walks.
TRACE_TRAFFIC = {
    # 1920x1080 at 8 spp = one full 2^24-path chunk of the 32-spp frame (profiles/k_trace_traffic_large_bvh_c4.md)
    ("C4", "packed"): {"bytes_per_ray": 366.0, "src": "b595122a4af8ee56"},
    ("C4", "quant8"): {"bytes_per_ray": 284.6, "src": "b595122a4af8ee56"},
    # 512x512 at 64 spp, the full frame, one pass per launch (profiles/k_trace_traffic_spheres_c2.md)
    ("C2", "decoded"): {"bytes_per_ray": 22.69, "src": "b595122a4af8ee56"},
}
# L2 bytes (lts__t_bytes) of the traversal kernel per traced ray on the large tree, from the same captures
TRACE_L2 = {
    ("C4", "packed"): {"bytes_per_ray": 1641.9, "src": "b595122a4af8ee56"},
    ("C4", "quant8"): {"bytes_per_ray": 1279.1, "src": "b595122a4af8ee56"},
}
NODE_FORMS = {1: "packed", 2: "decoded", 3: "quant8"}
TRACE_SOURCES = ("paper_2305_20061_gb300/csrc/trace.cu", "paper_2305_20061_gb300/csrc/device_common.cuh",
                 "paper_2305_20061_gb300/csrc/bvh_build.cpp")


def trace_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in TRACE_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def trace_l2_bytes(workload: str, node_form: str, rays: int):
    """L2 bytes of the traversal kernel over a frame of `rays` traced rays, or None (as trace_traffic)."""
    rec = TRACE_L2.get((workload, node_form))
    if rec is None or rec["src"] != trace_source_hash():
        return None
    return rec["bytes_per_ray"] * rays


def trace_traffic(workload: str, node_form: str, rays: int):
    """DRAM bytes of the traversal kernel over a frame of `rays` traced rays, or None when no capture of
    this workload and node form exists or the traversal source or the BVH builder changed since it was taken."""
    rec = TRACE_TRAFFIC.get((workload, node_form))
    if rec is None or rec["src"] != trace_source_hash():
        return None
    return rec["bytes_per_ray"] * rays


def peaks():
    try:
        with open(MEASURED) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(sm)}


def workload(name, spp=None, depth=None, rr=False):
    sc = I.make_scene(name)
    cfg = I.CONFIGS[name]["cfg"]
    if spp:  # smaller case for profiler captures only
        cfg = I.RenderCfg(cfg.width, cfg.height, spp, cfg.max_depth, cfg.seed)
    if depth or rr:  # the paper's perf mode: path length 10, Russian roulette from depth 3 (Section 3.1)
        cfg = I.RenderCfg(cfg.width, cfg.height, cfg.spp, depth or cfg.max_depth, cfg.seed, rr=bool(rr), rr_start=3)
    nif = I.nif_init(colour="identity" if name == "C1" else "yuv") if sc.env_const is None else None
    return sc, cfg, nif


def config_dict(name, cfg):
    """The workload of a line (the same for the GPU arm and the oracle arm; no model keys)."""
    rr = f"Russian roulette from depth {cfg.rr_start}" if cfg.rr else "no RR"
    return {"workload": f"{name}: {I.CONFIGS[name]['desc']}; rendered {cfg.width}x{cfg.height}, {cfg.spp} spp, "
                        f"max depth {cfg.max_depth}, {rr}",
            "paths_per_frame": cfg.n_slots,
            "l2": "per-step working set > L2 (wavefront queues ~2.7 GB per 2^24 paths) and a 512 MB L2 flush between "
                  "timed steps (outside the timed events)"}


def nif_dict(precision, trained):
    """The environment network of a line."""
    return {"shape": "F=64 Gaussian Fourier (sigma 10) -> 3x FC-128 ReLU -> FC-3 -> colour matrix -> exp",
            "weights": ("trained by pt_train_nif on the procedural 2048x1024 sky" if trained else
                        "random init (the work per path does not depend on the weights: the environment's values "
                        "change no path's geometry)"),
            "precision": precision}


def c5_config(cfg):
    return {"workload": f"C5: {I.CONFIGS['C5']['desc']}; a step = one frame = pt_train_cache ({N_TRAIN} training "
                        f"paths, depth {cfg.max_depth}, records at vertex {CACHE_VERTEX}) + pt_render_cached "
                        f"({cfg.width}x{cfg.height}, {cfg.spp} spp, paths end in the cache at vertex {CACHE_VERTEX})",
            "paths_per_frame": cfg.n_slots,
            "l2": "512 MB L2 flush between timed frames (outside the timed events)"}


# ----------------------------------------------------------------------------
def oracle_rate(sc, cfg, nif, target_s: float, n_threads: int):
    """Oracle paths/s on a bounded pixel sample of the workload (all samples
    of every m-th pixel), sized to take about target_s seconds."""
    from oracle import oracle as O
    osc = O.Scene(sc)
    onif = O.Nif(nif) if nif is not None else None
    n_pix_total = cfg.width * cfg.height

    def run(n_pix):
        step = max(1, n_pix_total // n_pix)
        pixels = np.arange(0, n_pix_total, step, dtype=np.int64)[:n_pix]
        t0 = time.perf_counter()
        O.render(osc, cfg, onif, pixels=pixels, n_threads=n_threads)
        return len(pixels), time.perf_counter() - t0

    n, dt = run(max(8 * n_threads, 128))
    rate = n / max(dt, 1e-6)
    n_pix = int(min(n_pix_total, max(n_threads, rate * target_s)))
    return run, n_pix


def bench_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    sc, cfg, nif = workload(args.workload, args.spp, args.depth, args.rr)
    if args.workload == "C5":
        cache0 = I.cache_init(*I.scene_bounds(sc))
        vals = []
        for i in range(args.warmup + args.steps):
            v, sample = oracle_c5_rate(sc, nif, cache0, cfg, args.ref_step_s)
            if i >= args.warmup:
                vals.append(v)
        value = float(np.mean(vals))
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * cfg.n_slots / (value * 1e6),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": c5_config(cfg), "nif": nif_dict("fp64-oracle", False),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return 0
    threads = os.cpu_count() or 1
    run, n_pix = oracle_rate(sc, cfg, nif, target_s=args.ref_step_s, n_threads=threads)
    for _ in range(args.warmup):
        run(max(threads, n_pix // 8))
    total_paths, total_t = 0, 0.0
    for _ in range(args.steps):
        n, dt = run(n_pix)
        total_paths += n * cfg.spp
        total_t += dt
    value = total_paths / total_t / 1e6
    sample = f"all {cfg.spp} samples of {n_pix} evenly strided pixels of the {cfg.width}x{cfg.height} frame per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(args.workload, cfg),
        "nif": nif_dict("fp64-oracle", False) if nif else None,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


def trace_kernels(pt, ctx, vertices):
    """Name of the traversal kernel of the last render (profile kind
    "trace") and its launches per chunk: on the wavefront schedule one
    traversal launch per vertex, labelled k_trace (the camera rays of a
    whole image go through k_trace_camera, the warp-packet variant; shading,
    k_bounce, is timed apart), one k_paths launch (traversal and shading
    together) on the path-per-thread schedule."""
    if pt.last_render_schedule(ctx) == "paths":
        return "k_paths", 1
    return "k_trace", vertices


def traversal_roofline(work, t_ms, kernel, launches, ffma_tflops, clock, context):
    """Roofline of the traversal kernel over one frame: algorithmic FLOPs of
    its tests (FLOP_*) per frame / its device time per frame, against the
    FP32 FMA rate measured on this device; the issue-rate fraction of the
    implementation's own instruction counts rides along."""
    flop = (FLOP_NODE * work["nodes"] + FLOP_SPHERE * work["sphere"] + FLOP_QUAD * work["quad"] +
            FLOP_TRI * work["triangle"])
    achieved = flop / (t_ms * 1e-3) / 1e12
    ops = (OPS_NODE * work["nodes"] + OPS_SPHERE * work["sphere"] + OPS_QUAD * work["quad"] +
           OPS_TRI * work["triangle"])
    issue_peak = SM_COUNT * FP32_LANES_PER_SM * clock * 1e6 / 1e12
    return {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": ffma_tflops, "unit": "TFLOP/s",
            "frac": achieved / ffma_tflops, "traffic": None,
            "per_unit": f"FP32 FLOP per node fetch (two child slabs) {FLOP_NODE}, per sphere/quad/triangle test "
                        f"{FLOP_SPHERE}/{FLOP_QUAD}/{FLOP_TRI}; {work['nodes']} node fetches and "
                        f"{work['sphere']}/{work['quad']}/{work['triangle']} sphere/quad/triangle tests per frame "
                        f"over {launches} launches, {t_ms:.3f} ms of {kernel} per frame{context}"
                        + (" (k_trace_camera traces the camera rays of a whole image)" if kernel == "k_trace" else ""),
            "peak_note": "FP32 FMA rate measured live by pt_microbench_ffma (8 chains per thread, 2048 threads "
                         "per SM, CUDA events)",
            "issue_frac": ops * 1e-12 / (t_ms * 1e-3) / issue_peak,
            "issue_note": f"implementation's FP32 instructions per node/sphere/quad/triangle step {OPS_NODE}/"
                          f"{OPS_SPHERE}/{OPS_QUAD}/{OPS_TRI} over {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x "
                          f"{clock:.0f} MHz"}


def profiled_split(pt, ctx, run_frame, steps, n_prof=3):
    """Per-kernel-kind device time and launch counts of `steps` frames, from
    n_prof extra frames run with per-launch CUDA events (the library then
    launches directly instead of replaying its graphs), scaled to `steps`."""
    import torch
    n_prof = max(1, min(steps, n_prof))
    pt.profile_enable(ctx, True)
    pt.profile_read(ctx)
    for i in range(n_prof):
        run_frame(i)
    torch.cuda.synchronize()
    raw = pt.profile_read(ctx)
    pt.profile_enable(ctx, False)
    return {k: (v[0] * steps / n_prof, int(round(v[1] * steps / n_prof))) for k, v in raw.items()}


def nif_quality(gnif, sky, dev):
    """Trained-NIF quality against the HDR sky at all of its pixel centres:
    log-RMSE (natural log, per channel) and PSNR of the Reinhard-tonemapped
    x / (1 + x) images (peak 1), for FP32 and BF16 evaluation."""
    import torch
    h, w = sky.shape[0], sky.shape[1]
    jj, ii = torch.meshgrid(torch.arange(h, device=dev), torch.arange(w, device=dev), indexing="ij")
    uv = torch.stack([(ii.reshape(-1) + 0.5) / w, (jj.reshape(-1) + 0.5) / h], 1).float().contiguous()
    ref = sky.reshape(-1, 3).double()
    out = {"grid": f"{w}x{h} pixel centres"}
    for prec in ("fp32", "bf16"):
        try:
            y = gnif.eval(uv, prec).double()
        except RuntimeError:   # no BF16 kernel for this shape
            continue
        lr = torch.sqrt(torch.mean((torch.log(torch.clamp(y, min=1e-6)) - torch.log(torch.clamp(ref, min=1e-6))) ** 2))
        ty, tr = y / (1 + y), ref / (1 + ref)
        mse = torch.mean((ty - tr) ** 2)
        out[f"log_rmse_{prec}"] = float(lr)
        out[f"psnr_tonemapped_{prec}"] = float(10 * torch.log10(1.0 / mse))
        if prec == "fp32":   # luma / chroma split of the tonemapped error (BT.601 Y, U, V)
            wts = torch.tensor([0.299, 0.587, 0.114], dtype=torch.float64, device=ty.device)
            ly, lr_ = ty @ wts, tr @ wts
            uy = torch.stack([0.492 * (ty[:, 2] - ly), 0.877 * (ty[:, 0] - ly)], 1)
            ur = torch.stack([0.492 * (tr[:, 2] - lr_), 0.877 * (tr[:, 0] - lr_)], 1)
            out["psnr_luma_fp32"] = float(10 * torch.log10(1.0 / torch.mean((ly - lr_) ** 2)))
            out["psnr_chroma_fp32"] = float(10 * torch.log10(1.0 / torch.mean((uy - ur) ** 2)))
    return out


def train_env_nif(pt, ctx, gnif, nif, steps, dev, precision):
    """Train the environment NIF on the procedural 2048 x 1024 HDR sky (not
    timed as a frame) with the given GEMM precision; copies the trained
    weights back into `nif`."""
    import torch
    sky = torch.from_numpy(I.procedural_sky()).to(dev)
    batch = 1 << 16
    gnif.train(sky, steps=5, batch=batch, lr=1e-3, seed=0, precision=precision)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    losses = gnif.train(sky, steps=steps, batch=batch, lr=1e-3, seed=0, precision=precision)
    t1.record()
    torch.cuda.synchronize()
    ctx.check()
    tms = t0.elapsed_time(t1)
    train = {"steps": steps + 5, "batch": batch, "gemm_precision": precision, "ms_per_step": tms / steps,
             "samples_per_s": steps * batch / (tms * 1e-3),
             "fwd_bwd_tflops": steps * batch * 3 * FLOP_PER_EVAL / (tms * 1e-3) / 1e12,
             "loss_first": float(losses[0].item()), "loss_last": float(losses[-50:].mean().item())}
    train["quality"] = nif_quality(gnif, sky, dev)
    # what the network replaces: the sky as an FP32 texture, at the quality above
    n_par = 2 * nif.n_freq + sum(W.size + b.size for W, b in zip(nif.W, nif.b))
    train["vs_texture"] = {"texture_bytes": int(sky.numel() * 4), "nif_bytes_fp32": int(4 * n_par),
                           "nif_bytes_bf16": int(2 * n_par),
                           "compression_bf16": float(sky.numel() * 4 / (2 * n_par))}
    del sky
    params = gnif.get_params()
    p = 2 * nif.n_freq
    for W, b in zip(nif.W, nif.b):
        W[:] = params[p:p + W.size].reshape(W.shape)
        p += W.size
        b[:] = params[p:p + b.size]
        p += b.size
    return train


# ----------------------------------------------------------------------------
def bench_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt

    dev = f"cuda:{local}"
    sc, cfg, nif = workload(args.workload, args.spp, args.depth, args.rr)
    uses_nif = nif is not None
    precision = args.precision if uses_nif else None
    ctx = pt.Context(local)
    t_build = time.perf_counter()
    scene = pt.Scene(ctx, sc, node_format=args.nodes)
    t_build = time.perf_counter() - t_build
    gnif = pt.Nif(ctx, nif) if uses_nif else None

    # the environment NIF is trained on the procedural 2048 x 1024 HDR sky first (not timed as a frame)
    train = (train_env_nif(pt, ctx, gnif, nif, args.train_steps, dev, args.train_precision)
             if uses_nif and args.train_steps > 0 else None)
    img = torch.empty((cfg.height, cfg.width, 3), dtype=torch.float32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    first_sample = R.first_sample(rank, world, cfg.spp)
    rprec = precision or "fp32"

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_frames(prec, steps, profile=False):
        for _ in range(args.warmup):
            pt.render(ctx, scene, gnif, cfg, prec, out=img, first_sample=first_sample)
        ctx.check()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        k0 = pt.kernel_launches()
        for i in range(steps):
            flush.fill_(float(i))           # evict L2 between timed steps (not timed)
            ev[i][0].record(stream)
            pt.render(ctx, scene, gnif, cfg, prec, out=img, first_sample=first_sample)   # a CUDA-graph replay
            ev[i][1].record(stream)
        barrier()
        kernels = pt.kernel_launches() - k0
        ctx.check()
        ms = R.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / steps, dev)
        prof = profiled_split(pt, ctx, lambda i: pt.render(ctx, scene, gnif, cfg, prec, out=img,
                                                           first_sample=first_sample), steps) if profile else None
        return ms, prof, kernels

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ms, prof, kernels = timed_frames(rprec, args.steps, profile=True)
    clocks = sampler.stop()
    counts = pt.last_render_counts(ctx, cfg.max_depth)
    work = pt.last_render_work(ctx)
    trace_kernel, trace_launches = trace_kernels(pt, ctx, cfg.max_depth)
    paths = cfg.n_slots
    value = world * paths / (ms * 1e-3) / 1e6
    evals = int(counts[cfg.max_depth])
    rays = int(counts[:cfg.max_depth].sum())
    nif_ms = prof["nif"][0] / args.steps
    trace_ms = prof["trace"][0] / args.steps

    # the other precision on the same frame, and the image difference between them
    other = "fp32" if rprec != "fp32" else "bf16"
    lowp = rprec if rprec != "fp32" else "bf16"
    ms_other, rel_rmse = None, None
    if uses_nif and not args.no_compare:
        ms_other, _, _ = timed_frames(other, max(2, min(args.steps, 5)))
        a = pt.render(ctx, scene, gnif, cfg, lowp, first_sample=first_sample).double()
        b = pt.render(ctx, scene, gnif, cfg, "fp32", first_sample=first_sample).double()
        ctx.check()
        rel_rmse = float(torch.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()).item())

    # standalone NIF throughput: 2^24 uniform (u, v) through each kernel
    nif_alone = {}
    if uses_nif and not args.no_compare:
        uv = torch.from_numpy(I.uniform_uv(1 << 24, seed=1)).to(dev)
        for prec in ("bf16", "fp8", "fp32"):
            gnif.eval(uv, prec)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 3
            e0.record(stream)
            for _ in range(reps):
                gnif.eval(uv, prec)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / reps
            flop = TC_FLOP_PER_EVAL if prec != "fp32" else FLOP_PER_EVAL
            nif_alone[prec] = {"evals_per_s": (1 << 24) / (t * 1e-3), "ms": t,
                               "tflops": (1 << 24) * flop / (t * 1e-3) / 1e12}
        ctx.check()
        # the tensor-core kernels against the measured dense peak (FP8: twice the BF16 burst), the FP32 kernel
        # against the measured FFMA rate
        meas0, which0 = peaks()
        for prec, rec in nif_alone.items():
            peak0 = (pt.ffma_rate_tflops(local) if prec == "fp32" else
                     float(meas0["bf16_tflops"]) * (2.0 if prec == "fp8" else 1.0))
            rec.update({"frac_of_peak": rec["tflops"] / peak0, "peak_tflops": peak0,
                        "peak": "FP32 FMA rate (pt_microbench_ffma)" if prec == "fp32" else
                                f"dense BF16 cuBLAS burst ({which0})" + (" x 2" if prec == "fp8" else "")})

    # live roofline of the dominant kernel of the timed frames
    meas, which = peaks()
    clock = float(meas.get("sm_max_mhz", 2070.0))
    dom = max(("trace", "shade", "nif", "reduce"), key=lambda k: prof[k][0])
    big_scene = scene.info()["node_bytes"] > 128 * 1024 * 1024   # BVH larger than L2
    if dom == "nif" and rprec in ("bf16", "fp8"):
        peak = float(meas["bf16_tflops"]) * (2.0 if rprec == "fp8" else 1.0)
        achieved = evals * TC_FLOP_PER_EVAL / (nif_ms * 1e-3) / 1e12
        roof = {"kernel": "k_nif_tc" if rprec == "bf16" else "k_nif_fp8", "bound": "tensor", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "per_unit": f"{TC_FLOP_PER_EVAL} tensor FLOP per NIF evaluation x {evals} evaluations per launch",
                "peak_note": (f"dense BF16 cuBLAS burst ({which}; the NIF launches are timed in a region of well "
                              f"under a second)" if rprec == "bf16" else
                              f"dense FP8 = BF16 cuBLAS burst ({which}) x 2 (nominal 4.5 / 2.25 PFLOP/s)")}
    elif dom == "nif":
        peak = SM_COUNT * FP32_LANES_PER_SM * 2 * clock * 1e6 / 1e12
        achieved = evals * FLOP_PER_EVAL / (nif_ms * 1e-3) / 1e12
        roof = {"kernel": "k_nif_fp32", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "per_unit": f"{FLOP_PER_EVAL} FLOP per NIF evaluation x {evals} evaluations per launch",
                "peak_note": f"FP32 FFMA derived: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 x {clock:.0f} MHz"}
    elif big_scene and dom == "trace":
        nbytes = (BYTES_NODE * work["nodes"] + BYTES_SPHERE * work["sphere"] + BYTES_QUAD * work["quad"] +
                  BYTES_TRI * work["triangle"] + BYTES_RAY_TRACE * rays)
        peak = float(meas["hbm_gbs"])
        achieved = nbytes / (trace_ms * 1e-3) / 1e9
        roof = {"kernel": trace_kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None,
                "per_unit": f"bytes per node fetch {BYTES_NODE}, per sphere/quad/triangle test "
                            f"{BYTES_SPHERE}/{BYTES_QUAD}/{BYTES_TRI}, per ray {BYTES_RAY_TRACE} (origin and "
                            f"direction in, hit out); {work['nodes']} node fetches, {work['triangle']} triangle "
                            f"tests, {rays} rays per frame over {trace_launches} launches",
                "peak_note": f"HBM copy bandwidth ({which}); BVH {scene.info()['node_bytes'] / 2**20:.0f} MiB > L2"}
        l2b = trace_l2_bytes(args.workload, NODE_FORMS[scene.info()["node_format"]], rays)
        if l2b is not None:
            l2_peak = pt.l2_read_rate_gbs(local)
            l2_gbs = l2b / (trace_ms * 1e-3) / 1e9
            roof["l2"] = {"achieved": l2_gbs, "peak": l2_peak, "unit": "GB/s", "frac": l2_gbs / l2_peak,
                          "bytes": l2b, "note": "L2 bytes per frame (lts__t_bytes per traced ray from the ncu capture "
                                                "in profiles/, times the frame's rays) over k_trace's time, against "
                                                "the L2 read rate measured live by pt_microbench_l2_read"}
    elif dom == "shade":
        shade_ms = prof["shade"][0] / args.steps
        nbytes = shade_bytes(counts, cfg.max_depth, bool(scene.info()["has_emission"]))
        achieved = nbytes / (shade_ms * 1e-3) / 1e9
        peak = float(meas["hbm_gbs"])
        roof = {"kernel": "k_bounce", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None,
                "per_unit": f"8 B per camera-ray hit, 104 B per later ray (queue read and survivor write; +32 B with "
                            f"emitters), 24 B per escape: {nbytes} B over {rays} rays per frame",
                "peak_note": f"HBM copy bandwidth ({which})"}
    else:
        roof = traversal_roofline(work, trace_ms, trace_kernel, trace_launches, pt.ffma_rate_tflops(local), clock,
                                  "")

    if roof["kernel"] in ("k_trace", "k_paths"):
        roof["traffic"] = (trace_traffic(args.workload, NODE_FORMS[scene.info()["node_format"]], rays)
                           if trace_kernel == "k_trace" else None)
        roof["traffic_note"] = ("DRAM bytes per frame of the traversal launches (k_trace_camera at vertex 1 of a "
                                "whole image, k_trace at the others), from the ncu capture in profiles/ scaled by "
                                "traced rays; null when no capture of this workload matches the current traversal "
                                "and BVH-builder source")
    # end to end through the C ABI with host buffers: scene + weights in, image out
    e2e = None
    if not args.no_e2e:
        host_img = torch.empty((cfg.height, cfg.width, 3), dtype=torch.float32, pin_memory=True)
        scene_arrays = (sc.sphere, sc.sphere_mat, sc.quad, sc.quad_axis, sc.quad_mat, sc.vert, sc.tri, sc.tri_mat,
                        sc.mat_type, sc.mat)
        h2d = sum(x.nbytes for x in scene_arrays) + (pt.nif_flat(nif).nbytes if uses_nif else 0)
        d2h = host_img.numel() * 4
        n_e2e = max(3, min(args.steps, 10)) if not big_scene else 1

        def inputs():
            return pt.Scene(ctx, sc, node_format=args.nodes), (pt.Nif(ctx, nif) if uses_nif else None)

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nxt = inputs()
        for i in range(n_e2e):
            s2, n2 = nxt
            pt.render(ctx, s2, n2, cfg, rprec, out=img, first_sample=first_sample)
            host_img.copy_(img, non_blocking=True)
            # the next step's scene and weights are built and uploaded while the GPU renders this one
            nxt = inputs() if i + 1 < n_e2e else None
            torch.cuda.synchronize()
            del s2, n2
        dt = (time.perf_counter() - t0) / n_e2e
        e2e = {"value": world * paths / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "note": "per step: pt_create_scene (host BVH build) + pt_load_nif from host arrays, pt_render, "
                       "image copied to pinned host memory; step i+1's scene and weights are built and uploaded "
                       "(context upload stream) while the GPU renders step i"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        run, n_pix = oracle_rate(sc, cfg, nif, target_s=args.cpu_s, n_threads=threads)
        n, dt = run(n_pix)
        cpu = {"value": n * cfg.spp / dt / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"all {cfg.spp} samples of {n} evenly strided pixels ({n * cfg.spp} paths), FP64 oracle"}
        # the same oracle on one thread, on a sample of about a fifth of the time
        run1, n1 = oracle_rate(sc, cfg, nif, target_s=args.cpu_s / 5, n_threads=1)
        n1, dt1 = run1(n1)
        cpu["single_thread"] = {"value": n1 * cfg.spp / dt1 / 1e6, "cores": 1,
                                "sample": f"all {cfg.spp} samples of {n1} evenly strided pixels"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": rprec if uses_nif and rprec != "fp32" else "f32",
            "data": "synthetic (procedural scene" + (" and sky, NIF trained on the sky" if train else "") + "; seeds 0)",
            "config": config_dict(args.workload, cfg), "nif": nif_dict(precision, train is not None) if uses_nif else None,
            "rays_per_step": rays, "traversal_work_per_step": work,
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "scene_build_s": t_build, "bvh_nodes": scene.info()["n_nodes"], "bvh_depth": scene.info()["bvh_depth"],
            "bvh_node_form": {1: "packed 48 B", 2: "decoded 64 B", 3: "quantised 32 B"}[scene.info()["node_format"]],
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": int(kernels),
        }
        if uses_nif:
            line.update({
                f"{other}_value": world * paths / (ms_other * 1e-3) / 1e6 if ms_other else None,
                f"{lowp}_vs_fp32_image_rel_rmse": rel_rmse,
                "nif_evals_per_step": evals,
                "nif_evals_per_s_in_render": evals / (nif_ms * 1e-3) if nif_ms > 0 else None,
                "nif_standalone_2p24": nif_alone, "nif_training": train})
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0

# ----------------------------------------------------------------------------
CACHE_FLOP_PER_QUERY = 2 * (78 * 64 + 4 * 64 * 64 + 64 * 3)   # 43,136: 5 x FC-64 + FC-3 on 78 inputs
N_TRAIN = 1 << 16
CACHE_VERTEX = 2
C5_FRAMES = 60


def image_stats(X_batches, R_mean, R_var):
    """Relative RMSE of the mean of X_batches against R_mean, and the bias
    with both images' noise taken out: E[(X - R)^2] = bias^2 + var X + var R
    per pixel and channel (variances of the means from the batch spread)."""
    import torch
    nb = X_batches.shape[0]
    X = X_batches.mean(0)
    vX = X_batches.var(0) / nb
    den = (R_mean ** 2).sum()
    d2 = ((X - R_mean) ** 2).sum()
    b2 = float((d2 - vX.sum() - R_var.sum()) / den)
    H, W = R_mean.shape[0], R_mean.shape[1]

    def blk(Y):
        return Y.reshape(H // 8, 8, W // 8, 8, 3).mean((1, 3))
    return {"rel_rmse": float(torch.sqrt(d2 / den)), "bias_rel_rmse": float(np.sign(b2) * np.sqrt(abs(b2))),
            "noise_rel_rmse": float(torch.sqrt(vX.sum() / den)),
            "rel_rmse_8x8_blocks": float(torch.sqrt(((blk(X) - blk(R_mean)) ** 2).sum() / (blk(R_mean) ** 2).sum()))}


def oracle_c5_rate(sc, nif, cache, cfg, target_s):
    """Oracle frame rate of the cached loop on a bounded sample: cached render
    paths, plain training paths with vertex records and the relative-L2
    loss/gradient, each timed on a slice and scaled to one frame (2^16
    training samples + W*H*spp render paths).  Single-threaded."""
    from oracle import oracle as O
    osc, onif, oc = O.Scene(sc), O.Nif(nif), O.Cache(cache)
    n_pix = cfg.width * cfg.height

    def rate(fn, n0):
        n = n0
        while True:
            t0 = time.perf_counter()
            fn(n)
            dt = time.perf_counter() - t0
            if dt > target_s / 6 or n >= 1 << 20:
                return n / dt, n
            n *= 4

    def render_paths(n):
        pix = np.arange(n, dtype=np.int64) * 7919 % n_pix
        O.trace_paths(osc, sc.camera, cfg.width, cfg.height, cfg.max_depth, 0, pix, np.zeros(n, np.int64),
                      nif=onif, cache=oc, cache_vertex=CACHE_VERTEX)

    def train_paths(n):
        pix = np.arange(n, dtype=np.int64) * 104729 % n_pix
        L, rec, _ = O.trace_paths(osc, sc.camera, cfg.width, cfg.height, cfg.max_depth, 0, pix,
                                  np.full(n, 1 << 30, np.int64), nif=onif, rec_vertex=CACHE_VERTEX)
        ok = rec[:, 15] == 1
        tgt = np.zeros((n, 3))
        tgt[ok] = (L[ok] - rec[ok, 12:15]) / rec[ok, 9:12]
        oc.loss_grad(rec[:, :9], tgt, mask=ok.astype(np.int32))

    r_render, n_r = rate(render_paths, 256)
    r_train, n_t = rate(train_paths, 64)
    frame_s = cfg.n_slots / r_render + N_TRAIN / r_train
    return cfg.n_slots / frame_s / 1e6, (f"{n_r} cached render paths and {n_t} training paths (+ loss/gradient) timed, "
                                          f"scaled to one frame of {cfg.n_slots} render paths + {N_TRAIN} training "
                                          f"samples; FP64 oracle, single-threaded")


def bench_c5(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt

    dev = f"cuda:{local}"
    sc, cfg, nif = workload("C5", args.spp)
    prec = args.precision
    ctx = pt.Context(local)
    t_build = time.perf_counter()
    scene = pt.Scene(ctx, sc, node_format=args.nodes)
    t_build = time.perf_counter() - t_build
    gnif = pt.Nif(ctx, nif)
    train = train_env_nif(pt, ctx, gnif, nif, args.train_steps, dev, args.train_precision) if args.train_steps > 0 else None
    lo, hi = I.scene_bounds(sc)
    cache0 = I.cache_init(lo, hi)
    gc = pt.Cache(ctx, cache0)
    W, H, spp = cfg.width, cfg.height, cfg.spp
    img = torch.empty((W * H, 3), dtype=torch.float32, device=dev)
    img_plain = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    losses = torch.zeros(max(C5_FRAMES, args.warmup + args.steps), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def frame(f):
        # each rank runs its own online loop on its own samples (replicas, no collective)
        gc.train_frame(scene, gnif, W, H, f * world + rank, n_train=N_TRAIN, max_depth=cfg.max_depth,
                       rec_vertex=CACHE_VERTEX, seed=0, precision=prec, loss=losses[f:f + 1],
                       train_precision=args.train_precision)
        pt.render_cached(ctx, scene, gnif, cfg, None, cache=gc, cache_vertex=CACHE_VERTEX, precision=prec,
                         first_sample=R.first_sample(rank, world, spp, f), out=img)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for f in range(args.warmup):
        frame(f)
    ctx.check()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    k0 = pt.kernel_launches()
    for i in range(args.steps):
        flush.fill_(float(i))           # evict L2 between timed frames (not timed)
        ev[i][0].record(stream)
        frame(args.warmup + i)          # renders replay the library's CUDA graphs
        ev[i][1].record(stream)
    barrier()
    kernels = pt.kernel_launches() - k0
    clocks = sampler.stop()
    ctx.check()
    ms = R.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / args.steps, dev)
    value = world * cfg.n_slots / (ms * 1e-3) / 1e6
    n_done = args.warmup + args.steps
    # per-kernel split from three more frames with per-launch events, scaled to the timed frames
    n_prof = min(args.steps, 3)
    prof = profiled_split(pt, ctx, lambda i: frame(n_done + i), args.steps, n_prof)
    n_done += n_prof
    pt.profile_enable(ctx, True)
    pt.profile_read(ctx)

    # split of one more frame: the training step, then the cached render alone
    gc.train_frame(scene, gnif, W, H, n_done * world + rank, n_train=N_TRAIN, max_depth=cfg.max_depth,
                   rec_vertex=CACHE_VERTEX, seed=0, precision=prec, loss=losses[n_done:n_done + 1],
                   train_precision=args.train_precision)
    prof_train = pt.profile_read(ctx)
    pt.render_cached(ctx, scene, gnif, cfg, None, cache=gc, cache_vertex=CACHE_VERTEX, precision=prec,
                     first_sample=(n_done * world + rank) * spp, out=img)
    prof_render = pt.profile_read(ctx)
    pt.profile_enable(ctx, False)
    counts = pt.last_render_counts(ctx, cfg.max_depth, with_cache=True)
    work = pt.last_render_work(ctx)
    trace_kernel, trace_launches = trace_kernels(pt, ctx, CACHE_VERTEX)
    n_done += 1
    ctx.check()

    # the plain full-depth frame of the same size, FP32 and the chosen precision
    def plain_ms(p, reps=3):
        pt.render(ctx, scene, gnif, cfg, p, out=img_plain)
        torch.cuda.synchronize()
        e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for i in range(reps):
            flush.fill_(float(i))
            e[i][0].record(stream)
            pt.render(ctx, scene, gnif, cfg, p, out=img_plain, first_sample=(i + 1) * spp)
            e[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in e) / reps
    plain = {"fp32_ms": plain_ms("fp32")}
    plain[f"{prec}_ms"] = plain_ms(prec)
    plain["fp32_msamples_s"] = cfg.n_slots / (plain["fp32_ms"] * 1e-3) / 1e6
    ctx.check()

    # bias of the cache after the 60-frame loop: frozen cache at 1024 spp vs the plain 4096-spp FP32 render
    bias = None
    if not args.no_bias and args.spp is None:
        while n_done < C5_FRAMES:
            frame(n_done)
            n_done += 1
        base = 1 << 24
        ref = []
        for b in range(16):
            rc = I.RenderCfg(W, H, 256, cfg.max_depth, 0)
            ref.append(pt.render(ctx, scene, gnif, rc, "fp32", first_sample=base + 256 * b).double())
        ref = torch.stack(ref)
        R_mean, R_var = ref.mean(0), ref.var(0) / ref.shape[0]
        del ref
        X = []
        for b in range(8):
            rc = I.RenderCfg(W, H, 128, cfg.max_depth, 0)
            X.append(pt.render_cached(ctx, scene, gnif, rc, None, cache=gc, cache_vertex=CACHE_VERTEX, precision=prec,
                                      first_sample=2 * base + 128 * b)[0].double().reshape(H, W, 3))
        X = torch.stack(X)
        ctx.check()
        bias = {"frames_trained": n_done, "reference": "plain FP32 render, 4096 spp (16 batches of 256)",
                "cached": f"frozen cache after {n_done} frames, {prec} NIF, 1024 spp (8 batches of 128)",
                "reference_noise_rel_rmse": float(torch.sqrt(R_var.sum() / (R_mean ** 2).sum()))}
        bias.update(image_stats(X, R_mean, R_var))
        del X

        # equal time: one cached frame (its training step included in the time) against plain frames of
        # about the same duration; each single frame's relative RMSE against the 4096-spp reference,
        # averaged over 8 independent frames
        def frame_rmse(render_one, n=8):
            v = []
            for i in range(n):
                Y = render_one(i).double().reshape(H, W, 3)
                v.append(float(torch.sqrt(((Y - R_mean) ** 2).sum() / (R_mean ** 2).sum())))
            return float(np.mean(v))
        spp_eq = max(1, int(round(spp * ms / plain[f"{prec}_ms"])))
        cfg_eq = I.RenderCfg(W, H, spp_eq, cfg.max_depth, 0)
        bias["equal_time"] = {
            "cached": {"ms": ms, "spp": spp, "rel_rmse": frame_rmse(lambda i: pt.render_cached(
                ctx, scene, gnif, cfg, None, cache=gc, cache_vertex=CACHE_VERTEX, precision=prec,
                first_sample=3 * base + spp * i)[0])},
            f"plain_{prec}": {"ms_est": plain[f"{prec}_ms"] * spp_eq / spp, "spp": spp_eq,
                              "rel_rmse": frame_rmse(lambda i: pt.render(ctx, scene, gnif, cfg_eq, prec,
                                                                         first_sample=4 * base + spp_eq * i))},
            "plain_fp32_same_spp": {"ms": plain["fp32_ms"], "spp": spp,
                                    "rel_rmse": frame_rmse(lambda i: pt.render(ctx, scene, gnif, cfg, "fp32",
                                                                               first_sample=5 * base + spp * i))}}
        ctx.check()
        del R_mean, R_var

    # roofline of the dominant kernel kind inside the frame
    meas, which = peaks()
    clock = float(meas.get("sm_max_mhz", 2070.0))
    kinds = {k: v[0] / args.steps for k, v in prof.items()}
    dom = max(("trace", "nif", "cache"), key=lambda k: kinds[k])
    rays = int(counts[:cfg.max_depth].sum())
    queries = int(counts[cfg.max_depth + 1])
    if dom == "cache":
        t_c = prof_render["cache"][0]
        peak = SM_COUNT * FP32_LANES_PER_SM * 2 * clock * 1e6 / 1e12
        achieved = queries * CACHE_FLOP_PER_QUERY / (t_c * 1e-3) / 1e12
        roof = {"kernel": "k_cache_eval", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "per_unit": f"{CACHE_FLOP_PER_QUERY} FLOP per query x {queries} queries per launch",
                "peak_note": f"FP32 FFMA derived: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 x {clock:.0f} MHz"}
    else:
        roof = traversal_roofline(work, prof_render["trace"][0], trace_kernel, trace_launches,
                                  pt.ffma_rate_tflops(local), clock, " (the cached render)")

    e2e = None
    if not args.no_e2e:
        host_img = torch.empty((W * H, 3), dtype=torch.float32, pin_memory=True)
        scene_arrays = (sc.sphere, sc.sphere_mat, sc.quad, sc.quad_axis, sc.quad_mat, sc.vert, sc.tri, sc.tri_mat,
                        sc.mat_type, sc.mat)
        cache_host = I.cache_init(lo, hi)
        flat = gc.get_params()
        pos = 0
        for Wl, bl in zip(cache_host.W, cache_host.b):
            Wl[:] = flat[pos:pos + Wl.size].reshape(Wl.shape)
            pos += Wl.size
            bl[:] = flat[pos:pos + bl.size]
            pos += bl.size
        h2d = sum(x.nbytes for x in scene_arrays) + pt.nif_flat(nif).nbytes + pt.cache_flat(cache_host).nbytes
        d2h = host_img.numel() * 4
        n_e2e = max(2, min(args.steps, 5))

        def inputs():
            return pt.Scene(ctx, sc, node_format=args.nodes), pt.Nif(ctx, nif), pt.Cache(ctx, cache_host)

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nxt = inputs()
        for i in range(n_e2e):
            s2, n2, c2 = nxt
            c2.train_frame(s2, n2, W, H, n_done + i, n_train=N_TRAIN, max_depth=cfg.max_depth,
                           rec_vertex=CACHE_VERTEX, seed=0, precision=prec, train_precision=args.train_precision)
            pt.render_cached(ctx, s2, n2, cfg, None, cache=c2, cache_vertex=CACHE_VERTEX, precision=prec,
                             first_sample=(n_done + i) * spp, out=img)
            host_img.copy_(img, non_blocking=True)
            # the next step's scene, weights and cache are built and uploaded while the GPU works on this one
            nxt = inputs() if i + 1 < n_e2e else None
            torch.cuda.synchronize()
            del s2, n2, c2
        dt = (time.perf_counter() - t0) / n_e2e
        e2e = {"value": world * cfg.n_slots / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "note": "per step: pt_create_scene (host BVH build) + pt_load_nif + pt_create_cache from host "
                       "arrays, pt_train_cache, pt_render_cached, image copied to pinned host memory; step "
                       "i+1's inputs are built and uploaded (context upload stream) while the GPU works on step i"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, sample = oracle_c5_rate(sc, nif, cache0, cfg, args.cpu_s)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}

    if rank == 0:
        loss_h = losses[:n_done].cpu().numpy()
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec,
            "data": "synthetic (procedural heightfield and sky, NIF trained on the sky, cache trained online; seeds 0)",
            "config": c5_config(cfg), "nif": nif_dict(prec, train is not None),
            "cache": {"shape": "12 freqs/axis position encoding + direction + normal (78) -> 5x FC-64 ReLU -> FC-3",
                      "training": "FP32 master weights, Adam lr 1e-2, relative L2",
                      "train_gemms": args.train_precision},
            "kernel_ms_per_step": kinds,
            "frame_split_ms": {"train": {k: v[0] for k, v in prof_train.items()},
                               "render": {k: v[0] for k, v in prof_render.items()}},
            "plain_full_depth": plain,
            "speedup_vs_plain_fp32": plain["fp32_ms"] / ms,
            "cache_bias": bias,
            "cache_loss": {"first": float(loss_h[0]), "last10_mean": float(loss_h[-10:].mean())},
            "rays_per_render": rays, "cache_queries_per_render": queries,
            "nif_evals_per_render": int(counts[cfg.max_depth]),
            "scene_build_s": t_build, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": int(kernels), "nif_training": train,
        }))
    if world > 1:
        dist.destroy_process_group()
    return 0


def bench_nif_sweep(args):
    """NIF size sweep (the paper's question of how large a network stays
    resident in on-chip SRAM, Section 3.3): for each shape, BF16-GEMM
    training on the procedural 2048 x 1024 sky, its quality against the sky,
    standalone FP32 and BF16 evaluation rates on 2^24 coordinates, and the C2
    frame rate with that network as the environment.  The BF16 kernel keeps
    every weight in shared memory; it takes H = 128 with 1 to 5 hidden layers
    (three, two, then one 128-row tile slot beside the weights) and H = 64
    or 32 with 1 to 8 (four slots), H = 256 with one (two 64 KB slots),
    and no shape beyond.  Networks wider than 128 are not trained (the
    training chains are 128 wide): their rows give the rates of the
    random-init network.  The last row is the paper's network (20
    frequencies, four layers of 128, the features joined after the second).
    One JSON line."""
    import torch
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt
    dev = "cuda:0"
    ctx = pt.Context(0)
    stream = torch.cuda.current_stream()
    sky = torch.from_numpy(I.procedural_sky()).to(dev)
    uv = torch.from_numpy(I.uniform_uv(1 << 24, seed=1)).to(dev)
    sc, cfg, _ = workload("C2")
    scene = pt.Scene(ctx, sc, node_format=args.nodes)
    img = torch.empty((cfg.height, cfg.width, 3), dtype=torch.float32, device=dev)
    steps = max(args.train_steps, 1)

    def ms_of(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    rows = []
    # (frequencies, width, hidden layers, skip layer); the last row is the paper's network: 20 frequencies,
    # four layers of 128, the second layer's output joined with the features (Section 3.2)
    shapes = [(64, H, L, 0) for H, L in ((128, 1), (128, 2), (128, 3), (128, 4), (128, 5), (128, 6), (128, 8),
                                         (64, 2), (64, 3), (64, 4), (64, 8), (32, 2), (32, 3), (32, 4), (32, 8),
                                         (256, 1), (256, 2), (256, 4), (256, 8))]
    shapes.append((20, 128, 4, I.paper_skip_layer(4)))
    for F, H, L, S in shapes:
        def make():
            return pt.Nif(ctx, I.nif_init(n_freq=F, hidden=H, n_hidden_layers=L, colour="yuv", skip_after=S))
        g = make()
        row = {"n_freq": F, "hidden": H, "layers": L, "skip_after": S, "params": g.param_count,
               "weights_kb_bf16": (g.param_count * 2) // 1024}
        if H <= 128:
            tprec = "bf16"
            try:
                g.train(sky, steps=1, batch=1024, lr=1e-3, seed=99, precision="bf16")
            except RuntimeError:   # the BF16 training chains need the weights resident in shared memory too
                tprec = "fp32"
            g = make()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.train(sky, steps=steps, batch=1 << 16, lr=1e-3, seed=0, precision=tprec)
            e1.record(stream)
            torch.cuda.synchronize()
            row.update({"train_gemms": tprec, "train_ms_per_step": e0.elapsed_time(e1) / steps,
                        "quality": nif_quality(g, sky, dev)})
        else:
            row.update({"train_gemms": None, "train_ms_per_step": None, "quality": None,
                        "train_note": "not trained: the training chains are 128 wide; rates of the random-init "
                                      "network"})
        row["fp32_evals_per_s"] = (1 << 24) / (ms_of(lambda: g.eval(uv, "fp32"), 2) * 1e-3)
        bf16_ok = ((F == 64 and S == 0 and ((H == 128 and 1 <= L <= 5) or (H in (64, 32) and 1 <= L <= 8) or
                                            (H == 256 and L == 1))) or (F, H, L, S) == (20, 128, 4, 2))
        if bf16_ok:
            row["bf16_evals_per_s"] = (1 << 24) / (ms_of(lambda: g.eval(uv, "bf16"), 3) * 1e-3)
            row["bf16_tile_slots"] = ({256: 2, 128: 3 if L <= 3 else (2 if L == 4 else 1)}.get(H, 4) if not S else 3)
            fr = ms_of(lambda: pt.render(ctx, scene, g, cfg, "bf16", out=img), 3)
            row["c2_bf16_msamples_s"] = cfg.n_slots / (fr * 1e-3) / 1e6
        else:
            row["bf16_evals_per_s"] = None
            row["bf16_note"] = ("not resident: the BF16 kernel needs H = 128 with L <= 5, H = 64 / 32 with L <= 8 "
                                "or H = 256 with L = 1")
            fr = ms_of(lambda: pt.render(ctx, scene, g, cfg, "fp32", out=img), 3)
            row["c2_fp32_msamples_s"] = cfg.n_slots / (fr * 1e-3) / 1e6
        ctx.check()
        rows.append(row)
        del g
    print(json.dumps({"metric": "NIF size sweep: quality vs evaluation and path rate", "n_gpus": 1,
                      "train_steps": steps, "unit": "evals/s, Msamples/s", "higher_is_better": True,
                      "config": {"sky": "procedural 2048x1024", "render": "C2 512x512 64 spp depth 8",
                                 "training": "Adam lr 1e-3, batch 2^16, BF16 tensor-core GEMMs where the shape "
                                             "fits (else FP32)"},
                      "rows": rows}))
    return 0


def bench_nif_eval(args):
    """Standalone NIF evaluation (the network of Section 3.2 that the renderer
    evaluates for its escaped rays), one kernel: 2^n uniform (u, v) through
    the --precision kernel, W untimed launches then K launches timed one by
    one with CUDA events, a 512 MB L2 flush between them (outside the events).
    The shape is the renderer's (F = 64, 3 x FC-128).  One JSON line with the
    evaluation rate and the kernel's roofline."""
    import torch
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt
    dev = "cuda:0"
    ctx = pt.Context(0)
    stream = torch.cuda.current_stream()
    n = 1 << args.nif_eval
    g = pt.Nif(ctx, I.nif_init(colour="yuv"))
    uv = torch.from_numpy(I.uniform_uv(n, seed=1)).to(dev)
    flush = torch.empty(128 << 20, dtype=torch.float32, device=dev)
    prec = args.precision
    for _ in range(max(args.warmup, 3)):
        g.eval(uv, prec)
    torch.cuda.synchronize()
    ctx.check()
    sampler = ClockSampler(0)
    sampler.start()
    times = []
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.eval(uv, prec)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    ctx.check()
    ms = float(np.mean(times))
    meas, which = peaks()
    if prec == "fp32":
        flop = FLOP_PER_EVAL
        peak = pt.ffma_rate_tflops(0)
        bound, kernel, note = "alu", "k_nif_fp32", "FP32 FMA rate measured live by pt_microbench_ffma"
    else:
        flop = TC_FLOP_PER_EVAL
        peak = float(meas["bf16_tflops"]) * (2.0 if prec == "fp8" else 1.0)
        bound, kernel = "tensor", ("k_nif_tc" if prec == "bf16" else "k_nif_fp8")
        note = (f"dense BF16 cuBLAS burst ({which})" if prec == "bf16" else
                f"dense FP8 = BF16 cuBLAS burst ({which}) x 2 (nominal 4.5 / 2.25 PFLOP/s)")
    achieved = n * flop / (ms * 1e-3) / 1e12
    print(json.dumps({"metric": "NIF evaluations per second (standalone)", "value": n / (ms * 1e-3), "unit": "evals/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
                      "ms_min": float(np.min(times)), "higher_is_better": True, "dtype": prec, "data": "synthetic",
                      "config": {"workload": f"2^{args.nif_eval} uniform (u, v), F=64 Fourier (sigma 10) -> 3x FC-128 "
                                             f"ReLU -> FC-3 -> colour matrix -> exp, random-init weights",
                                 "l2": "512 MB flush between timed launches"},
                      "roofline": {"kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak,
                                   "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                                   "per_unit": f"{flop} FLOP per evaluation x {n} evaluations per launch",
                                   "peak_note": note},
                      "clocks": clocks, "gpu_launches": args.steps}))
    return 0


def bench_colour_sweep(args):
    """Colour space of the NIF's output head (Section 3.2: the network predicts
    log colour in a chosen space and a fixed matrix maps it to RGB before exp):
    RGB, YUV (BT.601) and YCoCg heads trained alike on the procedural sun sky,
    quality against the sky (log-RMSE, tonemapped PSNR with its luma and
    chroma parts).  A synthetic stand-in for the paper's HDRI study.  One JSON
    line."""
    import torch
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt
    dev = "cuda:0"
    ctx = pt.Context(0)
    sky = torch.from_numpy(I.procedural_sky()).to(dev)
    steps = max(args.train_steps, 1)
    rows = []
    for colour in ("identity", "yuv", "ycocg"):
        g = pt.Nif(ctx, I.nif_init(colour=colour))
        losses = g.train(sky, steps=steps, batch=1 << 16, lr=1e-3, seed=0, precision=args.train_precision)
        ctx.check()
        rows.append({"head": {"identity": "RGB", "yuv": "YUV (BT.601)", "ycocg": "YCoCg"}[colour],
                     "loss_last": float(losses[-50:].mean().item()), "quality": nif_quality(g, sky, dev)})
    print(json.dumps({"metric": "NIF colour-space study: quality against the sky", "n_gpus": 1, "train_steps": steps,
                      "higher_is_better": True, "unit": "dB / log-RMSE",
                      "config": {"nif": "F=64, 3x FC-128, Adam lr 1e-3, batch 2^16",
                                 "train_gemms": args.train_precision, "sky": "procedural 2048x1024"},
                      "rows": rows}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["C1", "C2", "C3", "C4", "C5"], default="C2")
    ap.add_argument("--precision", choices=["bf16", "fp32", "fp8"], default="bf16")
    ap.add_argument("--spp", type=int, default=None, help="override spp (small cases for profiler captures)")
    ap.add_argument("--depth", type=int, default=None, help="override the maximum path length (C1-C4)")
    ap.add_argument("--rr", action="store_true", help="Russian roulette from depth 3 (the paper's perf mode; C1-C4)")
    ap.add_argument("--cpu-s", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--ref-step-s", type=float, default=4.0, help="seconds per reference-arm step")
    ap.add_argument("--train-steps", type=int, default=2000,
                    help="Adam steps of the environment NIF on the procedural sky before the frames (0: random init)")
    ap.add_argument("--train-precision", choices=["bf16", "fp32"], default="bf16",
                    help="GEMMs of NIF and radiance-cache training (tensor cores or CUDA cores)")
    ap.add_argument("--nodes", choices=["auto", "packed", "decoded", "quant8"], default="auto",
                    help="BVH node form the traversal reads (pt_scene_desc.node_format)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the other-precision frames and standalone NIF runs (profiler captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bias", action="store_true", help="C5: skip the bias measurement against the 4096-spp render")
    ap.add_argument("--nif-sweep", action="store_true",
                    help="NIF size sweep (hidden width and depth vs quality, evaluation and path rate); one JSON line")
    ap.add_argument("--nif-eval", type=int, default=None, metavar="LOG2N",
                    help="standalone NIF evaluation of 2^LOG2N coordinates in --precision; one JSON line")
    ap.add_argument("--colour-sweep", action="store_true",
                    help="NIF colour-space study (RGB / YUV / YCoCg heads); one JSON line")
    args = ap.parse_args()
    if args.nif_sweep:
        return bench_nif_sweep(args)
    if args.nif_eval is not None:
        return bench_nif_eval(args)
    if args.colour_sweep:
        return bench_colour_sweep(args)
    if args.impl == "reference":
        return bench_reference(args)
    if args.workload == "C5":
        return bench_c5(args)
    return bench_ours(args)


if __name__ == "__main__":
    sys.exit(main())
