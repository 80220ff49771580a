#!/usr/bin/env python3
"""Benchmark of the vector-valued Allen-Cahn time step on GB300.

Workload (default): the 4096 x 4096 RGB Voronoi-ramp image (8 regions, ramps
<= 0.2, noise sigma 0.05), N = 8 phases, eps = 3, lambda = 2, tau = 9, each
time step solved to a natural residual of 1e-6 by V(2,1) cycles; 3 untimed
steps, then the 100 time steps of the workload timed.  A "step" is one time
step: colour means + energy, right-hand side, and V-cycles until the
tolerance.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference ...   # the CPU oracle on the same workload

One JSON line on rank 0.  value = time steps per second of the whole job
(replicas: every rank advances its own image, no exchange).  The timed region
is K steps bracketed by a barrier and a device synchronize, timed with CUDA
events on the solver's stream; the phase field (1.07 GB in FP64) is larger
than L2, so no flush is needed between steps.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Allen-Cahn steps/s & GDOF/s at 4096² N=8; % HBM peak; vs plain FP64 GPU"
WORKLOAD = "c3_4096_n8_mixed"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 100 time steps of the 4096^2 workload, 30 image steps of the batch, "
                         "4 gradient evaluations of the adjoint)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--skip", type=int, default=0,
                    help="untimed time steps after the reset to the seeded start, before the timed ones (0: time "
                         "the workload's first steps; e.g. 40 for a sample after phase separation)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="steps of the plain FP64 form timed for the vs-FP64 ratio (default: --steps, the same "
                         "steps as the mixed form; 0: skip)")
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--projection", choices=["simplex", "node"], default="simplex",
                    help="data projection of the image (Sec. 4.2): exact moments by simplex, or nodal values with "
                         "the consistent mass matrix")
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--nu1", type=int, default=2, help="pre-smoothing red-black sweeps per V-cycle")
    ap.add_argument("--nu2", type=int, default=1, help="post-smoothing red-black sweeps per V-cycle")
    ap.add_argument("--crop", type=int, default=256, help="side of the image crop the CPU oracle times")
    ap.add_argument("--cpu-steps", type=int, default=3, help="oracle steps in the cpu_baseline sample")
    ap.add_argument("--workload", choices=["single", "batch", "adjoint", "refine"], default="single",
                    help="single: the 4096^2 N=8 image; batch: 256 uneven images (sizes 128^2..1024^2, N 2/4/6); "
                         "adjoint: gradients through 64 steps of the 512^2 N=4 disks image; refine: the 1024^2 "
                         "N=4 disks/polygons image on its pixel grid refined twice (4096^2 cells)")
    ap.add_argument("--refine", type=int, default=2, help="refinements of the pixel grid (refine workload)")
    ap.add_argument("--adj-steps", type=int, default=64, help="time steps differentiated (adjoint workload)")
    ap.add_argument("--adj-every", type=int, default=8, help="checkpoint interval (adjoint workload)")
    ap.add_argument("--adj-precond", choices=["f32", "f64"], default="f32",
                    help="precision of the V-cycles preconditioning the adjoint's FP64 flexible CG")
    ap.add_argument("--batch-images", type=int, default=256)
    ap.add_argument("--streams", type=int, default=16)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch sub-line of the default workload")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint sub-line of the default workload")
    ap.add_argument("--batch-steps", type=int, default=30, help="image steps of the batch sub-line (the workload's 30)")
    ap.add_argument("--adjoint-evals", type=int, default=2, help="gradient evaluations of the adjoint sub-line")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = {"single": 100, "batch": 30, "adjoint": 4, "refine": 20}[args.workload]
    if args.fp64_steps is None:
        args.fp64_steps = args.steps if args.workload == "single" else 3
    return args


def workload(args):
    from paper_0710_0736_gb300 import synth
    cfg = dict(synth.CONFIGS[WORKLOAD])
    cfg["W"] = cfg["H"] = args.size
    if args.tol is not None:
        cfg["tol"] = args.tol
    return cfg


def workload_config(cfg, args, extra=None):
    d = {
        "workload": f"{cfg['W']}x{cfg['H']} RGB Voronoi-ramp image (8 regions, ramp<=0.2, noise 0.05), "
                    f"N={cfg['N']}, eps={cfg['eps']}, lambda={cfg['lam']}, tau={cfg['tau']}, "
                    f"each step to natural residual {cfg['tol']:g}",
        "nodes": (cfg["W"] + 1) * (cfg["H"] + 1),
        "n_phases": cfg["N"],
        "precision": args.precision,
        "projection": args.projection,
        "tol": cfg["tol"],
        "l2": "no flush: the phase field and right-hand side (1.07 GB each in FP64) exceed the 129 MB L2",
        "timed_steps": f"{args.skip + 1}..{args.skip + args.steps} of the workload's time steps from the seeded start",
    }
    if extra:
        d.update(extra)
    return d


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax = float(row[2])
            except ValueError:
                continue
            for name, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes per node of one launch of k_smooth_fine<float, 8, shifted>: ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) at 2048 x 2048, 248.9 MB over
# 4,198,401 nodes (profiles/k_smooth_fine_mixed_2048_n8_ncu.md), scaled to
# the workload by nodes.  It holds for the kernel source it was taken on: the
# digest covers the kernel's text and that of the device helpers it calls.
BREAKDOWN_STEPS = 5  # profiled steps after the timed region, for the per-class breakdown


def job_rate(local_ms, local_units, world, device):
    """Whole-job rate over `world` replicas: the work units of every rank
    summed, divided by the slowest rank's time (the maximum over ranks).
    Returns (units per second, maximum ms).  With world > 1 a process group
    must be initialised (NCCL on the GPUs; gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    return float(u.item()) / (ms_max / 1e3), ms_max

SMOOTH_TRAFFIC = {"sha256": "a0467499a47d6f0029c4ad9328b3cf2a61457a4359bf305310fac607d20c5941",
                  "bytes_per_node": (201.543936e6 + 47.308032e6) / 4198401, "n_phases": 8, "precision": "mixed"}
SMOOTH_HELPERS = ("node_class", "edge_weights", "fslot", "geo_te", "geo_invD", "omega_t", "rcp_small", "proj_box",
                  "nbr_sum", "ldn", "ldn_rw", "stn", "mark_dirty")


def _function_text(src, name):
    import re
    m = re.search(r"\n((?:template <[^\n]*>\n)?__[^\n]*\b" + re.escape(name) + r"\([^;{]*\{)", src)
    if m is None:
        return ""
    i = m.start(1)
    return src[i:src.index("\n}\n", i) + 3]


def smooth_source_digest():
    import hashlib
    csrc = os.path.join(ROOT, "paper_0710_0736_gb300", "csrc")
    with open(os.path.join(csrc, "ac_kernels.cuh")) as f:
        kern = f.read()
    with open(os.path.join(csrc, "ac_device.cuh")) as f:
        dev = f.read()
    text = _function_text(kern, "k_smooth_fine") + "".join(_function_text(dev, n) for n in SMOOTH_HELPERS)
    return hashlib.sha256(text.encode()).hexdigest()


def smooth_bytes(prof):
    """Algorithmic bytes of all timed smoother launches: each launch moves the
    library's per-launch bytes (one colour's right-hand side and obstacle and
    the other colour's iterate read, its own colour written); a launch that
    also applies the pending coarse correction reads the other colour's
    correction d as well."""
    from paper_0710_0736_gb300 import ac
    return (prof.launches[ac.PROF_CLASSES.index("smooth")] * prof.smooth_bytes_per_launch
            + prof.smooth_corr_launches * prof.smooth_corr_extra_bytes)


def smooth_traffic(n_nodes, n_phases, precision):
    """Measured DRAM bytes of one smoother launch, or None when no capture of
    the current kernel source exists for this configuration."""
    t = SMOOTH_TRAFFIC
    if n_phases != t["n_phases"] or precision != t["precision"] or smooth_source_digest() != t["sha256"]:
        return None
    return t["bytes_per_node"] * n_nodes


def step_roofline(prof, breakdown, steps, ms, peak):
    """The whole step against the HBM roofline: the algorithmic bytes of every
    kernel class over the timed steps (the library's per-launch counts:
    every array element a launch is defined on read and written once, the
    coarse levels counted dense) per step, over the measured ms per step;
    per class, the bytes and event times of the profiled sample after the
    timed region."""
    from paper_0710_0736_gb300 import ac
    per_step = sum(prof.bytes) / steps
    achieved = per_step / (ms / steps / 1e3) / 1e9
    classes = {}
    for k, c in enumerate(ac.PROF_CLASSES):
        b, t = breakdown.bytes[k], breakdown.ms[k]
        if b <= 0 and t <= 0:
            continue
        classes[c] = {"gb_per_step": b / BREAKDOWN_STEPS / 1e9, "ms_per_step": t / BREAKDOWN_STEPS,
                      "achieved": (b / (t / 1e3) / 1e9) if t > 0 else None,
                      "frac": (b / (t / 1e3) / 1e9 / peak) if t > 0 else None}
    return {"alg_bytes_per_step": per_step, "achieved": achieved, "frac": achieved / peak, "unit": "GB/s",
            "target_frac": 0.6, "by_class_sample": classes}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# --------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# --------------------------------------------------------------------------

def oracle_sample(cfg, crop, steps, seed=0):
    """Time `steps` oracle steps (paper-literal SSC, V(2,2)) on the top-left
    crop x crop corner of the workload image; returns per-step seconds."""
    import oracle
    from paper_0710_0736_gb300 import synth
    oracle.build()
    img = synth.config_image(WORKLOAD, seed, cfg["W"], cfg["H"])[:crop, :crop].astype(np.float64)
    m = oracle.moments(img)
    u = synth.dirichlet_init(seed, (crop + 1) ** 2, cfg["N"])
    c = np.zeros((cfg["N"], 3))
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        u, c, it, rho, st = oracle.step(u, m, c, crop, crop, cfg["eps"], cfg["lam"], cfg["tau"], tol=cfg["tol"],
                                        nu1=2, nu2=2, max_iter=1000)
        times.append(time.perf_counter() - t0)
    return times


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = workload(args)
    # each step a bounded sample: the crop shrinks when many steps are asked
    # for, so that the whole run stays within a few minutes
    if args.warmup + args.steps > 20:
        args.crop = min(args.crop, 128)
    times = oracle_sample(cfg, args.crop, args.warmup + args.steps)
    timed = times[args.warmup:]
    full_nodes = (cfg["W"] + 1) * (cfg["H"] + 1)
    crop_nodes = (args.crop + 1) ** 2
    sec_full = float(np.mean(timed)) * full_nodes / crop_nodes  # the method's cost is linear in the nodes
    value = 1.0 / sec_full
    sample = (f"{args.steps} oracle steps (SSC, V(2,2), tol {cfg['tol']:g}) on the {args.crop}x{args.crop} corner "
              f"of the workload image after {args.warmup} untimed, scaled by nodes {full_nodes}/{crop_nodes}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_full * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(cfg, args, {"precision": "fp64",
                                                  "solver": "oracle: sequential SSC over all levels, V(2,2), FP64"}),
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def batch_leg(args, steps, warmup, fp64_steps):
    """The uneven batch: 256 shape images (as the 64x64 workload, scaled) of
    sizes 128^2..1024^2 and 768x512, N in {2,4,6}, noise sigma U[0.02,0.15],
    eps 2, lambda 1, tau 4, mixed precision to tol 1e-6, `steps` time steps
    per image timed after `warmup`.  value = image time steps per second
    (each timed step advances all images once).  The plain FP64 form is timed
    for fp64_steps steps twice: on the same stream pool as the mixed form
    (the precision's gain alone) and image after image on one stream (the
    unbatched form).  Returns the line as a dict."""
    import torch
    from paper_0710_0736_gb300 import ac, synth
    specs = synth.batch_specs(0, args.batch_images)
    tol = args.tol if args.tol is not None else 1e-6
    imgs = []
    for sp in specs:
        s = sp["W"] / 64.0
        imgs.append(synth.shapes_image(sp["seed"], sp["W"], sp["H"], sigma=sp["sigma"],
                                       rect_side=(max(1, int(8 * s)), max(1, int(32 * s))), disk_r=(4 * s, 16 * s)))
        sp.update(eps=2.0, lam=1.0, tau=4.0, tol=tol, max_cycles=1000)

    def make(precision, streams):
        for sp in specs:
            sp["precision"] = precision
        b = ac.Batch(specs, n_streams=streams)
        for k, im in enumerate(imgs):
            b.set_image(k, im)
        return b

    b = make(ac.AC_MIXED, args.streams)
    t_tune = 0.0
    if not args.no_tune:
        t0 = time.perf_counter()
        b.tune(trial_steps=2)
        t_tune = time.perf_counter() - t0
    b.step(warmup, allow_not_converged=True)
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    t0 = time.perf_counter()
    st = b.step(steps, allow_not_converged=True)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    clk = clocks.stop()
    b.close()
    value = st.images * steps / el

    def fp64_rate(streams):
        b64 = make(ac.AC_FP64, streams)
        b64.step(1, allow_not_converged=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s64 = b64.step(fp64_steps, allow_not_converged=True)
        torch.cuda.synchronize()
        el64 = time.perf_counter() - t0
        b64.close()
        return {"value": s64.images * fp64_steps / el64, "unit": "image-steps/s", "steps": fp64_steps,
                "streams": streams, "vcycles_per_image_step": s64.total_cycles / (s64.images * fp64_steps),
                "all_converged": s64.converged_images == s64.images}

    # the same batch with one graph launch per time step: every image's step
    # (its V-cycle loop on the device) in one CUDA graph
    b = make(ac.AC_MIXED, args.streams)
    if not args.no_tune:
        b.tune(trial_steps=2)
    b.set_launch(ac.AC_BATCH_ONE_GRAPH)
    b.step(warmup, allow_not_converged=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sg = b.step(steps, allow_not_converged=True)
    torch.cuda.synchronize()
    el_g = time.perf_counter() - t0
    b.close()
    one_graph = {"value": sg.images * steps / el_g, "unit": "image-steps/s", "steps": steps,
                 "ms_per_step": el_g / steps * 1e3,
                 "vcycles_per_image_step": sg.total_cycles / (sg.images * steps),
                 "all_converged": sg.converged_images == sg.images,
                 "launch": "one CUDA graph per time step holding every image's step, each image's V-cycle and "
                           "defect-correction loops under device-side WHILE nodes (AC_BATCH_ONE_GRAPH)",
                 "ratio_over_stream_pool": (sg.images * steps / el_g) / value}
    pooled = fp64_rate(args.streams)
    unbatched = fp64_rate(1)
    pooled["ratio_batched_mixed_over_this"] = value / pooled["value"]
    unbatched["ratio_batched_mixed_over_this"] = value / unbatched["value"]
    sizes = {}
    for sp in specs:
        key = f"{sp['W']}x{sp['H']}/N{sp['N']}"
        sizes[key] = sizes.get(key, 0) + 1
    return {"metric": "batched Allen-Cahn image time steps/s (256 uneven images)", "value": value,
            "unit": "image-steps/s", "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": el / steps * 1e3, "higher_is_better": True,
            "dtype": "f32 + double-float residual/means/rhs + f64 state",
            "config": {"workload": f"{st.images} images, sizes 128^2/256^2/512^2/1024^2/768x512, N in 2/4/6, "
                                   f"noise U[0.02,0.15], eps 2, lambda 1, tau 4, tol {tol:g}, mixed precision, "
                                   f"{args.streams} streams, autotuned {'no' if args.no_tune else 'yes'}",
                       "nodes": st.nodes, "dof": st.dof, "groups": sizes,
                       "l2": "no flush: the batch's fields (92 M nodes) exceed the 129 MB L2"},
            "gdof_per_s": st.dof_sweeps / el / 1e9,
            "vcycles_per_image_step": st.total_cycles / (st.images * steps),
            "all_converged": st.converged_images == st.images, "tune_seconds": t_tune, "clocks": clk,
            "launch": f"stream pool: {args.streams} streams, one host worker thread per stream, each image's "
                      "V-cycle loop on the host (AC_BATCH_STREAMS)",
            "one_graph": one_graph,
            "plain_fp64_gpu_same_pool": pooled, "plain_fp64_gpu_unbatched": unbatched,
            "ratio_mixed_over_fp64": value / unbatched["value"]}


def run_batch(args):
    line = batch_leg(args, args.steps, args.warmup, max(1, min(args.steps, args.fp64_steps or 1)))
    line.update({"scaling": "weak", "vs_baseline": None, "data": "synthetic"})
    print(json.dumps(line), flush=True)
    return 0


def adjoint_leg(args, steps, warmup, with_cpu):
    """Gradients through T = 64 time steps of the 512 x 512, N = 4 disks image
    (12 disks, noise 0.08; eps 2, lambda 1, tau 4, each step solved to 1e-10)
    of the misfit L = 1/2 sum Mhat |u^T - onehot(target)|^2 to a 6-seed Voronoi
    target, with respect to lambda, eps, the image and u^0.  One "step" here
    is one gradient evaluation: the forward with checkpoints every 8 steps
    (ac_adjoint_forward), then the backward sweep (ac_adjoint_backward),
    which recomputes each segment from its checkpoint.  value = gradient
    evaluations per second.  Returns the line as a dict."""
    import torch
    import oracle
    from paper_0710_0736_gb300 import ac, synth
    name = "c5_512_n4_adjoint"
    cfg = dict(synth.CONFIGS[name])
    W, H, N, T, every = cfg["W"], cfg["H"], cfg["N"], args.adj_steps, args.adj_every
    tol = args.tol if args.tol is not None else cfg["tol"]
    img = synth.config_image(name, 0).astype(np.float64)
    u0 = synth.dirichlet_init(1, (W + 1) * (H + 1), N)
    target = synth.voronoi_labels(2, W + 1, H + 1, n_seeds=6, n_labels=N)
    torch.cuda.set_device(0)
    # a stream of its own: torch's default stream is the legacy stream (handle 0),
    # on which the library cannot capture its CUDA graphs
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)  # torch's own work of this leg goes on the same stream
    dev = torch.device("cuda", 0)
    onehot = np.eye(N)[target.ravel().astype(int)]
    m0 = None

    def measure(precision, steps, warmup):
        nonlocal m0
        seg = ac.Segmenter(W, H, N, cfg["eps"], cfg["lam"], cfg["tau"], tol=tol, max_cycles=2000,
                           precision=precision, stream=stream.cuda_stream)
        ac.ac_set_adjoint_preconditioner(
            seg.ctx, ac.AC_ADJ_PRECOND_F64 if getattr(args, "adj_precond", "f32") == "f64" else ac.AC_ADJ_PRECOND_F32)
        if precision == ac.AC_MIXED:
            seg.set_image(torch.tensor(img, dtype=torch.float32, device=dev))
        else:
            seg.set_image(torch.tensor(img, device=dev))
        if m0 is None:
            m0 = torch.tensor(seg.moments()[:, 0], device=dev)
        u0_d = torch.tensor(u0, device=dev)
        oh = torch.tensor(onehot, device=dev)
        uT = torch.empty_like(u0_d)
        g_img = torch.empty((H, W, 3), dtype=torch.float64, device=dev)
        g_u0 = torch.empty_like(u0_d)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        t_fwd = t_bwd = 0.0
        cycles = 0
        for it in range(warmup + steps):
            seg.set_phase(u0_d)
            if it == warmup:
                torch.cuda.synchronize()
            evs[0].record(stream)
            ac.ac_adjoint_forward(seg.ctx, T, every)
            evs[1].record(stream)
            ac.ac_get_phase(seg.ctx, uT, seg.n_nodes, N)
            grad = m0[:, None] * (uT - oh)  # dL/du^T of the misfit
            gl, ge = ac.ac_adjoint_backward(seg.ctx, grad.contiguous(), g_img, g_u0)
            evs[2].record(stream)
            torch.cuda.synchronize()
            if it >= warmup:
                t_fwd += evs[0].elapsed_time(evs[1])
                t_bwd += evs[1].elapsed_time(evs[2])
        seg.close()
        return t_fwd / steps, t_bwd / steps, gl, ge

    clocks = Clocks(0)
    clocks.start()
    fwd_ms, bwd_ms, gl, ge = measure(ac.AC_FP64, steps, warmup)
    clk = clocks.stop()
    # the mixed-precision forward (FP32 sweeps, FP64 defect correction) with the same FP64 adjoint
    mfwd_ms, mbwd_ms, mgl, mge = measure(ac.AC_MIXED, max(1, steps // 2), warmup)
    ms = fwd_ms + bwd_ms
    value = 1e3 / ms

    cpu = None
    if with_cpu:
        crop, Tc = 128, 8
        ic = img[:crop, :crop]
        uc = synth.dirichlet_init(1, (crop + 1) ** 2, N)
        tc = synth.voronoi_labels(2, crop + 1, crop + 1, n_seeds=6, n_labels=N)
        t0 = time.perf_counter()
        states = oracle.forward_states(ic, uc, cfg["eps"], cfg["lam"], cfg["tau"], Tc, tol=tol)
        _, gT = oracle.misfit_loss(states[-1], oracle.moments(ic)[:, 0], tc)
        oracle.adjoint(ic, states, cfg["eps"], cfg["lam"], cfg["tau"], gT, cg_rtol=1e-12)
        sec = time.perf_counter() - t0
        scale = ((W + 1) * (H + 1)) / (crop + 1) ** 2 * T / Tc
        cpu = {"value": 1.0 / (sec * scale), "unit": "gradient evaluations/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle forward ({Tc} steps, SSC to {tol:g}) + FP64 adjoint (tangent CG to 1e-12) on "
                         f"the {crop}x{crop} corner, {sec:.1f} s, scaled by nodes and steps x{scale:.0f}"}
    return {"metric": "adjoint gradient evaluations/s (64 steps, 512^2 N=4)", "value": value,
            "unit": "gradient evaluations/s", "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f64 (the tangent solve's V-cycle preconditioner in "
                     + ("f64" if getattr(args, "adj_precond", "f32") == "f64" else "f32") + ")",
            "config": {"workload": f"{W}x{H} disks image (12 disks, noise 0.08), N={N}, eps={cfg['eps']}, "
                                   f"lambda={cfg['lam']}, tau={cfg['tau']}, {T} steps to tol {tol:g}, "
                                   f"checkpoints every {every}, misfit to a 6-seed Voronoi target",
                       "l2": "no flush: 14 MB of checkpoints plus segment states; small case, L2-resident"},
            "forward_ms": fwd_ms, "backward_ms": bwd_ms, "backward_over_forward": bwd_ms / fwd_ms,
            "grad_lambda": gl, "grad_eps": ge,
            "mixed_forward": {"forward_ms": mfwd_ms, "backward_ms": mbwd_ms, "grad_lambda": mgl, "grad_eps": mge,
                              "value": 1e3 / (mfwd_ms + mbwd_ms)},
            "cpu_baseline": cpu, "clocks": clk}


def run_adjoint(args):
    line = adjoint_leg(args, args.steps, args.warmup, not args.no_cpu)
    line.update({"scaling": "weak", "vs_baseline": None, "data": "synthetic"})
    print(json.dumps(line), flush=True)
    return 0


def run_refine(args):
    """The 1024 x 1024 image of 64 disks and convex polygons in 4 colours
    (noise 0.1; N = 4, eps = 2 px, lambda = 1, tau = 4) on its pixel grid
    refined r = 2 times (Sec. 4.1: several nodes per interface), i.e. a
    4096 x 4096 solve grid, mixed precision to natural residual 1e-6.
    value = time steps per second."""
    import torch
    import oracle
    from paper_0710_0736_gb300 import ac, synth
    name = "c2_1024_n4"
    cfg = dict(synth.CONFIGS[name])
    W, H, N, r = cfg["W"], cfg["H"], cfg["N"], args.refine
    tol = args.tol if args.tol is not None else cfg["tol_mixed"]
    img = synth.config_image(name, 0)
    torch.cuda.set_device(0)
    # a stream of its own: torch's default stream is the legacy stream (handle 0),
    # on which the library cannot capture its CUDA graphs
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)  # torch's own work of this leg goes on the same stream
    seg = ac.Segmenter(W, H, N, cfg["eps"], cfg["lam"], cfg["tau"], tol=tol, max_cycles=1000, precision=ac.AC_MIXED,
                       refine=r, nu1=args.nu1, nu2=args.nu2, stream=stream.cuda_stream)
    seg.set_image(torch.from_numpy(img).cuda())
    seg.step(args.warmup, allow_not_converged=True)
    # events around the smoother only: the timed region needs its launch times
    ac.ac_set_profiling_mask(seg.ctx, ["smooth"])
    launches0 = ac.ac_get_profile(seg.ctx).total_launches
    clocks = Clocks(0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    _, st = ac.ac_step(seg.ctx, args.steps, allow_not_converged=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = ac.ac_get_profile(seg.ctx)
    seg.close()
    n = (seg.Wr + 1) * (seg.Hr + 1)
    peaks, peak_kind = measured_peaks()
    sm_launches = prof.launches[ac.PROF_CLASSES.index("smooth")]
    sm_ms = prof.ms[ac.PROF_CLASSES.index("smooth")]
    achieved = smooth_bytes(prof) / max(1, sm_launches) / (sm_ms / 1e3 / max(1, sm_launches)) / 1e9
    cpu = None
    if not args.no_cpu:
        # the oracle on a 64 x 64 corner of the image, refined the same way
        crop, steps = 64, 2
        s = 1 << r
        ic = oracle.refine_image(img[:crop, :crop], r)
        e2, l2, t2 = oracle.refined_params(cfg["eps"], cfg["lam"], cfg["tau"], r)
        u = synth.dirichlet_init(0, (crop * s + 1) ** 2, N)
        t0 = time.perf_counter()
        oracle.run(ic, u, e2, l2, t2, steps, tol=tol, nu1=2, nu2=2, max_iter=1000)
        sec = (time.perf_counter() - t0) / steps * n / (crop * s + 1) ** 2
        cpu = {"value": 1.0 / sec, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{steps} oracle steps (SSC, V(2,2), tol {tol:g}) on the {crop}x{crop} corner refined "
                         f"{r} times, scaled by nodes"}
    line = {"metric": "refined-grid Allen-Cahn steps/s (1024^2 image, pixel grid refined twice)",
            "value": args.steps / (ms / 1e3), "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{W}x{H} disks/polygons image (64 shapes, 4 colours, noise 0.1), N={N}, "
                                   f"eps={cfg['eps']} px, lambda={cfg['lam']}, tau={cfg['tau']}, refine={r} "
                                   f"({seg.Wr}x{seg.Hr} cells), mixed, each step to natural residual {tol:g}",
                       "nodes": n, "solver": f"truncated monotone multigrid V({args.nu1},{args.nu2})"},
            "gdof_per_s": N * n * st.fine_sweeps / (ms / 1e3) / 1e9,
            "vcycles_per_step": st.total_cycles / max(1, st.steps), "all_converged": bool(st.converged),
            "roofline": {"bound": "hbm", "kernel": "k_smooth_fine<float,4,shifted>", "achieved": achieved,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                         "peak_kind": f"{peak_kind} hbm_gbs", "traffic": None},
            "gpu_launches": int(prof.total_launches - launches0), "cpu_baseline": cpu, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "refine":
        return run_refine(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_0710_0736_gb300 import ac, synth

    cfg = workload(args)
    W, H, N = cfg["W"], cfg["H"], cfg["N"]
    n_nodes = (W + 1) * (H + 1)
    prec = ac.AC_FP64 if args.precision == "fp64" else ac.AC_MIXED
    img = synth.config_image(WORKLOAD, rank, W, H)
    # a stream of its own: torch's default stream is the legacy stream (handle 0),
    # on which the library cannot capture its CUDA graphs
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)  # torch's own work of this leg goes on the same stream
    proj = ac.AC_PROJ_NODE if args.projection == "node" else ac.AC_PROJ_SIMPLEX
    seg = ac.Segmenter(W, H, N, cfg["eps"], cfg["lam"], cfg["tau"], tol=cfg["tol"], max_cycles=1000, seed=rank,
                       precision=prec, stream=stream.cuda_stream, nu1=args.nu1, nu2=args.nu2, projection=proj)
    dev_img = torch.from_numpy(img).cuda()
    seg.set_image(dev_img)
    seg.step(args.warmup, allow_not_converged=True)
    # back to the seeded start: the timed steps are the workload's first K
    # time steps (as the end-to-end leg below times them); the warm-up has
    # captured the graphs and loaded the kernels
    seg.set_image(dev_img)
    if args.skip > 0:
        seg.step(args.skip, allow_not_converged=True)
    torch.cuda.synchronize()

    # events around the smoother only (its launch times give the roofline); the
    # per-class breakdown comes from a few profiled steps after the timed region
    ac.ac_set_profiling_mask(seg.ctx, ["smooth"])
    launches0 = ac.ac_get_profile(seg.ctx).total_launches
    clocks = Clocks(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    rc, st = ac.ac_step(seg.ctx, args.steps, allow_not_converged=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = ac.ac_get_profile(seg.ctx)
    launches = prof.total_launches - launches0
    ac.ac_set_profiling(seg.ctx, True)
    ac.ac_step(seg.ctx, BREAKDOWN_STEPS, allow_not_converged=True)
    breakdown = ac.ac_get_profile(seg.ctx)
    ac.ac_set_profiling(seg.ctx, False)

    value, ms_max = job_rate(ms, args.steps, world, "cuda")
    gdof = job_rate(ms, N * n_nodes * float(st.fine_sweeps), world, "cuda")[0] / 1e9

    # roofline of the dominant kernel: the fine red-black smoother
    peaks, peak_kind = measured_peaks()
    sm_launches = prof.launches[ac.PROF_CLASSES.index("smooth")]
    sm_ms = prof.ms[ac.PROF_CLASSES.index("smooth")]
    avg_launch_s = sm_ms / 1e3 / max(1, sm_launches)
    bytes_avg = smooth_bytes(prof) / max(1, sm_launches)
    achieved = bytes_avg / avg_launch_s / 1e9
    kname = "k_smooth_fine<float,N,shifted>" if args.precision == "mixed" else "k_smooth_fine<double,N,direct>"
    roofline = {"bound": "hbm", "kernel": kname + " (one colour of a red-black projected sweep)",
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "peak_kind": f"{peak_kind} hbm_gbs", "traffic": smooth_traffic(n_nodes, N, args.precision),
                "traffic_unit": "bytes per plain launch (ncu capture at 2048^2 of launches without a pending "
                                "correction, scaled by nodes); compare plain_launch_bytes",
                "bytes_per_launch": bytes_avg, "plain_launch_bytes": prof.smooth_bytes_per_launch,
                "correction_launches": prof.smooth_corr_launches, "launches": sm_launches,
                "avg_launch_ms": avg_launch_s * 1e3, "share_of_step_time": sm_ms / max(1e-9, ms),
                "step": step_roofline(prof, breakdown, args.steps, ms, peaks["hbm_gbs"])}

    # end to end through the public API with host buffers: the same K steps
    # from the seeded start, the image copied in from pinned host memory
    e2e = None
    if not args.no_e2e and args.skip == 0:  # (with --skip the copy-in would precede untimed steps)
        host_img = torch.from_numpy(img).pin_memory()
        labels = torch.empty((H, W), dtype=torch.int8).pin_memory()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ac.ac_set_image(seg.ctx, host_img, W, H)
        for _ in range(args.steps):
            ac.ac_segment(seg.ctx, 1, labels, W, H, allow_not_converged=True, stats=False)
        torch.cuda.synchronize()
        e2e_value, _ = job_rate((time.perf_counter() - t0) * 1e3, args.steps, world, "cuda")
        e2e = {"value": e2e_value, "unit": "steps/s",
               "h2d_bytes_per_step": host_img.numel() * 4 / args.steps, "d2h_bytes_per_step": labels.numel(),
               "path": "ac_set_image from pinned host memory once (it resets u to the seeded start, as before "
                       "the device-timed steps), then per step ac_segment(1 step, no statistics) with the pixel "
                       "labels read back to pinned host memory: the same K time steps as value"}

    # the plain FP64 form on the same workload, for the mixed/FP64 ratio
    fp64 = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        seg.close()
        seg64 = ac.Segmenter(W, H, N, cfg["eps"], cfg["lam"], cfg["tau"], tol=cfg["tol"], max_cycles=1000, seed=rank,
                             precision=ac.AC_FP64, stream=stream.cuda_stream, nu1=args.nu1, nu2=args.nu2,
                             projection=proj)
        seg64.set_image(dev_img)
        seg64.step(args.warmup, allow_not_converged=True)
        seg64.set_image(dev_img)  # the same time steps from the seeded start as the mixed form
        if args.skip > 0:
            seg64.step(args.skip, allow_not_converged=True)
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        _, st64 = ac.ac_step(seg64.ctx, args.fp64_steps, allow_not_converged=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        v64, _ = job_rate(ev0.elapsed_time(ev1), args.fp64_steps, world, "cuda")
        fp64 = {"value": v64, "unit": "steps/s", "steps": args.fp64_steps, "from": "the seeded start",
                "vcycles_per_step": st64.total_cycles / max(1, st64.steps), "ratio_mixed_over_fp64": value / v64}
        seg = seg64

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        times = oracle_sample(cfg, args.crop, args.cpu_steps)
        full_nodes, crop_nodes = n_nodes, (args.crop + 1) ** 2
        cpu = {"value": 1.0 / (float(np.mean(times)) * full_nodes / crop_nodes), "unit": "steps/s", "cores": 1,
               "kind": "oracle",
               "sample": f"{args.cpu_steps} oracle steps (SSC, V(2,2), tol {cfg['tol']:g}) on the {args.crop}x"
                         f"{args.crop} corner of the workload image, {sum(times):.1f} s, scaled by nodes "
                         f"{full_nodes}/{crop_nodes}; an upper bound on the oracle's rate at full size (its "
                         f"per-node cost grows with the number of levels)"}

    # the other two workloads, bounded, each as a sub-line with its own config
    batch = adjoint = None
    if rank == 0 and world == 1:
        seg.close()
        if not args.no_batch:
            batch = batch_leg(args, args.batch_steps, args.warmup, 3)
        if not args.no_adjoint:
            adjoint = adjoint_leg(args, args.adjoint_evals, 1, False)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32 + double-float residual/means/rhs + f64 state",
                "data": "synthetic",
                "config": workload_config(cfg, args, {"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                                      "solver": f"truncated monotone multigrid V({args.nu1},{args.nu2})"}),
                "gdof_per_s": gdof, "vcycles_per_step": st.total_cycles / max(1, st.steps),
                "fine_sweeps_per_step": st.fine_sweeps / max(1, st.steps), "residual": st.residual,
                "outer_per_step": st.outer / max(1, st.steps), "plain_fp64_gpu": fp64,
                "all_converged": bool(st.converged), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk,
                # the library's kernel launches before the timed region (an ncu --launch-skip for it)
                "launches_before_timed": int(launches0),
                "profile_ms_sample": {"steps": BREAKDOWN_STEPS, "after": "the timed region, every class profiled",
                                      "ms": dict(zip(ac.PROF_CLASSES, [round(v, 3) for v in breakdown.ms]))},
                "batch": batch, "adjoint": adjoint}
        print(json.dumps(line), flush=True)
    seg.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
