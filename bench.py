#!/usr/bin/env python3
"""Benchmark of the RTM hot path on GB300.

One bench step is one full RTM shot of the single-shot throughput workload:
512^3 model (576^3 padded with a 32-cell sponge), 8th-order stencil, smooth
random velocity (1500-4500 m/s, sigma 8), 2000 steps, 20 Hz Ricker at the
surface centre, 512 x 512 receivers at depth index 2, checkpoints every 50
steps: forward modelling with checkpoints, then per segment a recompute with
snapshot writes and the receiver propagation with the imaging condition fused
into the backward stencil. The metric is stencil point-updates per second over
all three passes (3 x 2000 x 576^3 per shot).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (under torchrun) every rank runs its own shot (weak scaling); the
timing is the slowest rank's. ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpoint-updates/s vs HBM roofline; RTM shot time learned vs checkpoint @≤1e-2"
UNIT = "Gpoint-updates/s"
PROFILE = os.path.join(ROOT, "profiles", "stencil_tma_bwd_image_r4_smooth512.md")
STENCIL_SRC = os.path.join(ROOT, "paper_1603_03971_gb300", "csrc", "stencil_tma.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="smooth_512")
    ap.add_argument("--nt", type=int, default=0, help="override the step count (testing only)")
    ap.add_argument("--model", type=int, default=0,
                    help="override the model edge (profiling cases; the line is then not the "
                         "headline workload)")
    ap.add_argument("--ckpt-every", type=int, default=0, help="override the checkpoint interval")
    ap.add_argument("--radius", type=int, default=0, choices=(0, 4, 8),
                    help="override the stencil radius (profiling cases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ref-steps", type=int, default=20,
                    help="oracle time steps per bench step of the reference arm (the same "
                         "sample as the CPU baseline of our arm)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-compression leg (384^3, 3000 steps)")
    ap.add_argument("--learned-train-steps", type=int, default=8000)
    ap.add_argument("--learned-models", type=int, default=64)
    ap.add_argument("--learned-window", type=int, default=120,
                    help="exact window: the first steps whose snapshots are recomputed from the "
                         "zero state instead of coded (checkpoint-recompute fallback)")
    ap.add_argument("--zchunk", type=int, default=0,
                    help="z-slab height of the main run (0: autotuned)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the library's automatic slab height instead of the autotuner")
    ap.add_argument("--no-grad", action="store_true",
                    help="skip the velocity-gradient leg (gradient_256 workload)")
    ap.add_argument("--no-boundary", action="store_true",
                    help="skip the boundary-storage shot (reverse time stepping)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-shots leg (32 apertures, radius 8)")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the two-layer 64^3 full-RTM leg (per-shot time, CUDA graph)")
    ap.add_argument("--no-r8", action="store_true",
                    help="skip the radius-8 leg (smooth 512^3 model, 200 steps)")
    ap.add_argument("--no-decomp", action="store_true",
                    help="skip the 2 x 2 domain-decomposition leg (smooth 512^3 forward)")
    ap.add_argument("--batch-nt", type=int, default=1500)
    ap.add_argument("--batch-shots", default="all",
                    help="comma-separated aperture indices of the batched workload (default all 32)")
    ap.add_argument("--batch-ckpt", type=int, default=50, help="checkpoint interval of the batch")
    ap.add_argument("--batch-compare-nt", type=int, default=100,
                    help="steps of the comparison of the batch with single shots on the same "
                         "apertures (0: skip)")
    ap.add_argument("--imaging", action="store_true",
                    help="also time the imaging-condition variants (source illumination, "
                         "normalised and Laplacian-filtered image) on the main workload")
    ap.add_argument("--revolve", type=int, default=0, metavar="SLOTS",
                    help="also time one shot of the main workload with binomial checkpointing "
                         "in SLOTS checkpoint slots")
    ap.add_argument("--variant", type=int, default=0,
                    help="stencil plane-load variant and tile: 0 automatic, 1 vector loads, "
                         "2 TMA 16-row tiles, 3 TMA 8-row tiles")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args):
    import rtm_inputs

    w = rtm_inputs.WORKLOADS[args.workload]
    if args.nt:
        w = w.scaled(nt=args.nt)
    if args.model:
        n = args.model
        w = w.scaled(nx=n, ny=n, nz=n, src=(n // 2, n // 2, w.src[2]), name=w.name + "@%d" % n)
    if args.ckpt_every:
        w = w.scaled(ckpt_every=args.ckpt_every)
    if args.radius:
        w = w.scaled(radius=args.radius)
    return w


def config_of(w):
    NZ, NY, NX = w.padded_shape
    return {
        "workload": "%s: %dx%dx%d model (%dx%dx%d padded), r=%d stencil, %d steps, "
                    "%s velocity, %.0f Hz Ricker, %dx%d receivers, checkpoint every %d"
                    % (w.name, w.nx, w.ny, w.nz, NX, NY, NZ, w.radius, w.nt, w.velocity,
                       w.f0, w.nx, w.ny, w.ckpt_every),
        "grid": [w.nx, w.ny, w.nz],
        "padded": [NX, NY, NZ],
        "radius": w.radius,
        "nt": w.nt,
        "ckpt_every": w.ckpt_every,
        "updates_per_shot": 3 * w.nt * NX * NY * NZ,
        "l2": "inputs larger than L2 (each field %.0f MB > 129 MB L2)" % (NX * NY * NZ * 4 / 1e6),
    }


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import torch

            ident = str(self.dev)
            uuid = getattr(torch.cuda.get_device_properties(self.dev), "uuid", None)
            if uuid is not None:
                u = str(uuid)
                ident = u if u.startswith("GPU-") else "GPU-" + u
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", ident, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            out["reasons"] = ["unsampled"]
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            out["reasons"] = ["unsampled"]
            return out
        sm = sorted(float(r[1]) for r in rows if re.match(r"^[\d.]+$", r[1]))
        mx = [float(r[2]) for r in rows if re.match(r"^[\d.]+$", r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        out.update(sm_mhz=sm[len(sm) // 2] if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


# ----------------------------------------------------------------------------
# roofline helpers
# ----------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_code_digest(path: str) -> str:
    """SHA-256 of a CUDA source with its comments and blank lines removed:
    it names the kernel code a profile was taken on, whatever its comments
    say."""
    text = open(path).read()
    out, i, n = [], 0, len(text)
    while i < n:
        ch = text[i]
        if ch in "\"'":  # a string or character literal, kept whole
            j = i + 1
            while j < n and text[j] != ch:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(ch)
            i += 1
    lines = [line.rstrip() for line in "".join(out).splitlines()]
    return hashlib.sha256("\n".join(x for x in lines if x).encode()).hexdigest()


def profiled_traffic(radius: int, tile_rows: int, padded_shape, zchunk, alg_bytes):
    """DRAM bytes per launch of the backward imaging stencil from the committed
    ncu summary: its traffic / algorithmic ratio at the run's slab height,
    times the run's algorithmic bytes per launch; only if the summary was
    taken on the current kernel code with the same radius, tile rows and
    padded grid (else None)."""
    if not os.path.exists(PROFILE) or not zchunk:
        return None
    text = open(PROFILE).read()
    m_h = re.search(r"stencil_code_sha256:\s*([0-9a-f]{64})", text)
    m_r = re.search(r"tile_rows:\s*(\d+)", text)
    m_s = re.search(r"radius:\s*(\d+)", text)
    m_g = re.search(r"padded_grid:\s*([\dx]+)", text)
    m_t = re.search(r"traffic_ratio_zchunk_%d:\s*([\d.eE+]+)" % int(zchunk), text)
    if not (m_t and m_h and m_r and m_s and m_g) or int(m_r.group(1)) != tile_rows \
            or int(m_s.group(1)) != radius \
            or m_g.group(1) != "x".join(str(int(n)) for n in padded_shape):
        return None
    if kernel_code_digest(STENCIL_SRC) != m_h.group(1):
        return None
    return float(m_t.group(1)) * float(alg_bytes)


# ----------------------------------------------------------------------------
# CPU oracle timing (baseline and reference arm)
# ----------------------------------------------------------------------------

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the
    machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.machine()


def oracle_sample(w, vel_np, steps: int, lead: int = 3):
    """Time ``steps`` forward time steps of the FP64 oracle on the full padded
    grid of the workload, without its allocation: the oracle allocates and
    first touches its fields inside a forward call, within its first few
    steps, so the sample is the difference of a (lead + steps)-step and a
    lead-step run on the same prepared grid. Returns (seconds, updates,
    threads)."""
    import oracle

    rec = w.receivers()[:1]
    p = oracle.Problem(vel_np, w.nb, w.radius, w.dx, w.dt, lead + steps, w.f0, w.t0, w.src, rec)
    t = time.perf_counter()
    p.grid.forward(p.w[:lead], p.src, p.rec)
    t_short = time.perf_counter() - t
    t = time.perf_counter()
    p.grid.forward(p.w, p.src, p.rec)
    t_long = time.perf_counter() - t
    del p
    NZ, NY, NX = w.padded_shape
    return max(t_long - t_short, 1e-9), steps * NX * NY * NZ, oracle.num_threads()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    w = workload(args)
    vel = w.velocity_model(device=None) if w.nx <= 256 else None
    if vel is None:
        import torch

        dev = "cuda" if torch.cuda.is_available() else None
        v = w.velocity_model(device=dev)
        vel = v.double().cpu().numpy() if hasattr(v, "cpu") else v
    vel = np.asarray(vel, dtype=np.float64)
    NZ, NY, NX = w.padded_shape
    for _ in range(args.warmup):  # warm-up samples of two steps
        oracle_sample(w, vel, min(args.ref_steps, 2))
    total_s, total_u, threads = 0.0, 0, 1
    for _ in range(args.steps):
        s, u, threads = oracle_sample(w, vel, args.ref_steps)
        total_s += s
        total_u += u
    value = total_u / total_s / 1e9
    sample = ("%d forward time steps of the FP64 oracle on the %dx%dx%d padded grid per bench "
              "step, allocation and first touch excluded (a %d-step run minus a 3-step run)"
              % (args.ref_steps, NX, NY, NZ, args.ref_steps + 3))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# learned snapshot compression vs checkpoint recompute (384^3, 3000 steps)
# ----------------------------------------------------------------------------

def learned_leg(args, dev):
    """Train the codec on propagator snapshots of seeded random 192^3 models
    (untimed), then time one RTM shot of the 384^3 smooth-model workload
    (3000 steps, imaging every 4) with checkpoint recompute (every 50 steps)
    and with learned storage, and compare the two images."""
    import torch

    import paper_1603_03971_gb300 as rtm
    import rtm_inputs
    from paper_1603_03971_gb300 import learned

    t0 = time.perf_counter()
    data = learned.training_snapshots(n_models=args.learned_models, size=192, nt=1200, every=40,
                                      first=40, device=dev)
    P, losses = learned.train(data, steps=args.learned_train_steps, batch=4, lr=1e-3,
                              lr_min=5e-5, log_every=0, init="decimation")
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    n_snap = int(data.shape[0])
    del data
    w = rtm_inputs.WORKLOADS["learned_384"]
    # both shots run with the autotuned launch shape of this padded grid
    tuned = (tune_shape(w.radius, w.padded_shape)
             if args.variant == 0 and not args.no_autotune else None)
    v = w.velocity_model(device=dev).contiguous()
    rec = torch.from_numpy(w.receivers()).to(dev)
    pc = rtm.params_for(w, storage="ckpt", ckpt_every=50)
    ws = rtm.alloc_workspace(pc, dev)
    # observed data: the scattered field of thin beds (data of the model with
    # the beds minus the direct field of the smooth migration model)
    c_true = rtm.model_prep(pc, rtm_inputs.thin_bed_reflectors(v).contiguous(), ws)
    dobs = torch.empty((w.nt, pc.nrec), dtype=torch.float32, device=dev)
    rtm.forward(pc, c_true, rec, ws, data=dobs)
    del c_true
    c = rtm.model_prep(pc, v, ws)
    d_direct = torch.empty_like(dobs)
    rtm.forward(pc, c, rec, ws, data=d_direct)
    dobs -= d_direct
    del d_direct
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    img_c = torch.zeros((w.nz, w.ny, w.nx), dtype=torch.float32, device=dev)
    rtm.shot(pc, c, rec, dobs, ws, img_c)  # warm-up
    img_c.zero_()
    torch.cuda.synchronize()
    e0.record()
    rtm.shot(pc, c, rec, dobs, ws, img_c)
    e1.record()
    torch.cuda.synchronize()
    t_ckpt = e0.elapsed_time(e1) / 1e3
    ws_ckpt_gb = ws.numel() / 1e9
    del ws

    def run(storage, window):
        """One timed shot (after a warm-up) with learned or decimated storage
        and the given exact window; returns (seconds, image rel-L2 against the
        checkpoint image, the same below the top 16 model layers, workspace GB)."""
        q = rtm.params_for(w, storage=storage, ckpt_every=window)
        wq = rtm.alloc_workspace(q, dev)
        img = torch.zeros_like(img_c)

        def once():
            if storage == "learned":
                rtm.shot_learned(q, c, rec, dobs, P, wq, img)
            else:
                rtm.shot(q, c, rec, dobs, wq, img)
        once()
        img.zero_()
        torch.cuda.synchronize()
        e0.record()
        once()
        e1.record()
        torch.cuda.synchronize()
        rtm.check(wq)
        t = e0.elapsed_time(e1) / 1e3
        e = float((img - img_c).norm() / img_c.norm())
        ed = float((img[16:] - img_c[16:]).norm() / img_c[16:].norm())
        gb = wq.numel() / 1e9
        del wq, img
        return t, e, ed, gb

    W = args.learned_window
    t_learned, err, err_deep, ws_l_gb = run("learned", W)
    t_dec, err_dec, err_dec_deep, ws_d_gb = run("decimated", W)
    no_window = None
    if W > 0:
        tl0, el0, _, _ = run("learned", 0)
        td0, ed0, _, _ = run("decimated", 0)
        no_window = {"shot_s_learned": tl0, "image_rel_l2_learned": el0,
                     "shot_s_decimated": td0, "image_rel_l2_decimated": ed0}
    from paper_1603_03971_gb300 import codec

    enc_ms, dec_ms = codec._time_codec(w.nx, reps=10)
    # bf16 tensor-core work per snapshot as executed: E1 (2^3 patch, K padded
    # to 16) and E2 (3^3 x 32 taps); D1 (k4 s2: 2^3 taps x 16 channels per
    # output) and D2 (32 channels -> 2^3 outputs, N padded to 16)
    h, q = (w.nx // 2) ** 3, (w.nx // 4) ** 3
    enc_flop = 2 * h * 32 * 16 + 2 * q * 16 * 32 * 27
    dec_flop = 2 * h * 32 * 16 * 8 + 2 * h * 32 * 16
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16 = float(peaks.get("bf16_tflops_sustained", 1700.0))
    codec_tc = {
        "encode_gflop": enc_flop / 1e9, "decode_gflop": dec_flop / 1e9,
        "encode_tflops": enc_flop / (enc_ms * 1e-3) / 1e12,
        "decode_tflops": dec_flop / (dec_ms * 1e-3) / 1e12,
        "peak_tflops": bf16,
        "peak_kind": "measured sustained bf16" if "bf16_tflops_sustained" in peaks
        else "fallback sustained bf16",
    }
    codec_tc["encode_frac"] = codec_tc["encode_tflops"] / bf16
    codec_tc["decode_frac"] = codec_tc["decode_tflops"] / bf16
    NZ, NY, NX = w.padded_shape
    return {
        "workload": "learned_384: 384^3 model (448^3 padded), r=4, 3000 steps, smooth random "
                    "velocity, imaging every 4 steps (750 snapshots); observed data: scattered "
                    "field of three thin beds (+-8 %) at depths 96/192/288",
        "shot_s_checkpoint": t_ckpt, "checkpoint_every": 50,
        "workspace_gb_checkpoint": ws_ckpt_gb, "workspace_gb_learned": ws_l_gb,
        "exact_window_steps": W,
        "coded_snapshots": (w.nt - W) // w.image_every,
        "window_snapshots": W // w.image_every,
        "shot_s_learned": t_learned, "speedup_vs_checkpoint": t_ckpt / t_learned,
        "image_rel_l2_vs_checkpoint": err, "target_rel_l2": 1e-2,
        "image_rel_l2_below_z16": err_deep,
        # the non-learned 8x scheme at the same bytes and window: every other
        # sample per axis in float32, linear interpolation
        "decimated": {"shot_s": t_dec, "speedup_vs_checkpoint": t_ckpt / t_dec,
                      "image_rel_l2_vs_checkpoint": err_dec,
                      "image_rel_l2_below_z16": err_dec_deep, "workspace_gb": ws_d_gb},
        "learned_over_decimated_error_ratio": err / err_dec if err_dec > 0 else None,
        "no_window": no_window,
        "codec_ms_per_snapshot": {"encode": enc_ms, "decode": dec_ms},
        "codec_tensor": codec_tc,
        "compression": "8x (float32 snapshot -> 16 bfloat16 channels per 4^3 voxels)",
        "train": {"models": args.learned_models, "snapshots": n_snap, "init": "decimation",
                  "steps": args.learned_train_steps, "batch": 4, "seconds": train_s,
                  "final_loss": losses[-1][1]},
        "updates_per_shot_learned": 2 * w.nt * NX * NY * NZ,
        "tuning": tuned,
    }


def imaging_leg(p, c, rec, dobs, ws, dev):
    """The receiver pass with and without the source-illumination
    accumulation (same checkpoints, recomputed each time), and the image
    filters, on the main workload; CUDA events on the launching stream."""
    import torch

    import paper_1603_03971_gb300 as rtm

    img = torch.zeros((p.nz, p.ny, p.nx), dtype=torch.float32, device=dev)
    illum = torch.zeros_like(img)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        rtm.forward(p, c, rec, ws)
        torch.cuda.synchronize()
        ev[0].record()
        fn()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 1e3

    t_plain = timed(lambda: rtm.backward_image(p, c, rec, dobs, ws, img))
    t_illum = timed(lambda: rtm.backward_image_illum(p, c, rec, dobs, ws, img, illum))
    rtm.check(ws)
    torch.cuda.synchronize()
    ev[0].record()
    rtm.image_filter(p, img, ws, illum=illum, eps_rel=1e-3)
    ev[1].record()
    torch.cuda.synchronize()
    t_filter = ev[0].elapsed_time(ev[1]) / 1e3
    nmodel = p.nx * p.ny * p.nz
    n_img = p.nt // p.image_every
    illum_bytes = 12.0 * nmodel * n_img  # snapshot read, illumination read + write
    extra = t_illum - t_plain
    return {"backward_s": t_plain, "backward_with_illumination_s": t_illum,
            "illumination_overhead_s": extra,
            "illumination_pass_gbs": illum_bytes / extra / 1e9 if extra > 0 else None,
            "illumination_bytes_per_step": 12.0 * nmodel,
            "filter_s": t_filter}


def revolve_leg(w, slots, vel, rec, dobs, dev):
    """One shot of the main workload with binomial checkpointing in ``slots``
    slots (the forward pass models data only; the backward pass recomputes
    along the optimal schedule), CUDA events around the shot."""
    import torch

    import paper_1603_03971_gb300 as rtm

    p = rtm.params_for(w, storage="revolve", ckpt_every=slots)
    ws = rtm.alloc_workspace(p, dev)
    c = rtm.model_prep(p, vel, ws)
    img = torch.zeros((p.nz, p.ny, p.nx), dtype=torch.float32, device=dev)
    rtm.shot(p, c, rec, dobs, ws, img)  # warm-up (and the schedule's plan)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    rtm.shot(p, c, rec, dobs, ws, img)
    ev[1].record()
    torch.cuda.synchronize()
    rtm.check(ws)
    t = ev[0].elapsed_time(ev[1]) / 1e3
    nrecomp = rtm.revolve_cost(p.nt // p.image_every, slots) * p.image_every
    NZ, NY, NX = w.padded_shape
    steps = p.nt + nrecomp + p.nt  # data forward + recompute + backward
    res = {"slots": slots, "workspace_gb": ws.numel() / 1e9, "shot_s": t,
           "recomputed_forward_steps": nrecomp, "stencil_steps": steps,
           "gpoint_updates_per_s": steps * NX * NY * NZ / t / 1e9}
    del ws
    return res


def boundary_leg(w, vel, rec, dobs, dev, ref_image, ref_shot_s, ref_ws_gb, autotune=True):
    """One shot of the main workload with boundary storage: the forward pass
    keeps the model region's boundary band of every state, the backward pass
    recovers the source field by reverse time stepping (no recompute pass).
    CUDA events around the shot; the image is compared with the checkpoint
    image of the timed run."""
    import torch

    import paper_1603_03971_gb300 as rtm

    if autotune:
        tune_shape(w.radius, w.padded_shape)  # the main run's shape (cached)
    p = rtm.params_for(w, storage="boundary")
    ws = rtm.alloc_workspace(p, dev)
    c = rtm.model_prep(p, vel, ws)
    img = torch.zeros((p.nz, p.ny, p.nx), dtype=torch.float32, device=dev)
    rtm.shot(p, c, rec, dobs, ws, img)  # warm-up
    img.zero_()
    rtm.reset_stats()
    rtm.set_timing(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    rtm.shot(p, c, rec, dobs, ws, img)
    ev[1].record()
    torch.cuda.synchronize()
    rtm.set_timing(False)
    st = rtm.stats()
    rtm.check(ws)
    t = ev[0].elapsed_time(ev[1]) / 1e3
    num = float(torch.linalg.vector_norm((img - ref_image).double()))
    den = float(torch.linalg.vector_norm(ref_image.double()))
    NZ, NY, NX = w.padded_shape
    modes = {k: {"ms_per_launch": v["ms"] / v["launches"],
                 "gbs": v["bytes"] / v["ms"] / 1e6}
             for k, v in st["stencil"].items() if v["launches"] and v["ms"] > 0}
    # stencil updates: forward and receiver passes on the padded grid, the
    # reverse pass on the model region (nt - 2 steps)
    updates = 2 * p.nt * NX * NY * NZ + max(p.nt - 2, 0) * p.nx * p.ny * p.nz
    res = {"shot_s": t, "shot_s_checkpoint": ref_shot_s, "speedup_vs_checkpoint": ref_shot_s / t,
           "workspace_gb": ws.numel() / 1e9, "workspace_gb_checkpoint": ref_ws_gb,
           "image_rel_l2_vs_checkpoint": num / den if den > 0 else None,
           "gpoint_updates_per_s": updates / t / 1e9, "stencil_modes": modes}
    del ws
    return res


def tune_shape(radius, padded_shape):
    """Install the autotuned stencil launch shape for one padded grid."""
    from paper_1603_03971_gb300 import autotune

    choice = autotune.apply(radius, tuple(int(v) for v in padded_shape))
    return ({"zchunk": choice["zchunk"], "variant": choice["variant"],
             "zchunk_modes": choice.get("zchunk_modes", {})} if choice else None)


def grad_leg(dev, autotune=True):
    """The velocity gradient of the data misfit on the gradient_256 workload
    (256^3 smooth random model, 320^3 padded, 1000 steps, checkpoints every
    25): the forward pass (data + checkpoints), then rtm_grad (segment
    recompute writing L u, receiver propagation of the residual correlating
    it). CUDA events around both; per-mode bandwidth from the statistics."""
    import torch

    import paper_1603_03971_gb300 as rtm
    import rtm_inputs

    w = rtm_inputs.WORKLOADS["gradient_256"]
    tuned = tune_shape(w.radius, w.padded_shape) if autotune else None
    p = rtm.params_for(w, want_grad=True)
    ws = rtm.alloc_workspace(p, dev)
    c = rtm.model_prep(p, w.velocity_model(device=dev).contiguous(), ws)
    rec = torch.from_numpy(w.receivers()).to(dev)
    d = torch.empty((w.nt, p.nrec), dtype=torch.float32, device=dev)
    rtm.forward(p, c, rec, ws, data=d)
    resid = 1e-2 * d  # any residual times the same kernels
    rtm.grad(p, c, rec, resid, ws)  # warm-up
    rtm.forward(p, c, rec, ws, data=d)
    torch.cuda.synchronize()
    rtm.reset_stats()
    rtm.set_timing(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    rtm.forward(p, c, rec, ws, data=d)
    ev[1].record()
    g = rtm.grad(p, c, rec, resid, ws)
    ev[2].record()
    torch.cuda.synchronize()
    rtm.set_timing(False)
    st = rtm.stats()
    rtm.check(ws)
    t_f = ev[0].elapsed_time(ev[1]) / 1e3
    t_g = ev[1].elapsed_time(ev[2]) / 1e3
    NZ, NY, NX = w.padded_shape
    updates = 3 * w.nt * NX * NY * NZ
    hbm, _ = measured_peaks()
    modes = {k: {"ms_per_launch": v["ms"] / v["launches"], "gbs": v["bytes"] / v["ms"] / 1e6,
                 "frac": v["bytes"] / v["ms"] / 1e6 / hbm}
             for k, v in st["stencil"].items() if v["launches"] and v["ms"] > 0}
    res = {"workload": "gradient_256: 256^3 smooth random model (320^3 padded), r=4, %d steps, "
                       "checkpoint every %d" % (w.nt, w.ckpt_every),
           "forward_s": t_f, "gradient_s": t_g,
           "gpoint_updates_per_s": updates / (t_f + t_g) / 1e9,
           "gradient_finite": bool(torch.isfinite(g).all()), "stencil_modes": modes,
           "tuning": tuned}
    del ws
    return res


def small_leg(dev):
    """The two-layer 64^3 workload (104^3 padded, 300 steps, store every
    snapshot): a full RTM shot (forward with snapshot writes, receiver
    propagation with imaging) per step, launched directly and replayed from
    one CUDA graph of the same call (the workload is launch-bound: 1202
    launches of about 10 us of work each)."""
    import torch

    import paper_1603_03971_gb300 as rtm
    import rtm_inputs

    w = rtm_inputs.WORKLOADS["two_layer_64"]
    tuned = tune_shape(w.radius, w.padded_shape)
    p = rtm.params_for(w)
    ws = rtm.alloc_workspace(p, dev)
    c = rtm.model_prep(p, torch.from_numpy(w.velocity_model()).float().to(dev).contiguous(), ws)
    rec = torch.from_numpy(w.receivers()).to(dev)
    dobs = torch.empty((w.nt, p.nrec), dtype=torch.float32, device=dev)
    rtm.forward(p, c, rec, ws, data=dobs)
    img = torch.zeros((w.nz, w.ny, w.nx), dtype=torch.float32, device=dev)
    reps = 20
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(3):
        rtm.shot(p, c, rec, dobs, ws, img)
    rtm.check(ws)
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        rtm.shot(p, c, rec, dobs, ws, img)
    ev[1].record()
    torch.cuda.synchronize()
    t_direct = ev[0].elapsed_time(ev[1]) / 1e3 / reps
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rtm.shot(p, c, rec, dobs, ws, img)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        g.replay()
    ev[1].record()
    torch.cuda.synchronize()
    t_graph = ev[0].elapsed_time(ev[1]) / 1e3 / reps
    rtm.check(ws)
    NZ, NY, NX = w.padded_shape
    updates = 2 * w.nt * NX * NY * NZ
    del g
    # the same shot with its source at (32.4, 31.7, 4.5) and the receivers
    # half a cell off the grid on every axis (Kaiser-windowed sinc taps)
    import numpy as np

    xs, ys = np.meshgrid(np.arange(w.nx) + 0.5, np.arange(w.ny) + 0.5, indexing="xy")
    rec_off = np.column_stack([xs.ravel(), ys.ravel(), np.full(xs.size, 2.5)])
    rec_off = rec_off[(rec_off[:, 0] < w.nx - 1) & (rec_off[:, 1] < w.ny - 1)]
    po = p.copy(nrec=len(rec_off))
    wso = rtm.alloc_workspace(po, dev)
    taps = rtm.offgrid_taps(po, (32.4, 31.7, 4.5), rec_off, device=dev)
    d_off = torch.empty((w.nt, po.nrec), dtype=torch.float32, device=dev)
    rtm.forward_offgrid(po, c, taps, wso, data=d_off)
    for _ in range(3):
        rtm.shot_offgrid(po, c, taps, d_off, wso, img)
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        rtm.shot_offgrid(po, c, taps, d_off, wso, img)
    ev[1].record()
    torch.cuda.synchronize()
    rtm.check(wso)
    t_off = ev[0].elapsed_time(ev[1]) / 1e3 / reps
    del ws, wso
    return {"workload": "two_layer_64: 64^3 two-layer model (104^3 padded), r=4, 300 steps, "
                        "15 Hz Ricker, 64x64 receivers, every snapshot stored",
            "shot_s": t_direct, "shot_s_graph": t_graph,
            "gpoint_updates_per_s": updates / t_direct / 1e9,
            "gpoint_updates_per_s_graph": updates / t_graph / 1e9,
            "updates_per_shot": updates, "tuning": tuned,
            "off_grid": {"shot_s": t_off, "gpoint_updates_per_s": updates / t_off / 1e9,
                         "points": "source (32.4, 31.7, 4.5); %d receivers half a cell off "
                                   "the grid in x, y and z (512 taps each)" % len(rec_off)}}


def r8_leg(dev, hbm):
    """The single-shot workload with the radius-8 (16th-order) stencil: 512^3
    smooth random model (576^3 padded), 200 steps, checkpoints every 50, one
    full checkpointed RTM shot; per-mode bandwidth from the live statistics
    against the measured HBM copy rate."""
    import torch

    import paper_1603_03971_gb300 as rtm
    import rtm_inputs

    w = rtm_inputs.WORKLOADS["smooth_512"].scaled(radius=8, nt=200)
    tuned = tune_shape(w.radius, w.padded_shape)
    p = rtm.params_for(w)
    ws = rtm.alloc_workspace(p, dev)
    c = rtm.model_prep(p, w.velocity_model(device=dev).contiguous(), ws)
    rec = torch.from_numpy(w.receivers()).to(dev)
    dobs = torch.empty((w.nt, p.nrec), dtype=torch.float32, device=dev)
    rtm.forward(p, c, rec, ws, data=dobs)
    img = torch.zeros((w.nz, w.ny, w.nx), dtype=torch.float32, device=dev)
    rtm.shot(p, c, rec, dobs, ws, img)  # warm-up
    torch.cuda.synchronize()
    rtm.reset_stats()
    rtm.set_timing(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    rtm.shot(p, c, rec, dobs, ws, img)
    ev[1].record()
    torch.cuda.synchronize()
    rtm.set_timing(False)
    st = rtm.stats()
    rtm.check(ws)
    t = ev[0].elapsed_time(ev[1]) / 1e3
    NZ, NY, NX = w.padded_shape
    modes = {k: {"ms_per_launch": v["ms"] / v["launches"], "gbs": v["bytes"] / v["ms"] / 1e6,
                 "frac": v["bytes"] / v["ms"] / 1e6 / hbm}
             for k, v in st["stencil"].items() if v["launches"] and v["ms"] > 0}
    del ws
    return {"workload": "smooth_512 at radius 8: 512^3 model (576^3 padded), r=8 (16th order), "
                        "200 steps, checkpoint every 50",
            "shot_s": t, "gpoint_updates_per_s": 3 * w.nt * NX * NY * NZ / t / 1e9,
            "stencil_modes": modes, "tuning": tuned}


def decomp_leg(dev, px=2, py=2, nt=200):
    """The single-shot workload's forward modelling (576^3 padded, radius 4,
    200 steps) on a px x py X-Y decomposition with overlapped halo exchange,
    against the same forward pass on one domain (same tile, CUDA events)."""
    import torch

    import paper_1603_03971_gb300 as rtm
    import rtm_inputs

    w = rtm_inputs.WORKLOADS["smooth_512"].scaled(nt=nt)
    tune_shape(w.radius, w.padded_shape)
    p = rtm.params_for(w, storage="all", image_every=nt)
    ws = rtm.alloc_workspace(p, dev)
    c = rtm.model_prep(p, w.velocity_model(device=dev).contiguous(), ws)
    rec = torch.from_numpy(w.receivers()).to(dev)
    data = torch.empty((nt, p.nrec), dtype=torch.float32, device=dev)
    wsd = torch.empty(rtm.decomp_workspace_size(p, px, py), dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        fn()  # warm-up
        torch.cuda.synchronize()
        ev[0].record()
        fn()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 1e3

    t1 = timed(lambda: rtm.forward(p, c, rec, ws, data=data))
    ref = data.clone()
    td = timed(lambda: rtm.forward_decomposed(p, px, py, c, rec, wsd, data=data))
    rtm.check(wsd)
    same = bool(torch.equal(data, ref))
    NZ, NY, NX = w.padded_shape
    del ws, wsd
    return {"workload": "smooth_512 forward modelling, %d steps, %d x %d subdomains" % (nt, px, py),
            "forward_s_one_domain": t1, "forward_s_decomposed": td,
            "gpoint_updates_per_s_decomposed": nt * NX * NY * NZ / td / 1e9,
            "overhead": td / t1 - 1.0, "data_bitwise_equal": same,
            "note": "all subdomains on one GPU; the exchange is device copies on a "
                    "communication stream"}


def batch_leg(args, dev):
    """32 shots on seeded uneven apertures of a 1024 x 1024 x 512 layered /
    salt model, radius-8 stencil, each a full checkpointed RTM, in one
    persistent launch per wave inside one CUDA graph."""
    import torch

    import paper_1603_03971_gb300 as rtm
    import rtm_inputs
    from paper_1603_03971_gb300 import batch as B

    cfg = rtm_inputs.BATCH_WORKLOAD
    nz, ny, nx = cfg["model_shape"]
    nt = args.batch_nt
    vel = torch.from_numpy(rtm_inputs.layered_salt_velocity(nx, ny, nz, seed=cfg["seed"])).to(dev)
    origin, size = rtm_inputs.batch_apertures(cfg["nshots"], (nz, ny, nx), seed=cfg["seed"])
    aps = [B.Aperture(int(o[0]), int(o[1]), int(o[2]), int(s[0]), int(s[1]), int(s[2]),
                      int(s[0]) // 2, int(s[1]) // 2, 4, 2) for o, s in zip(origin, size)]
    if args.batch_shots != "all":  # a subset of the seeded apertures (profiling)
        aps = [aps[int(i)] for i in args.batch_shots.split(",")]
    dt = rtm_inputs.courant_dt(cfg["dx"], cfg["vmax"])
    p = rtm.make_params(nx, ny, nz, cfg["nb"], cfg["radius"], nt, cfg["dx"], dt, cfg["f0"],
                        1.0 / cfg["f0"], (0, 0, 0), 0, storage="ckpt",
                        ckpt_every=args.batch_ckpt)
    budget = 200 * 10 ** 9
    tuned = None
    if args.variant:  # a given kernel variant, automatic slabs
        rtm.set_tuning(p.radius, 0, args.variant)
    elif not args.no_autotune:  # tile rows x slab height, timed on an 8-step run
        from paper_1603_03971_gb300 import autotune

        tuned = autotune.tune_batch(p, aps, vel, nt=8, budget=budget)
        rtm.set_tuning(p.radius, 0, tuned["variant"])
    zchunk = tuned["zchunk"] if tuned else 0
    ws = B.alloc_workspace(p, aps, budget, device=dev)
    dobs = torch.zeros(B.data_size(p, aps), dtype=torch.float32, device=dev)
    img = torch.zeros((nz, ny, nx), dtype=torch.float32, device=dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    B.run(p, aps, vel, dobs, img, ws, budget=budget, zchunk=zchunk)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    rtm.check(ws)
    pts = sum((a.nx + 2 * p.nb) * (a.ny + 2 * p.nb) * (a.nz + 2 * p.nb) for a in aps)
    updates = 3 * nt * pts
    ws_gb = ws.numel() / 1e9
    del ws, dobs
    torch.cuda.empty_cache()
    # the same apertures as single shots, one after another, against the
    # batch over a shorter run: the batch's own rate relative to the
    # single-shot kernel at the apertures' sizes
    same = None
    if args.batch_compare_nt > 0:
        nc = args.batch_compare_nt
        pc = p.copy(nt=nc)
        wsb = B.alloc_workspace(pc, aps, budget, device=dev)
        dc = torch.zeros(B.data_size(pc, aps), dtype=torch.float32, device=dev)
        B.run(pc, aps, vel, dc, img, wsb, budget=budget, zchunk=zchunk)  # warm-up
        torch.cuda.synchronize()
        e0.record()
        B.run(pc, aps, vel, dc, img, wsb, budget=budget, zchunk=zchunk)
        e1.record()
        torch.cuda.synchronize()
        rtm.check(wsb)
        t_b = e0.elapsed_time(e1) / 1e3
        del wsb, dc
        torch.cuda.empty_cache()
        single = []
        for a in aps:
            q = rtm.make_params(a.nx, a.ny, a.nz, p.nb, p.radius, nc, p.dx, p.dt, p.f0, p.t0,
                                (a.src_x, a.src_y, a.src_z), a.nx * a.ny, storage="ckpt",
                                ckpt_every=p.ckpt_every)
            single.append(q)
        ws_s = torch.empty(max(rtm.workspace_size(q) for q in single), dtype=torch.uint8,
                           device=dev)
        cs, recs, ds = [], [], []
        for a, q in zip(aps, single):
            v = vel[a.oz:a.oz + a.nz, a.oy:a.oy + a.ny, a.ox:a.ox + a.nx].contiguous()
            cs.append(rtm.model_prep(q, v, ws_s))
            recs.append(torch.from_numpy(rtm_inputs.surface_receivers(a.nx, a.ny, a.rec_z)).to(dev))
            ds.append(torch.zeros((nc, q.nrec), dtype=torch.float32, device=dev))
        ims = [torch.zeros((a.nz, a.ny, a.nx), dtype=torch.float32, device=dev) for a in aps]
        for q, cc, rr, dd, im in list(zip(single, cs, recs, ds, ims))[:2]:  # warm-up
            rtm.shot(q, cc, rr, dd, ws_s, im)
        torch.cuda.synchronize()
        e0.record()
        for q, cc, rr, dd, im in zip(single, cs, recs, ds, ims):
            rtm.shot(q, cc, rr, dd, ws_s, im)
        e1.record()
        torch.cuda.synchronize()
        rtm.check(ws_s)
        t_s = e0.elapsed_time(e1) / 1e3
        del ws_s, cs, ds, ims
        u_c = 3 * nc * pts
        same = {"steps": nc, "batch_s": t_b, "single_shots_s": t_s,
                "batch_gpoint_updates_per_s": u_c / t_b / 1e9,
                "single_gpoint_updates_per_s": u_c / t_s / 1e9,
                "batch_over_single": t_s / t_b}
    rtm.set_tuning(p.radius, 0, 0)
    shots = ("32 shots" if args.batch_shots == "all"
             else "shots %s of the 32" % args.batch_shots)
    return {"workload": "%s, apertures 128-384 x 128-384 x 256-512 of a 1024x1024x512 "
                        "layered/salt model, r=8, %d steps, checkpoint every %d"
                        % (shots, nt, args.batch_ckpt),
            "seconds": t, "gpoint_updates_per_s": updates / t / 1e9, "updates": updates,
            "workspace_gb": ws_gb, "same_apertures_as_single_shots": same,
            "variant": args.variant or (tuned["variant"] if tuned else 0),
            "tuning": None if tuned is None else {
                "tile_rows": 8 if tuned["variant"] == 3 else 16, "zchunk": tuned["zchunk"],
                "trials_ms": tuned["trials"]}}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1603_03971_gb300 as rtm
    from paper_1603_03971_gb300 import shots

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    w = workload(args)
    cfg = config_of(w)
    NZ, NY, NX = w.padded_shape
    rtm.set_tuning(w.radius, args.zchunk, args.variant)
    cfg["stencil_variant"] = args.variant
    if args.zchunk > 0:
        cfg["zchunk"] = args.zchunk
    elif args.variant == 0 and not args.no_autotune:
        # the library's autotuner: slab height (and plane-load path) for this
        # padded shape, timed on a short checkpointed shot and cached
        cfg["autotune"] = tune_shape(w.radius, w.padded_shape)
    src = shots.shot_source(rank, world, w.nx, w.ny, w.src[2]) if world > 1 else w.src
    p = rtm.params_for(w, src=src)
    rec_np = w.receivers()
    rec = torch.from_numpy(rec_np).to(dev)
    vel = w.velocity_model(device=dev).contiguous()
    vel64 = vel.double().cpu().numpy() if (rank == 0 and world == 1) else None
    ws = rtm.alloc_workspace(p, dev, host_io=True)
    c = rtm.model_prep(p, vel, ws)

    # synthetic observed data: the modelled data of this shot
    dobs = torch.empty((w.nt, p.nrec), dtype=torch.float32, device=dev)
    rtm.forward(p, c, rec, ws, data=dobs)
    rtm.check(ws)
    image = torch.zeros((w.nz, w.ny, w.nx), dtype=torch.float32, device=dev)

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        rtm.shot(p, c, rec, dobs, ws, image)
    rtm.check(ws)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    sampler = ClockSampler(local)
    rtm.reset_stats()
    rtm.set_timing(True)
    sampler.start()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rtm.shot(p, c, rec, dobs, ws, image)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    rtm.set_timing(False)
    st = rtm.stats()
    rtm.check(ws)
    t_local = e0.elapsed_time(e1) / 1e3
    t_max = shots.max_over_ranks(t_local, device=dev)
    updates = cfg["updates_per_shot"]
    value = updates * args.steps * world / t_max / 1e9

    # roofline of the dominant kernel: the backward stencil with fused imaging
    hbm, peak_kind = measured_peaks()
    b = st["stencil"]["bwd_image"]
    launches = b["launches"]
    per_launch_bytes = b["bytes"] / max(launches, 1)
    per_launch_s = b["ms"] / max(launches, 1) / 1e3
    achieved = per_launch_bytes / per_launch_s / 1e9 if per_launch_s > 0 else None
    shares = {k: v["ms"] for k, v in st["stencil"].items() if v["launches"]}
    variant = args.variant or (cfg.get("autotune") or {}).get("variant", 0)
    tile_rows = 8 if variant == 3 else 16
    # slab height of the backward launches: the run's per-mode or general one
    tuned = cfg.get("autotune") or {}
    bwd_zchunk = (args.zchunk or (tuned.get("zchunk_modes") or {}).get("bwd_image")
                  or tuned.get("zchunk"))
    roofline = {
        "kernel": ("k_stencil_tma<%d, MODE_BWD_IMAGE, %d-row tiles>" % (w.radius, tile_rows)
                   if variant != 1 else "k_stencil<%d, MODE_BWD_IMAGE>" % w.radius)
                  + " (backward step + fused zero-lag imaging)",
        "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
        "frac": (achieved / hbm) if achieved else None, "peak_kind": peak_kind,
        "traffic": (profiled_traffic(w.radius, tile_rows, w.padded_shape, bwd_zchunk,
                                     per_launch_bytes) if variant != 1 else None),
        "traffic_slab_planes": bwd_zchunk,
        "algorithmic_bytes_per_launch": per_launch_bytes,
        "launch_ms": per_launch_s * 1e3,
        "stencil_ms_per_step": {k: v / args.steps for k, v in shares.items()},
    }

    # end to end: host buffers through rtm_shot_host
    e2e = None
    if not args.no_e2e:
        v_h = vel.cpu().pin_memory()
        rec_h = torch.from_numpy(rec_np).pin_memory()
        dobs_h = dobs.cpu().pin_memory()
        img_h = torch.empty((w.nz, w.ny, w.nx), dtype=torch.float32).pin_memory()
        rtm.shot_host(p, v_h, rec_h, dobs_h, img_h, ws)
        k_e2e = max(1, min(args.steps, 2))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            rtm.shot_host(p, v_h, rec_h, dobs_h, img_h, ws)
        t_e2e = shots.max_over_ranks(time.perf_counter() - t0, device=dev)
        h2d = v_h.numel() * 4 + rec_h.numel() * 4 + dobs_h.numel() * 4
        e2e = {"value": updates * k_e2e * world / t_e2e / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(img_h.numel() * 4),
               "steps": k_e2e, "s_per_step": t_e2e / k_e2e}
        del v_h, dobs_h

    if world > 1:
        shots.stack_images(image)  # the multi-shot stack (outside the timed region)
    imaging_res = None
    if rank == 0 and args.imaging:
        imaging_res = imaging_leg(p, c, rec, dobs, ws, dev)
    grad_res = None
    if rank == 0 and not args.no_grad:
        grad_res = grad_leg(dev, autotune=args.variant == 0 and not args.no_autotune)
    boundary_res = None
    if rank == 0 and not args.no_boundary:
        ref = image / float(args.warmup + args.steps)  # one shot's checkpoint image
        boundary_res = boundary_leg(w, vel, rec, dobs, dev, ref, t_max / args.steps,
                                    ws.numel() / 1e9,
                                    autotune=args.variant == 0 and not args.no_autotune)
        del ref
    revolve_res = None
    if rank == 0 and args.revolve > 0:
        revolve_res = revolve_leg(w, args.revolve, vel, rec, dobs, dev)
    del vel
    learned = None
    if rank == 0 and not args.no_learned:
        del ws
        torch.cuda.empty_cache()
        learned = learned_leg(args, dev)
        ws = None
    batch_res = None
    if rank == 0 and not args.no_batch:
        ws = None
        torch.cuda.empty_cache()
        batch_res = batch_leg(args, dev)
    small_res = None
    if rank == 0 and not args.no_small:
        ws = None
        torch.cuda.empty_cache()
        small_res = small_leg(dev)
    decomp_res = None
    if rank == 0 and not args.no_decomp:
        ws = None
        torch.cuda.empty_cache()
        decomp_res = decomp_leg(dev)
    r8_res = None
    if rank == 0 and not args.no_r8:
        ws = None
        torch.cuda.empty_cache()
        r8_res = r8_leg(dev, hbm)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ws = None
        torch.cuda.empty_cache()
        steps = 20
        s, u, threads = oracle_sample(w, vel64, steps)
        cpu = {"value": u / s / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d forward time steps of the FP64 oracle on the %dx%dx%d padded "
                         "grid (%.1f s), allocation and first touch excluded (a %d-step run "
                         "minus a 3-step run)" % (steps, NX, NY, NZ, s, steps + 3),
               "cpu": cpu_model()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded smooth random velocity; observed data modelled on it)",
            "config": cfg, "shot_s": t_max / args.steps, "roofline": roofline,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": st["launches"],
            "clocks": clocks, "impl": "ours", "learned": learned, "batch": batch_res,
            "two_layer_64": small_res, "radius8": r8_res, "decomposition": decomp_res,
            "imaging": imaging_res, "revolve": revolve_res, "boundary": boundary_res,
            "gradient": grad_res,
            # the paper's own reported improvements (relative speedups of a CPU
            # cluster code; context only, not comparable and not a target)
            "paper_context": {
                "copy_removal": "~10% faster (memcpy was 7% of execution)",
                "overall": "~30% faster",
                "hardware": "16 MPI ranks x 8 OpenMP threads on 8 multicore CPU nodes, "
                            "X-Y decompositions 4x4 and 2x8",
            },
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
