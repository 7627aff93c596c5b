#!/usr/bin/env python3
"""Throughput of the batched mixed-state multislice forward + adjoint.

One step = one gradient-descent iteration (ptycho_step) over one group of
scan positions: probe spectra, forward model through every slice, noise-model
loss, adjoint with the per-slice entry waves recomputed, object/probe
gradient reduction and the Adam update (arXiv 2505.14372 §3, §3.1, §3.2).

Default workload: 20 slices x 8 incoherent modes, 192x192 window,
1024x1024 object, 128x128 raster scan (16384 positions), groups of 512,
Poisson noise model, entry waves recomputed in the backward pass.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                    [--workload 1|2|3] [--waves recompute|store] [--no-baseline]

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica on its own GPU (the path has no exchange step), timing is the max over
ranks, and `value` counts the positions of all ranks.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+adjoint probe-positions/s (multislice, mixed-state); p50/p99 serve latency"
FP32_LANES_PER_SM = 128
# what the geometry's waves modes mean for the step: "recompute" runs the
# forward pass inside the adjoint kernel and keeps every slice's entry wave of
# the positions in flight in per-cluster HBM slots (4S 2-D FFTs per mode, no
# slice recomputed twice); "store" keeps the whole group's entry waves
WAVES_LABEL = {"recompute": "slot-stored (forward inside the adjoint kernel; entry waves of the positions in "
                            "flight in per-cluster HBM slots)",
               "store": "stored (the whole group's entry waves from a separate forward launch)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", type=int, default=3, choices=[1, 2, 3])
    ap.add_argument("--waves", default="recompute", choices=["recompute", "store"])
    ap.add_argument("--wave-prec", default="f32", choices=["f32", "f16", "bf16"],
                    help="storage format of the entry-wave copies read by the object gradient")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the single-slice workloads measured beside the headline line")
    ap.add_argument("--dft", default="fft", choices=["fft", "tf32x3", "bf16x3", "tf32", "bf16x6"],
                    help="DFT evaluation inside the tile (tensor-core variants: 192x192 window)")
    ap.add_argument("--e2e-steps", type=int, default=0, help="steps of the host-buffer leg (default: --steps, at most 10)")
    ap.add_argument("--serve", action="store_true",
                    help="serving mode: seeded Poisson arrivals of mixed-shape requests through ptycho_submit")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--iterations", type=int, default=50, help="iterations per served request")
    ap.add_argument("--max-scan", type=int, default=128, help="largest scan side of a served request")
    ap.add_argument("--rate", type=float, default=16.0, help="mean request arrivals per second")
    ap.add_argument("--max-active", type=int, default=4,
                    help="requests resident at once in the batched arm (0: all); 4 keeps the device within 1 %% "
                         "as busy as all 64 do, with iterations 6x faster at the tail")
    ap.add_argument("--skip-alone", action="store_true", help="serve: skip the one-at-a-time arm")
    ap.add_argument("--dft-micro", action="store_true",
                    help="time the DFT evaluations (FFT tile, warp-level tensor-core tiles, tcgen05 row GEMM) on "
                         "batches of 192 x 192 waves")
    ap.add_argument("--waves-count", type=int, default=512, help="waves per batch of --dft-micro")
    ap.add_argument("--paper-context", action="store_true",
                    help="seconds per full iteration of the paper-shaped case (80x80 scan, 20 slices, 128^2, 1 mode)")
    ap.add_argument("--precision", action="store_true",
                    help="relative L2 error of every DFT mode against the FP64 oracle on a 4-position sub-problem")
    ap.add_argument("--graph", action="store_true",
                    help="gradient engine: capture one step in a CUDA graph and replay it per step "
                         "(Adam step count in device memory; for launch-bound small workloads)")
    ap.add_argument("--engine", default="gd", choices=["gd", "epie", "lsqml"],
                    help="gd: gradient descent with Adam (ptycho_step); epie: the ePIE / 3PIE update "
                         "(ptycho_epie_step); lsqml: the LSQML update (ptycho_lsqml_step); the last two use "
                         "the amplitude noise model")
    ap.add_argument("--positions", type=int, default=0,
                    help="use only the first P scan positions (small profiling cases; the line says so)")
    ap.add_argument("--group", type=int, default=0,
                    help="override the group size (small cases for profiling; not a bench line)")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def workload_geometry(wl, waves, dft="fft", wave_prec="f32"):
    from paper_2505_14372_b300 import Geometry
    return Geometry(S=wl.S, K=wl.K, N=wl.N, H=wl.H, W=wl.W, dx=wl.dx, lam=wl.lam, dz=wl.dz,
                    bandlimit=wl.bandlimit, loss={0: "amplitude", 1: "poisson"}[wl.loss],
                    eps=wl.eps, c=wl.c, waves=waves, dft=dft, wave_prec=wave_prec)


def config_dict(wl, waves, dft="fft", wave_prec="f32"):
    return {"workload": wl.name, "dft": dft, "wave_storage": wave_prec, "slices": wl.S, "modes": wl.K, "window": wl.N, "object": [wl.H, wl.W],
            "positions": wl.P, "group": wl.B, "loss": {0: "amplitude", 1: "poisson"}[wl.loss],
            "waves": WAVES_LABEL.get(waves, waves), "grouping": "sparse, reshuffled every pass",
            "l2": "inputs larger than L2 (patterns %.1f GB, object %.0f MB) - no flush" % (
                wl.P * wl.N * wl.N * 4 / 1e9, wl.S * wl.H * wl.W * 8 / 1e6)}


def kernel_source_hash(N):
    """Hash of the sources the tile kernels of window N are built from (the
    shared headers and that window's instantiation unit)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2505_14372_b300", "csrc")
    for name in ("radix.cuh", "check.cuh", "tile.cuh", "kernels.cuh", "elementwise.cuh", "noise.cuh", "launch.h",
                 "engine_impl.cuh", f"tile{N}.cu"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def max_over_ranks(x, world, device):
    """The largest value of x over all ranks (the job's time is its slowest
    rank's): an all-reduce MAX, a no-op for one rank."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units every rank processed over the job's time."""
    return world * units_per_rank / seconds


def fft_flops(NP):
    return 5.0 * NP * math.log2(NP)


def adjoint_algorithmic_flops(wl, items, recompute):
    """Algorithmic FLOPs of one adjoint-kernel launch over `items` (position,
    mode) pairs: 5 NP log2 NP per 2-D FFT (2S for the backward chain, plus 2S
    for the forward recomputed inside it) and 6 per complex product of the
    pointwise steps."""
    NP = wl.N * wl.N
    S = wl.S
    ffts = (2 * S if recompute else 0) + 2 * S
    # pointwise complex products per element: forward recompute: shift ramp 2,
    # transmission S, propagator 2(S-1), seed 1; backward: object gradient S,
    # conj(O) S, propagator 2(S-1), probe ramp 2
    prods = (2 + S + 2 * (S - 1) + 1 if recompute else 1) + S + S + 2 * (S - 1) + 2
    return items * (ffts * fft_flops(NP) + prods * 6.0 * NP)


def hbm_algorithmic_bytes(wl):
    """Algorithmic HBM bytes of one position's forward + adjoint: the object
    patch read in the forward and again in the adjoint (S N^2 8 each), the
    measured pattern (N^2 4) and the object-gradient read-modify-write
    (S N^2 16); probe and tables stay in L2."""
    NP = wl.N * wl.N
    return wl.S * NP * 8 * 2 + NP * 4 + wl.S * NP * 16


def workload_leg(wl_id, steps, warmup, dev, fp32_peak_tf, hbm_gbs):
    """Device-timed steps of another workload of the path (one group per
    step, Adam included, inputs resident), with its tile kernel's share, its
    ALU and HBM roofline fractions; reported beside the headline line."""
    import torch
    from paper_2505_14372_b300 import AdamState, Context, adam_opt, make_groups, synth
    wl = synth.WORKLOADS[wl_id]
    B = wl.B
    geom = workload_geometry(wl, "recompute")
    P_np = synth.probe_modes(wl)
    Pd = torch.from_numpy(P_np).to(dev)
    Od = torch.ones((wl.S, wl.H, wl.W), dtype=torch.complex64, device=dev)
    pos_d = torch.from_numpy(synth.raster_positions(wl)).to(dev)
    Iexp_d = synth.cbed_like_patterns_device(wl, wl.P, device=dev)
    order = np.concatenate([make_groups(wl.P, B, seed=77, iteration=it, mode="sparse")
                            for it in range(max(1, 64 * B // wl.P))])
    ng = len(order) // B
    idx = torch.from_numpy(order.astype(np.int32)).to(dev)
    ctx = Context(geom, max_batch=B)
    st = AdamState(geom, device=dev)
    opt = adam_opt(lr_O=1e-3, lr_P=1e-4)
    stats = torch.zeros(2, dtype=torch.float64, device=dev)
    # warm-up by time, not by count: after an idle gap of a second or two the
    # GPU's clocks take a while to return (a 64 x 64 step measured 58 us
    # warm and 127 us right after a 2 s pause), so steps of tens of us need
    # a few hundred ms of work before they are timed
    t_w = time.perf_counter()
    i = 0
    while i < warmup or time.perf_counter() - t_w < 0.5:
        j = i % ng
        ctx.step(Od, Pd, st, opt, pos_d, Iexp_d, idx[j * B:(j + 1) * B], stats=stats)
        i += 1
        if i % 64 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(steps):
        j = (warmup + i) % ng
        ctx.step(Od, Pd, st, opt, pos_d, Iexp_d, idx[j * B:(j + 1) * B], stats=stats)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # the tile kernel alone, in separate steps with its launches bracketed
    ctx.set_timing(2)
    ctx.kernel_times(reset=True)
    for i in range(steps):
        j = (warmup + i) % ng
        ctx.step(Od, Pd, st, opt, pos_d, Iexp_d, idx[j * B:(j + 1) * B], stats=stats)
    torch.cuda.synchronize()
    kt = ctx.kernel_times()
    ctx.set_timing(False)
    ctx.check_status()
    ctx.close()
    tile_ms = kt["adjoint"][0] / kt["adjoint"][1]
    flops = adjoint_algorithmic_flops(wl, B * wl.K, True)
    nbytes = hbm_algorithmic_bytes(wl) * B
    return {"workload": wl.name, "positions_per_s": B / (ms / 1e3), "ms_per_step": ms, "steps": steps,
            "warmup": warmup, "group": B, "loss": {0: "amplitude", 1: "poisson"}[wl.loss],
            "tile_kernel_ms": tile_ms, "tile_share_of_step": tile_ms / ms,
            "roofline_alu": {"achieved_tflops": flops / (tile_ms / 1e3) / 1e12, "peak_tflops": fp32_peak_tf,
                             "frac": flops / (tile_ms / 1e3) / 1e12 / fp32_peak_tf,
                             "note": "tile kernel's nominal FFT flops over its launch time, of the measured FP32 peak"},
            "roofline_hbm": {"algorithmic_bytes_per_position": hbm_algorithmic_bytes(wl),
                             "achieved_gbs_step": nbytes / (ms / 1e3) / 1e9, "peak_gbs": hbm_gbs,
                             "frac_step": nbytes / (ms / 1e3) / 1e9 / hbm_gbs,
                             "note": "algorithmic bytes of a whole step over the step time, of the measured copy "
                                     "bandwidth (the object and patterns of this workload fit in L2)"}}


def host_buffer_order(order, used_groups, steps, P, B):
    """Positions of the host-buffer leg: the groups after the `used_groups`
    of the device-timed leg, else fresh passes; every step a full group of B."""
    from paper_2505_14372_b300 import make_groups
    h = order[used_groups * B:][: steps * B]
    if len(h) < steps * B:
        h = np.concatenate([make_groups(P, B, seed=99, iteration=it, mode="sparse")
                            for it in range(math.ceil(steps * B / P) + 1)])[: steps * B]
    assert len(h) == steps * B, "every host-buffer step carries a full group"
    return h


def cpu_oracle_leg(wl, geom, pos_all_np, n_pos_sample, O_init, P_np, sample_note, min_seconds=10.0, max_steps=200):
    """Times the FP64 oracle's steps on a bounded sample of the workload:
    consecutive steps of n_pos_sample positions each, until about
    min_seconds of CPU work (at most max_steps steps)."""
    import oracle as orc
    og = orc.Geom(S=wl.S, K=wl.K, h=wl.N, w=wl.N, H=wl.H, W=wl.W, dx=wl.dx, lam=wl.lam, dz=wl.dz,
                  bandlimit=wl.bandlimit, loss=wl.loss, eps=wl.eps, c=wl.c)
    from paper_2505_14372_b300 import synth
    idx = np.arange(n_pos_sample)
    E = synth.cbed_like_patterns(wl, n_pos_sample)
    O = O_init.astype(np.complex128)
    P = P_np.astype(np.complex128)
    mO, vO, mP, vP = np.zeros_like(O), np.zeros(O.shape), np.zeros_like(P), np.zeros(P.shape)
    npos = len(pos_all_np)
    dt, steps = 0.0, 0
    while dt < min_seconds and steps < max_steps:
        first = (steps * n_pos_sample) % max(npos - n_pos_sample + 1, 1)
        t0 = time.perf_counter()
        O, P, mO, vO, mP, vP, _, _ = orc.step(O, P, mO, vO, mP, vP, steps + 1,
                                              pos_all_np[first:first + n_pos_sample], E, idx, og, 1e-3, 1e-4)
        dt += time.perf_counter() - t0
        steps += 1
    return {"value": steps * n_pos_sample / dt, "unit": "positions/s", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle", "sample": f"{steps} {sample_note}", "seconds": dt}


def run_reference(args, wl, rank):
    """Reference arm: the FP64 oracle as it stands, on the host cores."""
    if rank != 0:
        return
    from paper_2505_14372_b300 import synth
    P_np = synth.probe_modes(wl)
    pos = synth.raster_positions(wl).astype(np.float64)
    O_init = np.ones((wl.S, wl.H, wl.W), np.complex64)
    per_step = 2 if wl.S > 1 else 16
    note = (f"{per_step} positions x {wl.K} modes x {wl.S} slices per step (all slices and modes of the "
            f"workload, object {wl.H}x{wl.W}), FP64 dense-DFT oracle incl. Adam on the full object")
    import oracle as orc
    og = orc.Geom(S=wl.S, K=wl.K, h=wl.N, w=wl.N, H=wl.H, W=wl.W, dx=wl.dx, lam=wl.lam, dz=wl.dz,
                  bandlimit=wl.bandlimit, loss=wl.loss, eps=wl.eps, c=wl.c)
    E = synth.cbed_like_patterns(wl, per_step * (args.steps + args.warmup))
    O = O_init.astype(np.complex128)
    P = P_np.astype(np.complex128)
    mO, vO = np.zeros_like(O), np.zeros(O.shape)
    mP, vP = np.zeros_like(P), np.zeros(P.shape)
    t = 0
    elapsed = 0.0
    for it in range(args.warmup + args.steps):
        sl = slice(it * per_step, (it + 1) * per_step)
        idx = np.arange(per_step)
        t0 = time.perf_counter()
        t += 1
        O, P, mO, vO, mP, vP, _, _ = orc.step(O, P, mO, vO, mP, vP, t, pos[sl], E[sl], idx, og, 1e-3, 1e-4)
        if it >= args.warmup:
            elapsed += time.perf_counter() - t0
    value = per_step * args.steps / elapsed
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "positions/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(wl, args.waves),
            "cpu_baseline": {"value": value, "unit": "positions/s", "cores": cores, "kind": "oracle",
                             "sample": note},
            "e2e": {"value": value, "unit": "positions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serve_requests(args):
    """Seeded mixed-shape requests: scan side 32..max_scan at 3 px steps,
    window 64/128/192/256, 1-30 slices, 1-8 modes, object = scan extent +
    window + 4 px, Poisson-noise CBED-like patterns, Poisson arrival times."""
    from paper_2505_14372_b300 import synth
    rng = np.random.default_rng(5000)
    out = []
    t = 0.0
    for i in range(args.requests):
        t += rng.exponential(1.0 / args.rate)
        n = int(rng.integers(32, args.max_scan + 1))
        N = int(rng.choice([64, 128, 192, 256]))
        S = int(rng.integers(1, 31))
        K = int(rng.integers(1, 9))
        side = (n - 1) * 3 + N + 4
        wl = synth.Workload(5000 + i, f"served {i}", S=S, K=K, N=N, H=side, W=side, scan=(n, n), step_px=3.0,
                            B=128, loss=1, eps=0.8, c=0.0, dose=5e4, alpha_mrad=24.0, defocus_A=50.0, C3_A=1e4,
                            weights=tuple(np.exp(-np.arange(K)) / np.exp(-np.arange(K)).sum()))
        out.append((t, wl))
    return out


def request_data(wl):
    from paper_2505_14372_b300 import synth
    P = synth.probe_modes(wl)
    pos = synth.raster_positions(wl)
    pool = synth.cbed_like_patterns(wl, 8)
    I = np.ascontiguousarray(np.resize(pool, (wl.P, wl.N, wl.N)))
    return P, pos, I


def run_serve(args):
    import threading
    import torch
    from paper_2505_14372_b300 import Server, adam_opt
    torch.cuda.set_device(0)
    reqs = serve_requests(args)
    budget = 150 * (1 << 30)
    opt = adam_opt(1e-3, 1e-4)

    def submit(srv, wl):
        P, pos, I = request_data(wl)
        geom = workload_geometry(wl, "recompute")
        return srv.submit(geom, pos, I, P, iterations=args.iterations, batch=wl.B, seed=wl.cid, opt=opt)

    # continuous batching: requests arrive on their own schedule
    srv = Server(budget, max_active=args.max_active or args.requests)
    tickets = []
    t0 = time.perf_counter()  # the server's clock started just before
    for t_arr, wl in reqs:
        dt = t_arr - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tickets.append(submit(srv, wl))
    for tk in tickets:
        srv.wait(tk, 3600e3)
    wall = time.perf_counter() - t0
    st = srv.stats()
    positions = sum(wl.P * args.iterations for _, wl in reqs)

    def latency(d):
        d = np.asarray(d)
        return {"p50_ms": float(np.percentile(d, 50)), "p99_ms": float(np.percentile(d, 99)),
                "mean_ms": float(d.mean())}

    # scheduled arrival -> finish of every request (the server's clock starts
    # with t0), queueing included
    done_ms = [srv.poll(t)["finish_ms"] for t in tickets]
    served = {"positions_per_s_wall": positions / wall, "positions_per_s_device": st["positions_per_s"],
              "p50_iter_ms": st["p50_iter_ms"], "p99_iter_ms": st["p99_iter_ms"], "wall_s": wall,
              "request_latency": latency([f - 1e3 * ta for f, (ta, _) in zip(done_ms, reqs)]),
              "launches": st["launches"], "failed": st["failed"]}
    srv.close()
    if args.skip_alone:
        line = {"metric": METRIC, "mode": "serve", "value": served["positions_per_s_wall"], "unit": "positions/s",
                "p50_iter_ms": served["p50_iter_ms"], "p99_iter_ms": served["p99_iter_ms"], "n_gpus": 1,
                "higher_is_better": True, "dtype": "f32", "data": "synthetic", "served": served,
                "config": {"requests": args.requests, "max_active": args.max_active or args.requests,
                           "iterations_per_request": args.iterations, "scan_sides": [32, args.max_scan],
                           "arrival_rate_per_s": args.rate}}
        print(json.dumps(line), flush=True)
        return 0
    # the same requests one at a time on the same arrival schedule: each is
    # submitted once it has arrived and the one before it is done (first
    # come, first served; only one request's data held at a time)
    srv = Server(budget, max_active=1)
    done1 = []
    t0 = time.perf_counter()
    for t_arr, wl in reqs:
        dt = t_arr - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tk = submit(srv, wl)
        srv.wait(tk, 3600e3)
        done1.append(1e3 * (time.perf_counter() - t0 - t_arr))
    wall1 = time.perf_counter() - t0
    st1 = srv.stats()
    one = {"positions_per_s_wall": positions / wall1, "positions_per_s_device": st1["positions_per_s"],
           "p50_iter_ms": st1["p50_iter_ms"], "p99_iter_ms": st1["p99_iter_ms"], "wall_s": wall1,
           "request_latency": latency(done1), "failed": st1["failed"]}
    srv.close()
    shapes = [(wl.P, wl.N, wl.S, wl.K) for _, wl in reqs]
    line = {"metric": METRIC, "mode": "serve", "value": served["positions_per_s_wall"], "unit": "positions/s",
            "p50_iter_ms": served["p50_iter_ms"], "p99_iter_ms": served["p99_iter_ms"], "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "served": served, "one_at_a_time": one,
            "config": {"workload": "serving: Poisson arrivals of mixed-shape reconstruction requests",
                       "requests": args.requests, "arrival_rate_per_s": args.rate,
                       "max_active": args.max_active or args.requests,
                       "iterations_per_request": args.iterations, "scan_sides": [32, args.max_scan],
                       "windows": [64, 128, 192, 256], "slices": [1, 30], "modes": [1, 8], "group": 128,
                       "hbm_budget_GB": 150, "positions_total": positions,
                       **({} if args.iterations == 50 and args.max_scan == 128 else
                          {"scaled_from": "50 iterations and scans up to 128x128 per request"}),
                       "shapes": shapes}}
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args):
    """Errors of intensities, loss and gradients against the FP64 oracle for
    each DFT evaluation mode, on four neighbouring scan positions of the
    workload (all slices and modes, full window; object cropped around them)."""
    import torch
    import oracle as orc
    from paper_2505_14372_b300 import Context, synth
    torch.cuda.set_device(0)
    wl = synth.WORKLOADS[args.workload]
    ny = wl.scan[1]
    P = synth.probe_modes(wl)
    pos = synth.raster_positions(wl)[[0, 1, ny, ny + 1]].astype(np.float64)
    org = np.floor(pos.min(0)).astype(int) - 1
    pos = (pos - org).astype(np.float32)
    import dataclasses
    small = dataclasses.replace(wl, H=wl.N + 8, W=wl.N + 8, atoms_per_slice=max(4, wl.atoms_per_slice // 20))
    O = synth.phase_object(small)
    E = synth.cbed_like_patterns(wl, 4)
    og = orc.Geom(S=wl.S, K=wl.K, h=wl.N, w=wl.N, H=small.H, W=small.W, dx=wl.dx, lam=wl.lam, dz=wl.dz,
                  bandlimit=wl.bandlimit, loss=wl.loss, eps=wl.eps, c=wl.c)
    rI = orc.forward(O, P, pos, og)
    L, rO, rP = orc.gradient(O, P, pos, E, og)
    rel = lambda a, b: float(np.linalg.norm((np.asarray(a, np.complex128) - b).ravel()) / np.linalg.norm(b.ravel()))
    out = {}
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for mode in (["fft", "tf32x3", "bf16x3", "tf32", "bf16x6"] if wl.N == 192 else ["fft"]):
        geom = workload_geometry(small, args.waves, mode)
        ctx = Context(geom, max_batch=4)
        I = ctx.forward(d(O), d(P), d(pos)).cpu().numpy()
        loss, gO, gP = ctx.adjoint(d(O), d(P), d(pos), d(E))
        ctx.check_status()
        out[mode] = {"I": rel(I, rI), "loss": abs(float(loss.item()) - L) / abs(L),
                     "gO": rel(gO.cpu().numpy(), rO), "gP": rel(gP.cpu().numpy(), rP)}
        ctx.close()
    # 16-bit entry-wave storage (FFT tile): errors against the unrounded
    # oracle (the accuracy given up) and the oracle rounding the same copies
    for prec in ("f16", "bf16"):
        geom = workload_geometry(small, args.waves, "fft", prec)
        ctx = Context(geom, max_batch=4)
        loss, gO, gP = ctx.adjoint(d(O), d(P), d(pos), d(E))
        ctx.check_status()
        _, rOr, _ = orc.gradient(O, P, pos, E, og, wave_fmt=prec)
        out["fft, " + prec + " entry waves"] = {"loss": abs(float(loss.item()) - L) / abs(L),
                                                "gO": rel(gO.cpu().numpy(), rO), "gP": rel(gP.cpu().numpy(), rP),
                                                "gO_vs_rounding_oracle": rel(gO.cpu().numpy(), rOr)}
        ctx.close()
    print(json.dumps({"mode": "precision", "metric": "relative L2 error against the FP64 oracle",
                      "config": {"workload": wl.name, "positions": "4 neighbouring raster positions",
                                 "object": [small.H, small.W], "waves": args.waves},
                      "errors": out}), flush=True)
    return 0


def run_paper_context(args):
    """Seconds per full iteration (every scan position once, groups of 512,
    Adam steps) of the paper-shaped multislice case: 80 x 80 scan, 20 slices,
    128 x 128 window, one mode.  The paper reports under 3 s per iteration
    for this scan size, slice count and window on an RTX 3080 (context, not
    a target: another machine, and its mode count is not stated)."""
    import torch
    from paper_2505_14372_b300 import AdamState, Context, adam_opt, make_groups, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wl = synth.PAPER_CONTEXT
    B = wl.B
    geom = workload_geometry(wl, "recompute")
    Pd = torch.from_numpy(synth.probe_modes(wl)).to(dev)
    Od = torch.ones((wl.S, wl.H, wl.W), dtype=torch.complex64, device=dev)
    pos_d = torch.from_numpy(synth.raster_positions(wl)).to(dev)
    Iexp_d = synth.cbed_like_patterns_device(wl, wl.P, device=dev)
    ctx = Context(geom, max_batch=B)
    st = AdamState(geom, device=dev)
    opt = adam_opt(lr_O=1e-3, lr_P=1e-4)
    stats = torch.zeros(2, dtype=torch.float64, device=dev)

    def iteration(it):
        perm = torch.from_numpy(make_groups(wl.P, B, seed=6, iteration=it, mode="sparse").astype(np.int32)).to(dev)
        for g0 in range(0, wl.P, B):
            ctx.step(Od, Pd, st, opt, pos_d, Iexp_d, perm[g0:g0 + B], stats=stats)

    for it in range(max(args.warmup, 1)):
        iteration(it)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(args.steps, 1)
    e0.record()
    for it in range(n):
        iteration(args.warmup + it)
    e1.record()
    torch.cuda.synchronize()
    ctx.check_status()
    s_per_iter = e0.elapsed_time(e1) / 1e3 / n
    print(json.dumps({"mode": "paper-context", "metric": "seconds per full iteration", "value": s_per_iter,
                      "unit": "s/iteration", "positions_per_s": wl.P / s_per_iter, "iterations": n,
                      "config": {"workload": wl.name, "positions": wl.P, "group": B, "slices": wl.S, "modes": wl.K,
                                 "window": wl.N, "object": [wl.H, wl.W]},
                      "paper": "under 3 s per iteration, 80x80 scan, 20 slices, 128x128 patterns, JAX on one "
                               "RTX 3080 (§4.1; mode count not stated)"}), flush=True)
    return 0


def run_dft_micro(args):
    """The DFT evaluations side by side on batches of N x N waves: the FFT
    tile and the warp-level tensor-core tiles (2-D transforms, ptycho_fft2_dft)
    and the tcgen05 row-DFT GEMM (ptycho_dft_rows_tc, one 1-D pass over the
    rows of every wave).  Times per wave and per 1-D pass (half a 2-D
    transform), CUDA events, best of the timed repeats; the tcgen05 GEMM's
    tensor rate against the measured bf16 peak (tf32 at half of it, the
    nominal ratio)."""
    import torch
    from paper_2505_14372_b300.api import dft_rows_tc, dft_rows_tc_check, fft2_dft
    torch.cuda.set_device(0)
    N, count = 192, args.waves_count
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    x = torch.complex(torch.randn((count, N, N), generator=g, device="cuda"),
                      torch.randn((count, N, N), generator=g, device="cuda")).contiguous()
    peaks, src = measured_peaks()

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    out = {}
    for dft in ("fft", "tf32x3", "bf16x3", "tf32", "bf16x6"):
        ms = timed(lambda: fft2_dft(x, dft))
        out[f"tile {dft} (2-D)"] = {"ms": ms, "us_per_wave_2d": 1e3 * ms / count,
                                    "us_per_wave_pass": 0.5e3 * ms / count}
    y = torch.empty_like(x)
    for mode in ("tf32x3", "bf16x3", "tf32"):
        ms = timed(lambda: dft_rows_tc(x, mode, out=y))
        prods = 1 if mode == "tf32" else 3
        flops = 2.0 * count * N * (2 * N) * (2 * N) * prods
        peak = peaks["bf16_tflops"] * (0.5 if mode.startswith("tf32") else 1.0)
        out[f"tcgen05 rows {mode} (1-D)"] = {"ms": ms, "us_per_wave_pass": 1e3 * ms / count,
                                            "tensor_tflops": flops / (ms / 1e3) / 1e12, "peak_tflops": peak,
                                            "frac": flops / (ms / 1e3) / 1e12 / peak}
    torch.cuda.synchronize()
    dft_rows_tc_check()
    print(json.dumps({"mode": "dft-micro", "config": {"N": N, "waves": count, "peak_source": f"{src} bf16"},
                      "results": out}), flush=True)
    return 0


def main():
    args = parse()
    if args.dft_micro:
        return run_dft_micro(args)
    if args.paper_context:
        return run_paper_context(args)
    if args.serve:
        return run_serve(args)
    if args.precision:
        return run_precision(args)
    from paper_2505_14372_b300 import synth
    wl = synth.WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return 0

    import torch
    import torch.distributed as dist
    from paper_2505_14372_b300 import AdamState, Context, adam_opt, kernels_launched, make_groups

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    if args.group:
        import dataclasses
        wl = dataclasses.replace(wl, B=args.group)
    if args.positions:  # fewer raster rows, same object and window
        import dataclasses
        nx = wl.scan[1]
        wl = dataclasses.replace(wl, scan=(max(1, min(args.positions, wl.P) // nx), nx))
    geom = workload_geometry(wl, args.waves, args.dft, args.wave_prec)
    if args.engine in ("epie", "lsqml"):  # their modulus update belongs to the amplitude model
        geom.loss, geom.eps, geom.c = "amplitude", 1e-3, 0.0
    B = wl.B

    # ---- inputs resident in HBM
    P_np = synth.probe_modes(wl)
    pos_np = synth.raster_positions(wl)
    Pd = torch.from_numpy(P_np).to(dev)
    Od = torch.ones((wl.S, wl.H, wl.W), dtype=torch.complex64, device=dev)
    pos_d = torch.from_numpy(pos_np).to(dev)
    Iexp_d = synth.cbed_like_patterns_device(wl, wl.P, device=dev)
    ngroups = wl.P // B
    order = []
    for it in range(math.ceil((args.warmup + args.steps) / ngroups) + 1):
        order.append(make_groups(wl.P, B, seed=1234 + rank, iteration=it, mode="sparse"))
    order = np.concatenate(order)
    idx_all = torch.from_numpy(order.astype(np.int32)).to(dev)

    ctx = Context(geom, max_batch=B)
    st = AdamState(geom, device=dev)
    opt = adam_opt(lr_O=1e-3, lr_P=1e-4)
    stats = torch.zeros(2, dtype=torch.float64, device=dev)

    def group(i):
        return idx_all[i * B:(i + 1) * B]

    lsq = dict(beta_O=0.5, beta_P=0.5, delta_O=1e-2, delta_P=1e-2, gamma=1e-6)

    def one_step(i):
        if args.engine == "epie":
            ctx.epie_step(Od, Pd, pos_d, Iexp_d, group(i), beta_O=0.5, beta_P=0.5, loss=stats[:1])
        elif args.engine == "lsqml":
            ctx.lsqml_step(Od, Pd, pos_d, Iexp_d, group(i), loss=stats[:1], **lsq)
        else:
            ctx.step(Od, Pd, st, opt, pos_d, Iexp_d, group(i), stats=stats)

    for i in range(args.warmup):
        one_step(i)
    torch.cuda.synchronize()
    ctx.check_status()
    if world > 1:
        dist.barrier()
    # per-launch CUDA events around the tile kernels only (events around
    # every short kernel would stretch the step of small problems by ~20 %)
    ctx.set_timing(2)
    ctx.kernel_times(reset=True)
    graph_launches = 0
    if args.graph and args.engine == "gd":
        # one step captured (with its per-kernel timing events), replayed per
        # step on the group copied into a fixed index buffer; the Adam step
        # count continues in device memory from the warm-up steps
        t_dev = torch.full((1,), st.t, dtype=torch.int64, device=dev)
        ctx.set_step_counter(t_dev)
        idx_buf = torch.empty(B, dtype=torch.int32, device=dev)
        kc = kernels_launched()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            ctx.step(Od, Pd, st, opt, pos_d, Iexp_d, idx_buf, stats=stats)
        graph_launches = kernels_launched() - kc

        def one_step(i):  # noqa: F811 - the replayed step
            idx_buf.copy_(group(i))
            graph.replay()
    # FP32 CUDA-core peak of this GPU (FFMA / FFMA2 microbenchmark), with
    # the SM clock it ran at: the denominator of the tile kernel's roofline
    from paper_2505_14372_b300.api import fp32_peak
    psamp = ClockSampler(local)
    psamp.start()
    peak_meas = fp32_peak()
    peak_meas["clocks"] = psamp.stop()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    k0 = kernels_launched()
    # one event between consecutive steps: the first and last bracket the
    # timed region, the others give the per-step spread
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0, e1 = evs[0], evs[-1]
    torch.cuda.synchronize()
    e0.record()
    for i in range(args.steps):
        one_step(args.warmup + i)
        evs[i + 1].record()
    torch.cuda.synchronize()
    launches = kernels_launched() - k0 + graph_launches * args.steps
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    step_ms = np.array([evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)])
    ctx.check_status()
    ktimes = ctx.kernel_times()
    ctx.set_timing(False)
    if graph_launches:
        # the captured timing events hold the last replay: per-step figures
        ktimes = {k: (v[0] * args.steps, v[1] * args.steps) for k, v in ktimes.items()}
    ms_max = max_over_ranks(ms, world, dev)
    if world > 1:
        dist.barrier()
    value = job_rate(B * args.steps, world, ms_max / 1e3)
    loss_last = stats.tolist()

    # ---- end to end through the C-ABI with host buffers (pinned), copies timed
    e2e_steps = args.e2e_steps or min(args.steps, 10)
    h_order = host_buffer_order(order, args.warmup + args.steps, e2e_steps, wl.P, B)
    sel = torch.from_numpy(h_order.astype(np.int64)).to(dev)
    I_host = Iexp_d.index_select(0, sel).cpu().pin_memory()
    pos_host = pos_d.index_select(0, sel).cpu().pin_memory()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    if args.engine in ("epie", "lsqml"):
        # the public ePIE / LSQML calls take device arrays: the timed region copies
        # each group's positions and patterns in and reads its loss back
        pos_g = torch.empty((B, 2), dtype=torch.float32, device=dev)
        I_g = torch.empty((B, wl.N, wl.N), dtype=torch.float32, device=dev)
        ident = torch.arange(B, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        if args.engine in ("epie", "lsqml"):
            pos_g.copy_(pos_host[i * B:(i + 1) * B], non_blocking=True)
            I_g.copy_(I_host[i * B:(i + 1) * B], non_blocking=True)
            if args.engine == "epie":
                float(ctx.epie_step(Od, Pd, pos_g, I_g, ident, beta_O=0.5, beta_P=0.5).item())
            else:
                float(ctx.lsqml_step(Od, Pd, pos_g, I_g, ident, **lsq).item())
        else:
            ctx.step_host(Od, Pd, st, opt, pos_host[i * B:(i + 1) * B], I_host[i * B:(i + 1) * B])
    t_e2e = time.perf_counter() - t0
    te = max_over_ranks(t_e2e, world, dev)
    e2e = {"value": job_rate(B * e2e_steps, world, te), "unit": "positions/s",
           "h2d_bytes_per_step": B * 2 * 4 + B * wl.N * wl.N * 4,
           "d2h_bytes_per_step": 8 if args.engine in ("epie", "lsqml") else 16,
           "api": (f"ptycho_{args.engine}_step after pinned host-to-device copies"
                   if args.engine in ("epie", "lsqml") else "ptycho_step_host (pinned host buffers)")}

    # ---- roofline of the dominant kernel (live CUDA events on the launching stream)
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    dom_ms, dom_n = ktimes[dom]
    peaks, peak_src = measured_peaks()
    recompute = args.waves == "recompute"
    if dom == "adjoint":
        flops = adjoint_algorithmic_flops(wl, B * wl.K, recompute)
    else:
        flops = B * wl.K * 2 * wl.S * fft_flops(wl.N * wl.N)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    nominal_tf = nsm * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    peak_tf = peak_meas["tflops"]
    achieved = flops / (dom_ms / dom_n / 1e3) / 1e12
    traffic_path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    traffic = None
    if os.path.exists(traffic_path):
        with open(traffic_path) as f:
            tj = json.load(f)
        key = f"{dom}/{args.workload}/{args.waves}/{args.wave_prec}" + ("" if args.engine == "gd" else "/" + args.engine)
        # counters are only valid for the kernel source they were taken on
        if key in tj and tj[key].get("kernel_source") == kernel_source_hash(wl.N):
            traffic = tj[key]["bytes_per_item"] * B * wl.K
    roofline = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved / peak_tf, "traffic": traffic,
                "peak_source": "measured: FP32 FFMA/FFMA2 microbenchmark on this GPU just before the timed "
                               "region (ptycho_fp32_peak_launch, best of 3 launches of ~0.3 s, CUDA events)",
                "peak_measurement": {"ffma_tflops": peak_meas["ffma"]["tflops"],
                                     "ffma2_tflops": peak_meas["ffma2"]["tflops"],
                                     "sm_mhz": peak_meas["clocks"].get("sm_mhz"),
                                     "reasons": peak_meas["clocks"].get("reasons")},
                "frac_of_nominal": achieved / nominal_tf,
                "nominal_peak": nominal_tf,
                "nominal_source": f"{nsm} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                                  f"{peaks.get('sm_max_mhz', 2032.0):.0f} MHz ({peak_src} max SM clock)",
                "ms_per_launch": dom_ms / dom_n,
                "share_of_step": dom_ms / ms,
                "kernels_ms_per_step": {k: v[0] / args.steps for k, v in ktimes.items()}}
    if traffic is not None:
        # the same kernel against the HBM roof: its DRAM bytes (ncu) over its live launch time
        gbs = traffic / (dom_ms / dom_n / 1e3) / 1e9
        roofline["dram"] = {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": gbs / peaks["hbm_gbs"], "peak_source": f"{peak_src} copy bandwidth"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "positions/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(config_dict(wl, args.waves, args.dft, args.wave_prec), engine=args.engine,
                               **({"graph": "one captured step replayed per step"} if graph_launches else {}),
                               **({"loss": "amplitude"} if args.engine in ("epie", "lsqml") else {}),
                               **({"positions_used": wl.P} if args.positions else {})),
                "step_ms": {"median": float(np.median(step_ms)), "p99": float(np.percentile(step_ms, 99)),
                            "min": float(step_ms.min()), "max": float(step_ms.max()), "n": int(args.steps)},
                "roofline": roofline, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clocks, "last_stats": loss_last}
        if world == 1 and args.workload == 3 and not (args.positions or args.group) and args.engine == "gd" \
                and args.dft == "fft" and args.wave_prec == "f32" and args.waves == "recompute" and not args.no_others:
            # the two single-slice workloads of the path, measured beside the headline
            line["other_workloads"] = {
                "1": workload_leg(1, 8000, 20, dev, peak_tf, peaks["hbm_gbs"]),
                "2": workload_leg(2, 1200, 10, dev, peak_tf, peaks["hbm_gbs"])}
        if world == 1 and not args.no_baseline:
            n_s = 8 if wl.S > 1 else 64
            line["cpu_baseline"] = cpu_oracle_leg(
                wl, geom, pos_np.astype(np.float64), n_s, np.ones((wl.S, wl.H, wl.W), np.complex64), P_np,
                f"oracle steps on {n_s} positions x {wl.K} modes x {wl.S} slices each (full object, Adam included)")
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
