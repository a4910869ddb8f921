#!/usr/bin/env python
"""Throughput of one pass of the ptychography hot path: forward model, loss and adjoint.

A step is one pty_loss_grad call over one batch of scan positions: shifted probes, all
transmissions and propagations, the far field, the Poisson loss and every gradient (object
amplitude and phase, probe, positions, tilts, dz).  The metric counts position x mode x slice
wavefield updates per second.  The default workload is the largest: 256 x 256 windows (four-CTA
clusters), 12 probe modes, 20 slices of 1024 x 1024, 16384 positions, batches of 256 positions
taken as contiguous raster blocks; the 128 x 128 multislice workload (6 modes, 8 slices of
512 x 512, batches of 512) is timed in the same run and reported under "also".  With several ranks
each step is the data-parallel step: every rank its own block of positions, an all-reduce of the
loss statistics and of every gradient.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "wavefield updates/s (fwd+adjoint, 1 GB300)"
UNIT = "position*mode*slice updates/s"
# name -> (description, default batch).  c3, the largest configuration, is the default.
WORKLOADS = {
    "c2": ("multislice N=128 M=6 Nz=8, object 8x512x512, 4096 positions", 512),
    "c1": ("single-slice N=64 M=1 Nz=1, object 128x128, 256 positions", 256),
    "c3": ("multislice N=256 M=12 Nz=20, object 20x1024x1024, 16384 positions", 256),
    "paper": ("paper-shaped N=128 M=12 Nz=6, object 6x614x614, 16384 positions", 16),
}

def fft2_flops(N):
    """Nominal 5 n log2 n flops of a complex FFT of n = N^2 points."""
    return 5.0 * N * N * math.log2(N * N)


def flops_per_wave(N, Nz, stage):
    """Algorithmic flops of one (position, mode) wave in the forward or adjoint kernel.

    Forward: 2 Nz 2D FFTs (shift, Nz-1 propagation pairs, far field) + per pixel: shift ramp
    (2 complex products, 12), Nz transmissions (6 each), Nz-1 propagator products (12 each), far-field
    scale and |.|^2 (5).  Adjoint: 2 Nz 2D FFTs + per pixel: 2 dL/dI Psi (4), Nz x (conj(psi) g 6,
    conj(T) g 6), Nz-1 x (propagator 12, dz/tilt term 4), probe ramp and position term (12 + 6 + 4)."""
    px = N * N
    if stage == "forward":
        return 2 * Nz * fft2_flops(N) + px * (12 + 6 * Nz + 12 * (Nz - 1) + 5)
    return 2 * Nz * fft2_flops(N) + px * (4 + 12 * Nz + 16 * (Nz - 1) + 22)


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("fft_smem.cuh", "fft_cluster.cuh", "pipeline.cuh"):
        with open(os.path.join(ROOT, "paper_2505_07814_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload, B):
    """DRAM bytes per launch of `kernel` on `workload` at batch B from the committed ncu summary
    (profiles/traffic.json), if it was taken on the current kernel source; None otherwise."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash() or e.get("full_batch") != B:
        return None
    return e.get("dram_bytes_per_launch_full_size")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu_id)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def gpu_smi_id(torch, dev):
    try:
        p = torch.cuda.get_device_properties(dev)
        return "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        return str(dev.index or 0)


def make_inputs(workload, positions, first=0):
    """The workload, the default flat start and measured patterns for the given scan positions
    (a dict position -> row of the returned [len(positions)][N][N] float32 array).  first > 0 keeps
    only the first `first` scan positions (small profiling captures)."""
    from paper_2505_07814_gb300 import synth

    w = synth.workload(workload)
    if first > 0:
        w.pos, w.tilt = w.pos[:first], w.tilt[:first]
    amp0, phase0 = synth.flat_object(w.Nz, w.H, w.W)  # default start of a reconstruction
    used = sorted(set(positions))
    I_rows = synth.vacuum_patterns(w.probe, len(used))
    return w, amp0, phase0, I_rows, {p: r for r, p in enumerate(used)}


def batch_indices(step, B, Ntot):
    s = (step * B) % Ntot
    return [(s + i) % Ntot for i in range(B)]


def rank_batches(rank, world, B, Ntot, n=8):
    """The n position batches rank `rank` of `world` takes: global batches rank, rank + world, ... of
    contiguous raster blocks (weak scaling: every rank its own blocks, no collective on the data path)."""
    return [batch_indices(k * world + rank, B, Ntot) for k in range(n)]


def max_over_ranks(value, dist, device):
    """The largest `value` over all ranks (the job's time is its slowest rank's)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def row_runs(idx):
    """Maximal runs [lo, hi) of consecutive indices (a contiguous batch that wraps gives two)."""
    runs, lo = [], idx[0] if idx else 0
    for a, b in zip(idx, idx[1:] + [None]):
        if b != a + 1:
            runs.append((lo, a + 1))
            lo = b
    return runs


def cpu_oracle_sample(w, amp0, phase0, I_meas, idx_all, seconds):
    """Time the FP64 oracle's loss and gradient on a bounded sample of one batch."""
    import numpy as np

    from oracle import ptycho as O

    geom = O.Geometry(N=w.N, M=w.M, Nz=w.Nz, H=w.H, W=w.W, dx=w.dx, lam=w.lam)
    t0 = time.perf_counter()
    O.loss_and_grad(geom, amp0, phase0, w.probe, w.pos, w.tilt, w.dz, I_meas, idx_all[:1])
    t1 = time.perf_counter() - t0
    P = max(1, min(len(idx_all), int(seconds / max(t1, 1e-3))))
    t0 = time.perf_counter()
    O.loss_and_grad(geom, amp0, phase0, w.probe, w.pos, w.tilt, w.dz, I_meas, idx_all[:P])
    dt = time.perf_counter() - t0
    return P, dt


_ORACLE_WORKER = None


def _oracle_worker_init(workload, positions):
    """Pool initialiser: one single-threaded oracle per process, on the same inputs as the parent."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    global _ORACLE_WORKER
    from oracle import ptycho as O
    w, amp0, phase0, I_rows, row_of = make_inputs(workload, positions)
    geom = O.Geometry(N=w.N, M=w.M, Nz=w.Nz, H=w.H, W=w.W, dx=w.dx, lam=w.lam)
    _ORACLE_WORKER = (O, geom, w, amp0, phase0, _Rows(I_rows, row_of))


def _oracle_worker(j):
    O, geom, w, amp0, phase0, rows = _ORACLE_WORKER
    O.loss_and_grad(geom, amp0, phase0, w.probe, w.pos, w.tilt, w.dz, rows, [j])
    return j


def cpu_oracle_all_cores(workload, idx, seconds_per_position, seconds):
    """The same oracle on every host core: a spawn-started pool (no fork of a CUDA process), one
    position per task, over a bounded sample of the batch.  Returns (positions, wall seconds, cores)."""
    import multiprocessing as mp
    procs = os.cpu_count() or 1
    P = max(procs, min(len(idx), int(procs * seconds / max(seconds_per_position, 1e-3))))
    sample = list(idx[:P])
    with mp.get_context("spawn").Pool(procs, initializer=_oracle_worker_init, initargs=(workload, sample)) as pool:
        pool.map(_oracle_worker, sample[:procs], chunksize=1)  # every worker initialised and warm
        t0 = time.perf_counter()
        pool.map(_oracle_worker, sample, chunksize=1)
        dt = time.perf_counter() - t0
    return len(sample), dt, procs


def _ntot(workload):
    return {"c1": 256, "c2": 4096, "c3": 16384, "paper": 16384}[workload]


class _Rows:
    """Measured patterns indexed by scan position, backed by the rows that were generated."""

    def __init__(self, rows, row_of):
        self.rows, self.row_of = rows, row_of

    def __getitem__(self, j):
        return self.rows[self.row_of[j]]


def run_reference(args, rank):
    if rank != 0:
        return
    import numpy as np

    P = 1 if args.workload == "c3" else 2  # positions per step: a bounded sample of one batch
    batches = [batch_indices(k, args.batch, _ntot(args.workload))[:P] for k in range(args.warmup + args.steps)]
    w, amp0, phase0, I_rows, row_of = make_inputs(args.workload, [p for b in batches for p in b])
    from oracle import ptycho as O
    import numpy as np

    I_meas = _Rows(I_rows, row_of)
    geom = O.Geometry(N=w.N, M=w.M, Nz=w.Nz, H=w.H, W=w.W, dx=w.dx, lam=w.lam)
    times = []
    for k in range(args.warmup + args.steps):
        idx = batches[k]
        t0 = time.perf_counter()
        O.loss_and_grad(geom, amp0, phase0, w.probe, w.pos, w.tilt, w.dz, I_meas, idx)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    upd = P * w.M * w.Nz
    value = upd * len(times) / sum(times)
    sample = "%d positions (%d updates) of a %d-position batch per step; FP64 numpy oracle" % (P, upd, args.batch)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][0], "N": w.N, "M": w.M, "Nz": w.Nz,
                       "positions": w.Ntot, "batch": args.batch, "sample_positions_per_step": P},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sweep_ckpt(args, w, geometry, params, I_meas, idx_t, flush, dev, torch, Ptycho):
    """Checkpoint-vs-recompute sweep: one JSON line per ckpt_stride with the step time and the bytes
    the forward record takes."""
    B = args.batch
    for K in [int(x) for x in args.sweep_ckpt.split(",")]:
        geom = geometry(K)
        pt = Ptycho(geom, B, device=dev)
        grads = params.zeros_like()
        for k in range(args.warmup):
            pt.loss_grad(params, idx_t[k % 8], I_meas, grads=grads)
        torch.cuda.synchronize()
        ms = 0.0
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for k in range(args.steps):
            flush.zero_()
            ev[0].record()
            pt.loss_grad(params, idx_t[k % 8], I_meas, grads=grads)
            ev[1].record()
            ev[1].synchronize()
            ms += ev[0].elapsed_time(ev[1])
        assert pt.status() == 0
        print(json.dumps({"workload": WORKLOADS[args.workload][0], "batch": B, "ckpt_stride": K,
                          "checkpoint_bytes": geom.checkpoint_bytes(B), "workspace_bytes": pt.ws_bytes,
                          "ms_per_step": ms / args.steps,
                          "updates_per_s": B * w.M * w.Nz * args.steps / (ms / 1e3)}), flush=True)
        del pt, grads
        torch.cuda.empty_cache()


def sweep_shape(args, w, amp0, phase0, I_meas, idx_t, flush, dev, torch, Geometry, Params, Ptycho):
    """Step time against batch size, probe modes and slices on the multislice workload (the shape of
    the paper's Fig. 3b-d): one JSON line per point.  Extra modes are the workload's modes scaled by
    1/2 per repeat, extra slices repeat its slices; values do not change the work."""
    import numpy as np
    f32 = dict(dtype=torch.float32, device=dev)
    points = [("batch", B, w.M, w.Nz) for B in (64, 128, 256, 512)]
    points += [("modes", 256, M, w.Nz) for M in (1, 2, 4, 6, 8, 12)]
    points += [("slices", 256, w.M, Nz) for Nz in (1, 2, 4, 8, 12, 16)]
    for axis, B, M, Nz in points:
        probe = np.stack([w.probe[m % w.M] * 0.5 ** (m // w.M) for m in range(M)])
        amp = np.stack([amp0[s % w.Nz] for s in range(Nz)])
        phase = np.stack([phase0[s % w.Nz] for s in range(Nz)])
        params = Params(amp=torch.tensor(amp, **f32), phase=torch.tensor(phase, **f32),
                        probe=torch.tensor(probe, dtype=torch.complex64, device=dev), pos=torch.tensor(w.pos, **f32),
                        tilt=torch.tensor(w.tilt, **f32), dz=torch.tensor([w.dz], **f32))
        geom = Geometry(N=w.N, M=M, Nz=Nz, H=w.H, W=w.W, Ntot=w.Ntot, dx=w.dx, lam=w.lam, loss="poisson")
        pt = Ptycho(geom, B, device=dev)
        grads = params.zeros_like()
        idx = [t[:B] for t in idx_t]
        for k in range(args.warmup):
            pt.loss_grad(params, idx[k % len(idx)], I_meas, grads=grads)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ms = 0.0
        for k in range(args.steps):
            flush.zero_()
            ev[0].record()
            pt.loss_grad(params, idx[k % len(idx)], I_meas, grads=grads)
            ev[1].record()
            ev[1].synchronize()
            ms += ev[0].elapsed_time(ev[1])
        assert pt.status() == 0
        ms /= args.steps
        print(json.dumps({"sweep": axis, "workload": WORKLOADS[args.workload][0], "batch": B, "modes": M,
                          "slices": Nz, "ms_per_step": ms, "updates_per_s": B * M * Nz / (ms / 1e3),
                          "s_per_pass": ms / 1e3 * (w.Ntot / B)}), flush=True)
        del pt, grads, params
        torch.cuda.empty_cache()


def run_nmse(args):
    """Time to object NMSE <= target on the multislice workload (object seed 1234, measured counts
    simulated by the forward model): the flat start (Sec. "Preprocessing and initialization") with
    FP32 FFTs and with split-precision DFT-GEMMs, against the start stitched from the learned
    initialiser's predictions (network trained on 65536 pairs from 16 other random volumes).  Adam
    on the object phase only (probe, positions, tilt, dz at the truth), batch 64, each start at the
    better of two phase learning rates.  Times are GPU seconds of reconstruction (and of inference +
    stitching for the learned start), NMSE evaluation excluded.  With --nmse-probe-defocus the same
    comparison is repeated from a probe with the wrong defocus that Adam refines with the object
    ("wrong_probe" in the line)."""
    import torch

    from paper_2505_07814_gb300 import _lib, build
    from paper_2505_07814_gb300 import learned_init as L
    from paper_2505_07814_gb300.cnn import Cnn

    build.build()
    _lib.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    target, batch, lrs = args.nmse_target, 64, (1e-3, 3e-3)
    prob = L.problem("c2")
    amp_f, ph_f = L.flat_object(prob)

    def best(amp0, ph0, fft="fp32", iters=6):
        runs = []
        for lr in lrs:
            hist, _ = L.reconstruct(prob, amp0, ph0, iters=iters, batch=batch, lr={"phase": lr}, target=target, fft=fft)
            it, e, t = hist[-1]
            runs.append({"lr_phase": lr, "reached": e <= target, "iterations": it, "nmse": e, "seconds": t,
                         "nmse_start": hist[0][1]})
        ok = [r for r in runs if r["reached"]]
        return (min(ok, key=lambda r: r["seconds"]) if ok else None), runs

    L.reconstruct(prob, amp_f, ph_f, iters=1, batch=batch, lr={"phase": lrs[0]}, target=1.0)  # warm-up
    flat, flat_runs = best(amp_f, ph_f)
    split = {}
    for fft in args.nmse_split.split(",") if args.nmse_split else []:
        split[fft] = best(amp_f, ph_f, fft=fft)[0]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    I, Y = L.training_set(prob, n_objects=16, per_object=4096)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    net = Cnn(S=128, max_batch=256)
    ev0.record()
    losses = L.train(net, I, Y, epochs=args.nmse_epochs, batch=256, lr=1e-3)
    ev1.record()
    ev1.synchronize()
    train_s = ev0.elapsed_time(ev1) / 1e3
    del I, Y
    # inference in batches of 1024 patterns (the kernels' largest batch; 14% more patterns/s than 256)
    net_inf = Cnn(S=128, max_batch=1024, params=net.params)
    L.initial_object(net_inf, prob, batch=1024)  # warm-up
    ev0.record()
    amp_c, ph_c = L.initial_object(net_inf, prob, batch=1024)
    ev1.record()
    ev1.synchronize()
    infer_s = ev0.elapsed_time(ev1) / 1e3
    learned, learned_runs = best(amp_c, ph_c)
    value = learned["seconds"] + infer_s if learned else None
    wrong = None
    if args.nmse_probe_defocus:
        # Both starts begin from a probe with the wrong defocus and refine it with the object; the
        # learned start is stitched with that probe too.
        P0 = L.probe_estimate(prob, args.nmse_probe_defocus)
        lr_p = args.nmse_probe_lr

        def best_p(amp0, ph0):
            runs = []
            for lr in lrs:
                hist, _ = L.reconstruct(prob, amp0, ph0, iters=args.nmse_probe_iters, batch=batch,
                                        lr={"phase": lr, "probe": lr_p}, target=target, probe0=P0)
                it, e, t = hist[-1]
                runs.append({"lr_phase": lr, "reached": e <= target, "iterations": it, "nmse": e, "seconds": t,
                             "nmse_start": hist[0][1]})
            ok = [r for r in runs if r["reached"]]
            return (min(ok, key=lambda r: r["seconds"]) if ok else None), runs

        ev0.record()
        amp_w, ph_w = L.initial_object(net_inf, prob, batch=1024, probe=P0)
        ev1.record()
        ev1.synchronize()
        infer_w = ev0.elapsed_time(ev1) / 1e3
        flat_w, flat_w_runs = best_p(amp_f, ph_f)
        learned_w, learned_w_runs = best_p(amp_w, ph_w)
        value_w = learned_w["seconds"] + infer_w if learned_w else None
        wrong = {"probe_start": "the workload's probe model with defocus %g A (truth 50 A)" % args.nmse_probe_defocus,
                 "lr_probe": lr_p, "max_iterations": args.nmse_probe_iters, "flat": flat_w, "flat_runs": flat_w_runs,
                 "learned": dict(learned_w or {}, inference_stitch_seconds=infer_w), "learned_runs": learned_w_runs,
                 "speedup_vs_flat": (flat_w["seconds"] / value_w) if (flat_w and value_w) else None}
    line = {"metric": "time to object NMSE <= %g (learned start vs flat start, 1 GB300)" % target, "value": value,
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": WORKLOADS["c2"][0] + ", measured counts from the forward model (dose 1e5)",
                       "batch": batch, "optimiser": "Adam, object phase only", "nmse": "depth-summed phase, ROI of the "
                       "window centres, offset removed", "lr_grid_phase": list(lrs)},
            "flat_fp32": flat, "flat_runs": flat_runs, "split_precision_flat": split,
            "learned": dict(learned or {}, inference_stitch_seconds=infer_s), "learned_runs": learned_runs,
            "training": {"pairs": 65536, "objects": 16, "epochs": args.nmse_epochs, "batch": 256,
                         "generation_seconds": gen_s, "training_seconds": train_s, "epoch_losses": losses},
            "speedup_vs_flat": (flat["seconds"] / value) if (flat and value) else None}
    if wrong is not None:
        line["wrong_probe"] = wrong
    print(json.dumps(line), flush=True)


CONSTRAIN_KINDS = {
    # kind: (pty_constrain settings, description, HBM bytes per object voxel as designed or None)
    "blur": (dict(phase_positivity=1.0, rz_sigma=1.0), "depth blur (sigma 1 slice) + positivity", 16),
    # five passes: x (amp, phase -> z), y, depth columns, y, x (z, amp, phase -> amp, phase)
    "kz": (dict(kz_beta=1.0, kz_alpha=0.01, kz_relax=1.0), "k_z filter (beta 1, alpha 0.01 A^2)", 88),
    "ortho": (dict(orthogonalize_probe=True), "probe-mode orthogonalisation", None),
}


def run_constrain(args, w, geom, params, flush, torch, Ptycho):
    """pty_constrain on the workload's object or probe; the object constraints are HBM-bound."""
    from paper_2505_07814_gb300.ptycho import constrain
    kw, what, per_voxel = CONSTRAIN_KINDS[args.constrain]
    pt = Ptycho(geom, 1)
    for _ in range(args.warmup):
        constrain(pt, params, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0.record()
        constrain(pt, params, **kw)
        e1.record()
        e1.synchronize()
        total += e0.elapsed_time(e1)
    ms = total / args.steps
    line = {"metric": "%s per call" % what, "value": ms, "unit": "ms", "higher_is_better": False,
            "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": WORKLOADS[args.workload][0], "object": [w.Nz, w.H, w.W], "modes": w.M, "N": w.N,
                       **{k: (float(v) if not isinstance(v, bool) else v) for k, v in kw.items()}}}
    if per_voxel:
        peak = None
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                peak = json.load(fh).get("hbm_gbs")
        except (OSError, ValueError):
            pass
        peak = peak or 6800.0
        nbytes = per_voxel * w.Nz * w.H * w.W
        gbs = nbytes / (ms / 1e3) / 1e9
        line["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                            "bytes": nbytes, "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    print(json.dumps(line), flush=True)


def cnn_flops(S=128, train=True):
    """Algorithmic flops of the learned initialiser per pattern: 2 x MACs of the six 3x3
    convolutions at their output resolutions (nearest upsampling counted on the upsampled grid);
    a training step adds the input gradient of layers 2..6 and the weight gradient of every layer,
    each with the forward's MAC count."""
    layers = ((1, 48, 2, 1), (48, 96, 2, 1), (96, 192, 2, 1), (192, 384, 2, 1), (384, 256, 1, 2), (256, 2, 1, 4))
    h, fwd, dgrad = S, [], 0
    for ic, oc, st, up in layers:
        h = (h * up + st - 1) // st
        fwd.append(2 * h * h * oc * 9 * ic)
    total = sum(fwd)
    if train:
        total += sum(fwd[1:]) + sum(fwd)
    return total


def run_cnn(args):
    """Training and inference throughput of the learned initialiser's kernels (patterns 128 x 128,
    batches of 256, synthetic patterns and targets): one line with patterns/s and the achieved
    tensor FLOP/s against the measured bf16 peak."""
    import numpy as np
    import torch

    from paper_2505_07814_gb300 import _lib, build
    from paper_2505_07814_gb300.cnn import Cnn

    build.build()
    _lib.load()
    dev = torch.device("cuda", 0)
    S, B = 128, args.batch if args.batch > 0 else 256
    net = Cnn(S=S, max_batch=B)
    rng = np.random.default_rng(0)
    I = torch.tensor(rng.gamma(1.5, 40.0, (B, S, S)).astype(np.float32), device=dev)
    Y = torch.tensor((0.2 * rng.standard_normal((B, S // 2, S // 2, 2))).astype(np.float32), device=dev)
    for _ in range(args.warmup):
        net.train_step(I, Y)
        net.predict(I)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = _lib.pty_launch_count()
    e0.record()
    for _ in range(args.steps):
        net.train_step(I, Y)
    e1.record()
    e1.synchronize()
    train_ms = e0.elapsed_time(e1) / args.steps
    e0.record()
    for _ in range(args.steps):
        net.predict(I)
    e1.record()
    e1.synchronize()
    pred_ms = e0.elapsed_time(e1) / args.steps
    launches = _lib.pty_launch_count() - n0
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak = json.load(fh).get("bf16_tflops")
    except (OSError, ValueError):
        pass
    peak = peak or 1900.0
    tr = B * cnn_flops(S, True) / (train_ms / 1e3) / 1e12
    pr = B * cnn_flops(S, False) / (pred_ms / 1e3) / 1e12
    print(json.dumps({"metric": "learned-initialiser training step (bf16 implicit-GEMM convolutions, 1 GB300)",
                      "value": B / (train_ms / 1e3), "unit": "patterns/s", "higher_is_better": True,
                      "ms_per_step": train_ms, "steps": args.steps, "warmup": args.warmup, "dtype": "bf16 (FP32 accumulate)",
                      "data": "synthetic", "config": {"workload": "CNN 1.76M params, patterns 128x128", "batch": B},
                      "inference": {"ms_per_batch": pred_ms, "patterns_per_s": B / (pred_ms / 1e3)},
                      "roofline": {"bound": "tensor", "achieved": tr, "peak": peak, "unit": "TFLOP/s",
                                   "frac": tr / peak, "inference_achieved": pr, "inference_frac": pr / peak,
                                   "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)"},
                      "gpu_launches": launches}), flush=True)


def fma_peak_tflops(torch, dev):
    """Measured FP32 fused-multiply-add throughput of this GPU (pty_fma_probe), TFLOP/s, best of 5."""
    from paper_2505_07814_gb300 import _lib
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    blocks, iters = 4 * sms, 2048
    flops = blocks * 512 * iters * 256
    st = torch.cuda.current_stream(dev).cuda_stream
    _lib.pty_fma_probe(sink.data_ptr(), blocks, 64, st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 0.0
    for _ in range(5):
        e0.record()
        _lib.pty_fma_probe(sink.data_ptr(), blocks, iters, st)
        e1.record()
        e1.synchronize()
        best = max(best, flops / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best


def alu_peak_tflops(sms, mhz):
    """FP32 CUDA-core peak from unit counts: SMs x 128 FP32 lanes x 2 flop (FMA) x clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


class Workload:
    """One workload on this rank's GPU: inputs resident in HBM, the Ptycho problem, the batches this
    rank takes, and (one GPU) a CUDA graph of each batch's step."""

    def __init__(self, args, name, B, dev, rank, world):
        import torch

        from paper_2505_07814_gb300.ptycho import Geometry, Params, Ptycho
        self.name, self.B, self.dev, self.world = name, B, dev, world
        Ntot = args.positions if args.positions > 0 else _ntot(name)
        # weak scaling: every rank its own blocks of B positions (a global batch of world x B); with
        # more than one rank each step is the data-parallel step (statistics and gradient all-reduce)
        self.idx_h = rank_batches(rank, world, B, Ntot)
        w, amp0, phase0, I_rows, row_of = make_inputs(name, [p for b in self.idx_h for p in b], args.positions)
        self.w, self.amp0, self.phase0, self.I_rows, self.row_of = w, amp0, phase0, I_rows, row_of
        f32 = dict(dtype=torch.float32, device=dev)
        self.params = Params(amp=torch.tensor(amp0, **f32), phase=torch.tensor(phase0, **f32),
                             probe=torch.tensor(w.probe, dtype=torch.complex64, device=dev),
                             pos=torch.tensor(w.pos, **f32), tilt=torch.tensor(w.tilt, **f32),
                             dz=torch.tensor([w.dz], **f32))
        # measured patterns [Ntot][N][N] on the device; only the rows the timed batches read are filled
        self.I_meas = torch.zeros((w.Ntot, w.N, w.N), **f32)
        rows_t = torch.tensor(I_rows, **f32)
        for p_, r_ in row_of.items():
            self.I_meas[p_] = rows_t[r_]
        del rows_t
        self.idx_t = [torch.tensor(i, dtype=torch.int32, device=dev) for i in self.idx_h]
        self.geom = Geometry(N=w.N, M=w.M, Nz=w.Nz, H=w.H, W=w.W, Ntot=w.Ntot, dx=w.dx, lam=w.lam, loss="poisson",
                             ckpt_stride=args.ckpt_stride, fft=args.fft, w_pacbed=args.w_pacbed,
                             w_sparse=args.w_sparse)
        self.pt = Ptycho(self.geom, B, device=dev)
        self.grads = self.params.zeros_like()
        self.graphs = None
        self.per_step_launches = None

    def step(self, k, params=None, I_meas=None, grads=None):
        """One pass over batch k: loss and every gradient (the data-parallel step on several ranks)."""
        params = params or self.params
        I_meas = self.I_meas if I_meas is None else I_meas
        grads = grads or self.grads
        if self.world == 1:
            return self.pt.loss_grad(params, self.idx_t[k % 8], I_meas, grads=grads)[0]
        import torch.distributed as dist

        from paper_2505_07814_gb300 import data_parallel as DP
        return DP.loss_grad(self.pt, params, self.idx_t[k % 8], I_meas, grads, dist.all_reduce)[0]

    def capture(self, steps):
        """One CUDA graph per batch (one GPU, FP32 FFTs): replays remove the host launch gaps."""
        import torch

        from paper_2505_07814_gb300 import _lib
        self.graphs = []
        for k in range(min(8, steps)):
            g_ = torch.cuda.CUDAGraph()
            c0 = _lib.pty_launch_count()
            # thread-local capture: other threads may use CUDA meanwhile
            with torch.cuda.graph(g_, capture_error_mode="thread_local"):
                self.step(k)
            self.per_step_launches = _lib.pty_launch_count() - c0  # the library's kernels in one step
            self.graphs.append(g_)
        torch.cuda.synchronize()

    def run(self, k):
        if self.graphs:
            self.graphs[k % len(self.graphs)].replay()
        else:
            self.step(k)

    @property
    def updates_per_step(self):
        return self.B * self.w.M * self.w.Nz


def time_steps(wl, steps, warmup, graph, flush, clock_id):
    """Warm-up, then exactly `steps` timed steps (CUDA events on the launching stream, L2 flushed
    before each outside the events), clocks sampled meanwhile.  Returns (total ms, launches, stage
    times per call, calls, clock summary)."""
    import torch

    from paper_2505_07814_gb300 import _lib
    for k in range(warmup):
        wl.step(k)
    torch.cuda.synchronize()
    assert wl.pt.status() == 0
    if graph:
        wl.capture(steps)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    _lib.pty_profile_enable(True)
    n0 = _lib.pty_launch_count()
    if wl.world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(clock_id) as clk:
        for k in range(steps):
            flush.zero_()
            starts[k].record()
            wl.run(k)
            ends[k].record()
        torch.cuda.synchronize()
    if wl.world > 1:
        dist.barrier()
    launches = _lib.pty_launch_count() - n0
    ncalls, stage_ms = _lib.pty_profile_read()
    _lib.pty_profile_enable(False)
    if graph:
        # replays pass neither the host launch counter nor the stage events: count the captured
        # kernels, and take the stage times from a few eager steps after the timed region
        launches = wl.per_step_launches * steps
        _lib.pty_profile_enable(True)
        for k in range(warmup):
            flush.zero_()
            wl.step(k)
        torch.cuda.synchronize()
        ncalls, stage_ms = _lib.pty_profile_read()
        _lib.pty_profile_enable(False)
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    return total_ms, launches, stage_ms, ncalls, clk.summary()


def roofline_of(wl, args, stage_ms, ncalls, sms, clocks, fma_tflops):
    """The dominant kernel against the FP32 ALU roofline (the wave never leaves shared memory), or
    the split-precision GEMMs against the measured bf16 tensor peak."""
    w, B = wl.w, wl.B
    if args.fft == "fp32":
        dom = max(("forward", "adjoint"), key=lambda s: stage_ms[s])
        avg_ms = stage_ms[dom] / max(ncalls, 1)
        flops = B * w.M * flops_per_wave(w.N, w.Nz, dom)
        achieved = flops / (avg_ms / 1e3) / 1e12
        max_mhz = clocks.get("sm_max_mhz") or 2070.0
        peak = alu_peak_tflops(sms, max_mhz)
        traffic = ncu_traffic("k_" + dom, wl.name, B)
        r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
             "traffic": traffic, "kernel": "k_" + dom, "avg_launch_ms": avg_ms, "flops_per_launch": flops,
             "peak_source": "%d SMs (device) x 128 FP32 lanes x 2 flop x %.0f MHz max SM clock (derived)" % (
                 sms, max_mhz)}
        if clocks.get("sm_mhz"):
            p2 = alu_peak_tflops(sms, clocks["sm_mhz"])
            r["peak_at_sampled_clock"] = p2
            r["frac_at_sampled_clock"] = achieved / p2
        if fma_tflops:
            r["measured_fma_peak"] = fma_tflops
            r["frac_of_measured_fma_peak"] = achieved / fma_tflops
        return r
    # split-precision DFTs: 8 Nz GEMMs of [B M N rows x terms 2N] x [terms 2N x 2N] per pass; the
    # time is the whole forward + adjoint (pointwise stages and operand splits included), so this is
    # a lower bound on the GEMMs' own rate
    terms = {"bf16": 3, "fp16": 3, "bf16x3": 6}[args.fft]
    gemm_flops = 8 * w.Nz * 2.0 * (B * w.M * w.N) * (2 * w.N) * (terms * 2 * w.N)
    avg_ms = (stage_ms["forward"] + stage_ms["adjoint"]) / max(ncalls, 1)
    achieved = gemm_flops / (avg_ms / 1e3) / 1e12
    peak = 1900.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak = json.load(fh).get("bf16_tflops") or peak
    except (OSError, ValueError):
        pass
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "k_gemm_tc (every DFT GEMM of the pass)", "avg_pass_ms": avg_ms,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst; fp16 taken equal)"}


def end_to_end(wl, e_steps, flush):
    """The metric end to end through the public API from pinned host buffers: every step copies its
    inputs in (every parameter and the batch's measured patterns) and every gradient and the loss
    out.  The copies run on a second stream into double buffers, so that step k + 1's inputs and
    step k's outputs move while the next step computes; the timed region spans all e_steps steps,
    with the L2 flush before each step timed separately and taken out."""
    import torch
    params, grads, I_meas, w = wl.params, wl.grads, wl.I_meas, wl.w
    names = ("amp", "phase", "probe", "pos", "tilt", "dz")
    host = {n: getattr(params, n).cpu().pin_memory() for n in names}
    h_rows = torch.tensor(wl.I_rows).pin_memory()
    h_grads = [{n: torch.empty_like(getattr(grads, n), device="cpu").pin_memory() for n in names} for _ in range(2)]
    h_loss = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    d_params = [params, params.zeros_like()]
    d_grads = [grads, params.zeros_like()]
    d_meas = [I_meas, torch.zeros_like(I_meas)]
    d_loss = [torch.zeros(1, dtype=torch.float64, device=wl.dev) for _ in range(2)]
    comp = torch.cuda.current_stream(wl.dev)
    cs = torch.cuda.Stream(device=wl.dev)
    in_ready, comp_done, out_done = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))
    h2d = sum(host[n].numel() * host[n].element_size() for n in names)
    h2d += sum((hi - lo) * w.N * w.N * 4 for lo, hi in row_runs(wl.idx_h[0]))
    d2h = sum(h_grads[0][n].numel() * h_grads[0][n].element_size() for n in names) + 8

    def issue_inputs(k):
        j = k % 2
        if k >= 2:
            cs.wait_event(comp_done[j])  # step k - 2 is done with buffer j
        with torch.cuda.stream(cs):
            for n in names:
                getattr(d_params[j], n).copy_(host[n], non_blocking=True)
            for lo, hi in row_runs(wl.idx_h[k % 8]):  # the measured patterns this batch reads
                r0 = wl.row_of[lo]
                d_meas[j][lo:hi].copy_(h_rows[r0:r0 + hi - lo], non_blocking=True)
        in_ready[j].record(cs)

    es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fl = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e_steps)]
    torch.cuda.synchronize()
    es.record(comp)
    issue_inputs(0)
    for k in range(e_steps):
        j = k % 2
        if k + 1 < e_steps:
            issue_inputs(k + 1)
        fl[k][0].record(comp)
        flush.zero_()
        fl[k][1].record(comp)
        comp.wait_event(in_ready[j])
        if k >= 2:
            comp.wait_event(out_done[j])  # step k - 2's gradients have left buffer j
        loss = wl.step(k, d_params[j], d_meas[j], d_grads[j])
        d_loss[j].copy_(loss)
        comp_done[j].record(comp)
        cs.wait_event(comp_done[j])
        with torch.cuda.stream(cs):
            for n in names:
                h_grads[j][n].copy_(getattr(d_grads[j], n), non_blocking=True)
            h_loss[j].copy_(d_loss[j], non_blocking=True)
        out_done[j].record(cs)
    for j in range(2):
        comp.wait_event(out_done[j])
    ee.record(comp)
    ee.synchronize()
    e2e_ms = es.elapsed_time(ee) - sum(a.elapsed_time(b) for a, b in fl)
    assert wl.pt.status() == 0
    for n in names:  # the last step's gradients reached the host
        assert torch.equal(h_grads[(e_steps - 1) % 2][n], getattr(d_grads[(e_steps - 1) % 2], n).cpu())
    return e2e_ms, h2d, d2h


def cpu_baseline(args, wl):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload (one host core; the
    same on every core as context)."""
    w = wl.w
    P, dt = cpu_oracle_sample(w, wl.amp0, wl.phase0, _Rows(wl.I_rows, wl.row_of), wl.idx_h[0], args.cpu_seconds)
    cpu = {"value": P * w.M * w.Nz / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "FP64 numpy oracle, loss + all gradients for the first %d positions of one %d-position "
                     "batch (%d updates, %.1f s, single-threaded pocketfft)" % (P, wl.B, P * w.M * w.Nz, dt)}
    try:  # the same oracle on every host core (context; the single-core figure above is the baseline)
        Pa, dta, procs = cpu_oracle_all_cores(wl.name, wl.idx_h[0], dt / P, args.cpu_seconds / 3)
        cpu["all_cores"] = {"value": Pa * w.M * w.Nz / dta, "cores": procs,
                            "sample": "%d positions of the same batch, one per task, %d spawn-started processes, "
                                      "%.1f s" % (Pa, procs, dta)}
    except Exception as e:  # a host without process pools still gets its single-core line
        cpu["all_cores"] = {"unavailable": str(e)[:200]}
    return cpu


def config_of(args, wl):
    w, B = wl.w, wl.B
    return {"workload": "%s, batch %d" % (WORKLOADS[wl.name][0], B), "N": w.N, "M": w.M, "Nz": w.Nz,
            "positions": w.Ntot, "batch": B, "ckpt_stride": args.ckpt_stride, "fft": args.fft,
            "w_pacbed": args.w_pacbed, "w_sparse": args.w_sparse, "checkpoint_bytes": wl.geom.checkpoint_bytes(B),
            "object": [w.Nz, w.H, w.W], "loss": "poisson", "grads": "amp,phase,probe,pos,tilt,dz",
            "batches": "contiguous raster blocks", "start": "flat object (amp 1, phase U[0,1e-8])",
            "l2": "flushed before every step (256 MiB write outside the step events)",
            "parallelism": "dp%d" % wl.world, "cuda_graph": bool(wl.graphs)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--also", default="c2",
                    help="comma-separated workloads also timed (device only) in the same run and reported under "
                         "'also' ('none' for none)")
    ap.add_argument("--batch", type=int, default=0, help="positions per step (0: the workload's default)")
    ap.add_argument("--positions", type=int, default=0,
                    help="keep only the first P scan positions (0: all); small profiling captures")
    ap.add_argument("--ckpt-stride", type=int, default=1, help="adjoint memory plan (pty_geom.ckpt_stride)")
    ap.add_argument("--fft", default="fp32", choices=["fp32", "bf16", "fp16", "bf16x3"],
                    help="per-slice DFTs: FP32 shared-memory FFT or split-precision tensor-core GEMMs")
    ap.add_argument("--sweep-ckpt", default="", help="comma-separated strides: print one timing line per stride")
    ap.add_argument("--eager", dest="graph", action="store_false",
                    help="launch every step's kernels from the host instead of replaying a CUDA graph captured "
                         "once per batch (the default on one GPU)")
    ap.add_argument("--sweep-shape", action="store_true",
                    help="step time against batch size, probe modes and slices (one line per point)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nmse", action="store_true",
                    help="time to object NMSE: flat start vs learned initialiser (and split precision)")
    ap.add_argument("--nmse-target", type=float, default=0.05)
    ap.add_argument("--nmse-probe-defocus", type=float, default=80.0,
                    help="also time both starts from a probe with this defocus (A; the truth has 50), refined "
                         "with the object (0: off)")
    ap.add_argument("--nmse-probe-lr", type=float, default=1e-2)
    ap.add_argument("--nmse-probe-iters", type=int, default=20)
    ap.add_argument("--nmse-epochs", type=int, default=8)
    ap.add_argument("--nmse-split", default="bf16,fp16", help="split-precision forms to time from the flat start")
    ap.add_argument("--cnn", action="store_true", help="learned-initialiser training / inference throughput")
    ap.add_argument("--w-pacbed", type=float, default=0.0, help="weight of the PACBED loss term (Eq. 7)")
    ap.add_argument("--w-sparse", type=float, default=0.0, help="weight of the phase-sparsity loss term (Eq. 8)")
    ap.add_argument("--constrain", nargs="?", const="blur", default=None, choices=sorted(CONSTRAIN_KINDS),
                    help="time one kind of pty_constrain on the workload's object / probe instead")
    args = ap.parse_args()
    if args.cnn:
        run_cnn(args)
        return
    if args.nmse:
        run_nmse(args)
        return
    if args.batch <= 0:
        args.batch = WORKLOADS[args.workload][1]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch

    from paper_2505_07814_gb300 import _lib, build
    from paper_2505_07814_gb300.ptycho import Geometry, Params, Ptycho

    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    build.build()
    _lib.load()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MiB > 129 MB L2

    if args.sweep_ckpt or args.constrain or args.sweep_shape:
        wl = Workload(args, args.workload, args.batch, dev, rank, world)
        geometry = lambda K: dataclasses.replace(wl.geom, ckpt_stride=K)  # noqa: E731
        if args.sweep_ckpt:
            sweep_ckpt(args, wl.w, geometry, wl.params, wl.I_meas, wl.idx_t, flush, dev, torch, Ptycho)
        elif args.constrain:
            run_constrain(args, wl.w, geometry(1), wl.params, flush, torch, Ptycho)
        else:
            sweep_shape(args, wl.w, wl.amp0, wl.phase0, wl.I_meas, wl.idx_t, flush, dev, torch, Geometry, Params,
                        Ptycho)
        return

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clock_id = gpu_smi_id(torch, dev)
    graph = args.graph and args.fft == "fp32" and world == 1
    # (the split-precision forms keep the eager path: their first call on a device builds DFT tables)
    wl = Workload(args, args.workload, args.batch, dev, rank, world)
    total_ms, launches, stage_ms, ncalls, clocks = time_steps(wl, args.steps, args.warmup, graph, flush, clock_id)
    if world > 1:
        total_ms = max_over_ranks(total_ms, dist, dev)
    value = world * wl.updates_per_step * args.steps / (total_ms / 1e3)
    fma = fma_peak_tflops(torch, dev) if rank == 0 else None
    roofline = roofline_of(wl, args, stage_ms, ncalls, sms, clocks, fma)
    stages = {k: v / max(ncalls, 1) for k, v in stage_ms.items()}
    e_steps = min(args.e2e_steps, args.steps)
    e2e_ms, h2d, d2h = end_to_end(wl, e_steps, flush)
    if world > 1:
        e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    e2e_value = world * wl.updates_per_step * e_steps / (e2e_ms / 1e3)
    cpu = cpu_baseline(args, wl) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    config = config_of(args, wl)

    also = {}
    for name in [a for a in args.also.split(",") if a in WORKLOADS and a != args.workload]:
        del wl
        torch.cuda.empty_cache()
        wl = Workload(args, name, WORKLOADS[name][1], dev, rank, world)
        t_ms, l_, st_ms, nc, clk2 = time_steps(wl, args.steps, args.warmup, graph, flush, clock_id)
        if world > 1:
            t_ms = max_over_ranks(t_ms, dist, dev)
        also[name] = {"value": world * wl.updates_per_step * args.steps / (t_ms / 1e3), "unit": UNIT,
                      "ms_per_step": t_ms / args.steps, "steps": args.steps, "gpu_launches": l_,
                      "config": config_of(args, wl), "roofline": roofline_of(wl, args, st_ms, nc, sms, clk2, fma),
                      "stage_ms_per_call": {k: v / max(nc, 1) for k, v in st_ms.items()}, "clocks": clk2}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.fft == "fp32" else "f32 (DFTs: %s split, f32 accumulate)" % args.fft,
                "data": "synthetic", "config": config, "roofline": roofline, "stage_ms_per_call": stages,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "steps": e_steps, "copies": "pinned host buffers, second stream, double-buffered "
                        "(inputs of step k+1 and outputs of step k overlap the next step's compute)"},
                "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clocks, "also": also}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
