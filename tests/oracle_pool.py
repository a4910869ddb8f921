"""The FP64 oracle over many scan positions on every host core (spawn-started worker processes).

With the Poisson loss L = -sum(d log(I + eps) - I) / S over a batch, S = sum of the batch's measured
counts, the loss and gradient of a chunk of positions computed on its own (normaliser S_chunk) are
those of the whole batch restricted to the chunk times S_chunk / S.  So the batch's loss and every
gradient are the sums over chunks of the rescaled chunk results, and each chunk can run in its own
process.  Workers are spawned (never forked), so a parent that already uses CUDA is safe.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_STATE = {}


def _init(args):
    _STATE["args"] = args


def _chunk(job):
    from oracle import ptycho as O
    idx, I_rows = job
    geom, amp, phase, probe, pos, tilt, dz, Ntot = _STATE["args"]
    I_meas = {j: I_rows[k] for k, j in enumerate(idx)}
    r = O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx)
    return r, float(sum(I_rows[k].sum() for k in range(len(idx))))


def poisson_loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx, procs=None):
    """O.loss_and_grad(...) of the batch idx (Poisson), computed chunk by chunk in parallel.
    I_meas: indexable by scan position.  Returns the same fields."""
    from oracle import ptycho as O
    assert geom.loss == O.POISSON and not geom.w_pacbed and not geom.w_sparse
    idx = [int(j) for j in idx]
    procs = procs or min(16, os.cpu_count() or 1, len(idx))
    procs = min(procs, len(idx))
    chunks = [idx[k::procs] for k in range(procs)]
    jobs = [(c, np.stack([np.asarray(I_meas[j], dtype=np.float64) for j in c])) for c in chunks]
    S = sum(float(r.sum()) for _, r in jobs)
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(jobs), initializer=_init,
                  initargs=((geom, amp, phase, probe, pos, tilt, dz, len(pos)),)) as pool:
        out = pool.map(_chunk, jobs)
    tot = None
    I_model = np.zeros((len(idx), geom.N, geom.N))
    for k, (r, s) in enumerate(out):
        I_model[k::procs] = r.I_model  # chunk k holds batch entries k, k + procs, ...
        f = s / S
        if tot is None:
            tot = O.Gradients(loss=f * r.loss, I_model=I_model, amp=f * r.amp, phase=f * r.phase, probe=f * r.probe,
                              pos=f * r.pos, tilt=f * r.tilt, dz=f * r.dz)
        else:
            tot.loss += f * r.loss
            tot.amp += f * r.amp
            tot.phase += f * r.phase
            tot.probe += f * r.probe
            tot.pos += f * r.pos
            tot.tilt += f * r.tilt
            tot.dz += f * r.dz
    return tot
