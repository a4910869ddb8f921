"""Learned initialisation of the object: training pairs simulated by the forward model, CNN training,
inference + stitching into an initial object, and the reconstruction loop used to compare it with
the flat start (Sec. "Preprocessing and initialization") by iterations and wall time to a target
object NMSE.

Every GPU step runs in the library's kernels (pty_forward for the simulation, pty_cnn_* for the
network, pty_step for the reconstruction); torch supplies device memory, the Poisson sampler that
makes synthetic counts, and the host loop.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import synth
from .cnn import Cnn, Stitcher, targets
from .ptycho import Adam, Geometry, Params, Ptycho, step


@dataclasses.dataclass
class Problem:
    """A reconstruction problem: geometry, true parameters (device), measured patterns (device)."""
    geom: Geometry
    truth: Params
    I_meas: torch.Tensor
    roi: tuple  # (r0, r1, c0, c1) of the depth-summed phase that the NMSE covers


def simulate(pt: Ptycho, params: Params, idx: np.ndarray, batch: int, gen: torch.Generator,
             out: torch.Tensor | None = None) -> torch.Tensor:
    """Poisson counts of the modelled patterns for scan positions idx, [len(idx), N, N] float32."""
    N = pt.geom.N
    if out is None:
        out = torch.empty((len(idx), N, N), dtype=torch.float32, device=pt.device)
    for s in range(0, len(idx), batch):
        b = idx[s:s + batch]
        I = pt.forward(params, b)
        out[s:s + len(b)] = torch.poisson(I, generator=gen)
    return out


def problem(name: str = "c2", seed: int = 1237, device="cuda", batch: int = 512) -> Problem:
    """The synthetic workload `name` (synth.workload) with measured patterns simulated on the GPU."""
    w = synth.workload(name)
    truth = Params.from_numpy(w, device=device)
    geom = Geometry(N=w.N, M=w.M, Nz=w.Nz, H=w.H, W=w.W, Ntot=w.Ntot, dx=w.dx, lam=w.lam, loss="poisson",
                    grads=("amp", "phase"))
    pt = Ptycho(geom, batch, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    I = simulate(pt, truth, np.arange(w.Ntot), batch, gen)
    pos = w.pos
    r0 = int(np.floor(pos[:, 0].min())) + w.N // 2
    r1 = int(np.ceil(pos[:, 0].max())) + w.N // 2
    c0 = int(np.floor(pos[:, 1].min())) + w.N // 2
    c1 = int(np.ceil(pos[:, 1].max())) + w.N // 2
    return Problem(geom, truth, I, (r0, r1, c0, c1))


def nmse(phase_hat: torch.Tensor, phase: torch.Tensor, roi) -> float:
    """Object NMSE on the depth-summed phase inside roi with the global offset removed:
    sum (d - mean d)^2 / sum (phi - mean phi)^2, d = phi_hat - phi."""
    r0, r1, c0, c1 = roi
    a = phase_hat.sum(0)[r0:r1, c0:c1].double().cpu().numpy()
    b = phase.sum(0)[r0:r1, c0:c1].double().cpu().numpy()
    d = a - b
    d -= d.mean()
    e = b - b.mean()
    return float((d * d).sum() / (e * e).sum())


def training_set(prob: Problem, n_objects: int, per_object: int, seed0: int = 2000, batch: int = 512):
    """(I [n, N, N], Y [n, N/2, N/2, 2]) on the device: random Gaussian-atom volumes of the problem's
    shape (seeds seed0, seed0 + 1, ...), random window positions, the problem's probe, tilt and dz."""
    g = prob.geom
    dev = prob.I_meas.device
    n = n_objects * per_object
    I = torch.empty((n, g.N, g.N), dtype=torch.float32, device=dev)
    Y = torch.empty((n, g.N // 2, g.N // 2, 2), dtype=torch.float32, device=dev)
    geom = dataclasses.replace(g, Ntot=per_object, grads=())
    pt = Ptycho(geom, batch, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed0)
    for k in range(n_objects):
        rng = np.random.default_rng(seed0 + k)
        amp, phase = synth.make_object_3d(g.Nz, g.H, g.W, g.dx, seed=seed0 + k)
        pos = np.stack([rng.uniform(0, g.H - g.N - 1, per_object), rng.uniform(0, g.W - g.N - 1, per_object)], 1)
        tilt = prob.truth.tilt[:1].expand(per_object, 2).contiguous()
        f32 = dict(dtype=torch.float32, device=dev)
        params = Params(amp=torch.tensor(amp, **f32), phase=torch.tensor(phase, **f32), probe=prob.truth.probe,
                        pos=torch.tensor(pos, **f32), tilt=tilt, dz=prob.truth.dz)
        sl = slice(k * per_object, (k + 1) * per_object)
        simulate(pt, params, np.arange(per_object), batch, gen, out=I[sl])
        idx = torch.arange(per_object, dtype=torch.int32, device=dev)
        targets(g.N, params.amp, params.phase, params.pos, idx, out=Y[sl])
    return I, Y


def train(net: Cnn, I: torch.Tensor, Y: torch.Tensor, epochs: int, batch: int, lr: float, seed: int = 2100,
          log=None) -> list:
    """Adam over shuffled batches; returns the mean training loss of every epoch."""
    n = I.shape[0]
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        perm = torch.tensor(rng.permutation(n), device=I.device)
        tot = torch.zeros((), dtype=torch.float64, device=I.device)
        nb = 0
        for s in range(0, n - batch + 1, batch):
            sel = perm[s:s + batch]
            loss = net.train_step(I[sel].contiguous(), Y[sel].contiguous(), lr=lr)
            tot += loss[0]
            nb += 1
        hist.append(tot.item() / max(nb, 1))
        if log:
            log("epoch %d loss %.4g" % (ep, hist[-1]))
    return hist


def probe_weight(probe: torch.Tensor) -> torch.Tensor:
    """Stitching weight: intensity of the first probe mode on the central (N/2)^2 of the window."""
    N = probe.shape[-1]
    q = N // 4
    w = probe[0].abs() ** 2
    return (w / w.max())[q:q + N // 2, q:q + N // 2].float().contiguous()


def probe_estimate(prob: Problem, defocus_A: float, dose: float = 1e5) -> torch.Tensor:
    """A starting probe from nominal settings: the workload's probe model (synth.make_probe: same
    aperture, modes, mode powers and dose) with defocus `defocus_A` instead of the true value."""
    g = prob.geom
    p = synth.make_probe(g.N, g.M, g.dx, defocus_A=defocus_A, dose=dose)
    return torch.tensor(p, dtype=torch.complex64, device=prob.I_meas.device)


def initial_object(net: Cnn, prob: Problem, batch: int = 256, probe: torch.Tensor | None = None):
    """CNN predictions for every measured pattern, stitched into amp, phase [Nz, H, W].  The
    stitching weight comes from `probe` (default: the true probe)."""
    g = prob.geom
    w = probe_weight(prob.truth.probe if probe is None else probe)
    st = Stitcher(g.N, g.Nz, g.H, g.W, w, device=prob.I_meas.device)
    for s in range(0, g.Ntot, batch):
        idx = torch.arange(s, min(s + batch, g.Ntot), dtype=torch.int32, device=prob.I_meas.device)
        pred = net.predict(prob.I_meas[s:s + idx.numel()].contiguous())
        st.add(pred, prob.truth.pos, idx)
    return st.finish()


def flat_object(prob: Problem, seed: int = 1234):
    """The paper's default start: amplitude 1, phase U[0, 1e-8]."""
    g = prob.geom
    amp, phase = synth.flat_object(g.Nz, g.H, g.W, seed=seed)
    f32 = dict(dtype=torch.float32, device=prob.I_meas.device)
    return torch.tensor(amp, **f32), torch.tensor(phase, **f32)


def reconstruct(prob: Problem, amp0: torch.Tensor, phase0: torch.Tensor, iters: int, batch: int, lr: dict,
                target: float = 0.05, seed: int = 7, fft: str = "fp32", eval_every: int = 8,
                probe0: torch.Tensor | None = None):
    """Adam on the object from (amp0, phase0), with positions, tilt and dz frozen at the truth; the
    probe is the truth, or starts at `probe0` and is refined too when `lr` has a "probe" rate.  One
    iteration = one pass over all positions in shuffled batches.  The NMSE is evaluated every
    `eval_every` batches (outside the timed work).  Returns the list of (iterations done, NMSE, GPU
    seconds of reconstruction so far), stopping once NMSE <= target."""
    names = ("amp", "phase") + (("probe",) if lr.get("probe") else ())
    g = dataclasses.replace(prob.geom, grads=names, fft=fft)
    dev = prob.I_meas.device
    pt = Ptycho(g, batch, device=dev)
    probe = prob.truth.probe if probe0 is None else probe0.clone()
    params = Params(amp=amp0.clone(), phase=phase0.clone(), probe=probe, pos=prob.truth.pos,
                    tilt=prob.truth.tilt, dz=prob.truth.dz)
    grads = params.zeros_like()
    adam = Adam(params, lr)
    rng = np.random.default_rng(seed)
    steps_per_pass = (g.Ntot + batch - 1) // batch
    hist = [(0.0, nmse(params.phase, prob.truth.phase, prob.roi), 0.0)]
    work = 0.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for it in range(iters):
        idx_all = torch.tensor(rng.permutation(g.Ntot).astype(np.int32), device=dev)
        for k in range(steps_per_pass):
            if k % eval_every == 0:
                ev0.record()
            step(pt, params, grads, adam, idx_all[k * batch:(k + 1) * batch], prob.I_meas)
            if (k + 1) % eval_every == 0 or k + 1 == steps_per_pass:
                ev1.record()
                ev1.synchronize()
                work += ev0.elapsed_time(ev1) / 1e3
                e = nmse(params.phase, prob.truth.phase, prob.roi)
                hist.append((it + (k + 1) / steps_per_pass, e, work))
                if e <= target:
                    return hist, params
    return hist, params
