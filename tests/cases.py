"""Seeded parity cases shared by the GPU tests: inputs from the generator module, expected values
from the FP64 oracle, the same float32-rounded numbers fed to both sides."""
from __future__ import annotations

import dataclasses

import numpy as np

from oracle import ptycho as O
from paper_2505_07814_gb300 import synth

F32 = np.float32


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def c64(x):
    return np.asarray(x, dtype=np.complex64).astype(np.complex128)


@dataclasses.dataclass
class Case:
    geom: O.Geometry
    amp: np.ndarray
    phase: np.ndarray
    probe: np.ndarray
    pos: np.ndarray
    tilt: np.ndarray
    dz: float
    I_meas: np.ndarray  # [Ntot][N][N]

    @property
    def Ntot(self):
        return self.pos.shape[0]


def make_case(N=64, M=3, Nz=3, scan=(3, 4), loss=O.POISSON, global_tilt=False, seed=0, step=5,
              pad=(7, 10), dz=2.0, dose=1e5, perturb=True) -> Case:
    w = synth.workload("small", N=N, M=M, Nz=Nz, scan=scan, step=step, pad0=pad[0], pad1=pad[1], dz=dz,
                       dose=dose, seed=1234 + seed)
    geom = O.Geometry(N=N, M=M, Nz=Nz, H=w.H, W=w.W, dx=w.dx, lam=float(F32(w.lam)), loss=loss,
                      global_tilt=global_tilt)
    tilt = w.tilt[0] if global_tilt else w.tilt
    # the truth (float32-exact) produces the measured data
    amp_t, phase_t, probe_t, pos_t, tilt_t = f32(w.amp), f32(w.phase), c64(w.probe), f32(w.pos), f32(tilt)
    dz_t = float(F32(w.dz))
    I = O.model_patterns(geom, amp_t, phase_t, probe_t, pos_t, tilt_t, dz_t, range(len(pos_t)))
    I_meas = f32(synth.poisson_counts(I, seed=1237 + seed))
    if not perturb:
        return Case(geom, amp_t, phase_t, probe_t, pos_t, tilt_t, dz_t, I_meas)
    # the point at which loss and gradients are evaluated: a perturbed estimate
    rng = np.random.default_rng(500 + seed)
    amp = f32(amp_t * (1.0 + 0.02 * rng.standard_normal(amp_t.shape)))
    phase = f32(0.8 * phase_t + 0.01 * rng.standard_normal(phase_t.shape))
    probe = c64(probe_t * (1.0 + 0.05 * (rng.standard_normal(probe_t.shape) + 1j * rng.standard_normal(probe_t.shape))))
    pos = f32(pos_t + rng.uniform(-0.2, 0.2, pos_t.shape))
    tilt_e = f32(tilt_t + 2e-4 * rng.standard_normal(tilt_t.shape))
    return Case(geom, amp, phase, probe, pos, tilt_e, float(F32(dz_t * 1.1)), I_meas)


def oracle_grads(case: Case, idx):
    g = case.geom
    return O.loss_and_grad(g, case.amp, case.phase, case.probe, case.pos, case.tilt, case.dz, case.I_meas, idx)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)
