"""What a plain FP32 evaluation of the forward model and its adjoint reaches against the FP64 oracle.

The same formulas as the oracle (Eq. 1-6 and the hand-written adjoint), evaluated with numpy's
complex64 FFTs (pocketfft computes them in single precision) and every array in complex64 /
float32.  This is not a reference for the CUDA kernels: it measures the error floor of FP32
arithmetic on a given input, so that a GPU result that misses a bar can be told apart from one
that any FP32 evaluation would miss too.  Object gradients only (the Poisson loss).
"""
from __future__ import annotations

import numpy as np

from oracle import ptycho as O

C = np.complex64
F = np.float32


def object_gradients_fp32(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx):
    """(dL/damp, dL/dphase) of the Poisson loss of batch idx, every step in single precision."""
    assert geom.loss == O.POISSON and geom.K == 1 and geom.power == 1.0
    N, M, Nz = geom.N, geom.M, geom.Nz
    T = (np.asarray(amp) * np.exp(1j * np.asarray(phase))).astype(C)
    recs, I_model = [], np.zeros((len(idx), N, N), F)
    for b, j in enumerate(idx):
        r, dr = O.crop_index(pos[j])
        Mj = O.propagator(N, geom.dx, geom.lam, dz, O.tilt_of(geom, tilt, j)).astype(C)
        R = O.shift_ramp(N, dr).astype(C)
        Oj = T[:, r[0]:r[0] + N, r[1]:r[1] + N]
        waves = []
        I = np.zeros((N, N), F)
        for m in range(M):
            psi = np.fft.ifft2(np.fft.fft2(probe[m].astype(C)) * R)
            psi_in = []
            for s in range(Nz):
                psi_in.append(psi)
                u = Oj[s] * psi
                psi = np.fft.ifft2(Mj * np.fft.fft2(u)) if s < Nz - 1 else u
            Psi = np.fft.fft2(psi, norm="ortho")
            I += Psi.real ** 2 + Psi.imag ** 2
            waves.append((psi_in, Psi))
        I_model[b] = np.fft.fftshift(I)
        recs.append((r, Mj, Oj, waves))
    Im = np.stack([np.asarray(I_meas[j], dtype=F) for j in idx])
    S = F(Im.astype(np.float64).sum())
    dLdI = (-(Im / (I_model + F(geom.eps)) - F(1)) / S).astype(F)
    gT = np.zeros_like(T)
    for b, (r, Mj, Oj, waves) in enumerate(recs):
        w = np.fft.ifftshift(dLdI[b])
        for psi_in, Psi in waves:
            g = np.fft.ifft2((F(2) * w * Psi).astype(C), norm="ortho")
            for s in range(Nz - 1, -1, -1):
                gT[s, r[0]:r[0] + N, r[1]:r[1] + N] += np.conj(psi_in[s]) * g
                g = np.conj(Oj[s]) * g
                if s > 0:
                    g = np.fft.ifft2(np.conj(Mj) * np.fft.fft2(g))
    g_amp = np.real(np.conj(np.exp(1j * np.asarray(phase)).astype(C)) * gT)
    g_phase = np.imag(np.conj(T) * gT)  # Re(conj(i T) gT)
    return g_amp.astype(np.float64), g_phase.astype(np.float64)
