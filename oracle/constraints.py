"""FP64 oracle of the constraints applied after each optimiser step (Sec. "Physical constraints"):
positivity, the r_z filter of "Real-space depth regularization" (Eq. 13), the k_z "missing wedge"
filter of "Fourier-space depth regularization" (Eq. 10-12) and the orthogonalisation of the
mixed-state probe modes.

TEST INFRASTRUCTURE ONLY: imported by tests/ alone.

Readings where the paper is silent (also listed in the design notes):
  C1  every constraint is applied with a relaxation r in [0, 1]: x <- x + r (C(x) - x), r = 1 being
      the plain constraint (the paper allows "relaxation to permit partial deviation");
  C2  the depth blur convolves the amplitude and the phase arrays separately (the object is stored
      and optimised as these two arrays) along the slice axis with a Gaussian of standard deviation
      sigma slices, truncated at 4 sigma; at the top and bottom of the volume the kernel is cut off
      and renormalised (no wrap, no padding);
  C3  order: k_z filter, then depth blur, then positivity (clipping negative phase to zero), so the
      result of a step is non-negative when the positivity relaxation is 1;
  C4  the k_z filter, like the blur, acts on the amplitude and the phase arrays separately, through
      the periodic 3D DFT of the object's own Nz x H x W extent (no padding: the wrap-around the
      paper describes); k_x, k_y, k_z are the DFT frequencies in cycles per angstrom for the pixel
      size dx and the slice spacing dz; eps = 1e-3 (per square angstrom) as printed under Eq. 10;
  C5  orthogonalisation: the probe modes P_m (the rows of an M x N^2 matrix A) are replaced by the
      eigenmodes of their density matrix, Q = U^H A with A A^H = U diag(lambda) U^H, ordered by
      decreasing power lambda; each column of U is given the phase that makes its largest-magnitude
      entry real and positive, so the result is unique where the powers are distinct.  It is not
      relaxed.

Pins (tests/test_oracle_constraints.py): closed forms (constant volumes, sigma -> 0, full and zero
relaxation, symmetry under reversing the slice order) and scipy's 1D Gaussian filter as a library
special case (normalised convolution with zero padding); for the k_z filter, plane waves (the DFT's
eigenfunctions) at frequencies where Eq. 10 takes closed values (W = 1 laterally and at k = 0,
W = 1/2 where beta^2 k_z^2 = k_r^2 + eps); for the orthogonalisation, numpy's SVD as a library
special case, the invariant density matrix, orthonormal output and sorted powers.
"""
from __future__ import annotations

import math

import numpy as np


def relax(x, cx, r):
    return x + r * (cx - x)


def positivity(phase, r=1.0):
    """Clip negative phase to zero, relaxed by r."""
    phase = np.asarray(phase, dtype=np.float64)
    return relax(phase, np.maximum(phase, 0.0), r)


def rz_weights(sigma):
    """Gaussian taps w[d], d = -R..R, R = ceil(4 sigma) (unnormalised)."""
    R = int(math.ceil(4.0 * sigma))
    d = np.arange(-R, R + 1, dtype=np.float64)
    return d, np.exp(-0.5 * (d / sigma) ** 2)


def rz_blur(x, sigma, r=1.0):
    """Depth blur of [Nz, H, W] along axis 0 (reading C2), relaxed by r."""
    x = np.asarray(x, dtype=np.float64)
    if sigma <= 0:
        return x.copy()
    Nz = x.shape[0]
    d, w = rz_weights(sigma)
    out = np.zeros_like(x)
    for s in range(Nz):
        num = np.zeros(x.shape[1:])
        den = 0.0
        for dd, ww in zip(d, w):
            t = s + int(dd)
            if 0 <= t < Nz:
                num += ww * x[t]
                den += ww
        out[s] = num / den
    return relax(x, out, r)


KZ_EPS = 1e-3  # per square angstrom, the stabilising constant of Eq. 10


def kz_weights(shape, dx, dz, beta, alpha):
    """W_a(k) of Eq. 10-11 on the 3D DFT grid of an object of shape (Nz, H, W) (reading C4)."""
    Nz, H, W = shape
    kz = np.fft.fftfreq(Nz, dz)[:, None, None]
    ky = np.fft.fftfreq(H, dx)[None, :, None]
    kx = np.fft.fftfreq(W, dx)[None, None, :]
    kr2 = kx ** 2 + ky ** 2
    w = 1.0 - (2.0 / np.pi) * np.arctan(beta ** 2 * kz ** 2 / (kr2 + KZ_EPS))
    return w * np.exp(-alpha * kr2)


def kz_filter(x, dx, dz, beta, alpha, r=1.0):
    """O' = F3^-1[W_a F3[O]] (Eq. 12) on one real array of shape (Nz, H, W), relaxed by r."""
    x = np.asarray(x, dtype=np.float64)
    y = np.real(np.fft.ifftn(kz_weights(x.shape, dx, dz, beta, alpha) * np.fft.fftn(x)))
    return relax(x, y, r)


def orthogonalize_probe(probe):
    """Eigenmodes of the mixed-state probe's density matrix (reading C5); probe is [M][N][N]."""
    probe = np.asarray(probe, dtype=np.complex128)
    M = probe.shape[0]
    A = probe.reshape(M, -1)
    G = A @ A.conj().T  # G[m][n] = sum_p P_m[p] conj(P_n[p])
    lam, U = np.linalg.eigh(G)
    order = np.argsort(-lam, kind="stable")
    lam, U = lam[order], U[:, order]
    for k in range(M):
        m = int(np.argmax(np.abs(U[:, k])))
        if abs(U[m, k]) > 0:
            U[:, k] *= np.conj(U[m, k]) / abs(U[m, k])
    return (U.conj().T @ A).reshape(probe.shape), lam


def constrain(amp, phase, positivity_relax=0.0, rz_sigma=0.0, rz_relax=1.0, kz_beta=0.0, kz_alpha=0.0,
              kz_relax=0.0, dx=1.0, dz=1.0):
    """One constraint step on the object (reading C3 for the order)."""
    amp = np.asarray(amp, dtype=np.float64)
    phase = np.asarray(phase, dtype=np.float64)
    if kz_relax > 0 and (kz_beta > 0 or kz_alpha > 0):
        amp = kz_filter(amp, dx, dz, kz_beta, kz_alpha, kz_relax)
        phase = kz_filter(phase, dx, dz, kz_beta, kz_alpha, kz_relax)
    if rz_sigma > 0 and rz_relax > 0:
        amp = rz_blur(amp, rz_sigma, rz_relax)
        phase = rz_blur(phase, rz_sigma, rz_relax)
    if positivity_relax > 0:
        phase = positivity(phase, positivity_relax)
    return amp, phase
