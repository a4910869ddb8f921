"""FP64 oracle of the object constraints applied after each optimiser step (Sec. "Physical
constraints": "Positivity and sparsity", and the r_z filter of "Real-space depth regularization",
Eq. 13).

TEST INFRASTRUCTURE ONLY: imported by tests/ alone.

Readings where the paper is silent (also listed in the design notes):
  C1  every constraint is applied with a relaxation r in [0, 1]: x <- x + r (C(x) - x), r = 1 being
      the plain constraint (the paper allows "relaxation to permit partial deviation");
  C2  the depth blur convolves the amplitude and the phase arrays separately (the object is stored
      and optimised as these two arrays) along the slice axis with a Gaussian of standard deviation
      sigma slices, truncated at 4 sigma; at the top and bottom of the volume the kernel is cut off
      and renormalised (no wrap, no padding);
  C3  order: depth blur, then positivity (clipping negative phase to zero), so the result of a step
      is non-negative when the positivity relaxation is 1.

Pins (tests/test_oracle_constraints.py): closed forms (constant volumes, sigma -> 0, full and zero
relaxation, symmetry under reversing the slice order) and scipy's 1D Gaussian filter as a library
special case (normalised convolution with zero padding).
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


def constrain(amp, phase, positivity_relax=0.0, rz_sigma=0.0, rz_relax=1.0):
    """One constraint step on the object (reading C3 for the order)."""
    amp = np.asarray(amp, dtype=np.float64)
    phase = np.asarray(phase, dtype=np.float64)
    if rz_sigma > 0 and rz_relax > 0:
        amp = rz_blur(amp, rz_sigma, rz_relax)
        phase = rz_blur(phase, rz_sigma, rz_relax)
    if positivity_relax > 0:
        phase = positivity(phase, positivity_relax)
    return amp, phase
