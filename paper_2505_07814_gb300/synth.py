"""Seeded synthetic inputs for multislice electron ptychography.

This module only *draws* inputs: probes, objects, scan positions, tilts, noise.
It holds none of the forward model or its adjoint, and it imports neither the
CUDA binding nor the FP64 oracle, so both sides of every parity test can take
their inputs from here without sharing arithmetic.

Shapes and value distributions follow the workloads the paper reconstructs
(Sec. "Physical model", mixed-state probe of M modes, multislice object of Nz
slices, raster scan with sub-pixel positions; Sec. "Preprocessing and
initialization" for the flat default start).  All arrays are numpy, float64 /
complex128, row-major, axis 0 = rows ("y"), axis 1 = columns ("x").
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Relativistic electron wavelength (Kirkland, "Advanced Computing in Electron
# Microscopy", Eq. 2.5): lambda = h / sqrt(2 m0 e V (1 + e V / (2 m0 c^2))).
# With lambda in angstrom and V in volt the constants are 12.2643 and 0.978476e-6.


def electron_wavelength_A(kV: float) -> float:
    V = kV * 1e3
    return 12.2643 / math.sqrt(V * (1.0 + 0.978476e-6 * V))


@dataclasses.dataclass
class Workload:
    """One synthetic reconstruction problem (all the inputs of a batch pass)."""

    N: int  # probe window / detector size (pixels per side)
    M: int  # incoherent probe modes
    Nz: int  # object slices
    H: int  # object rows
    W: int  # object columns
    dx: float  # real-space pixel size (angstrom)
    lam: float  # electron wavelength (angstrom)
    dz: float  # slice separation (angstrom)
    amp: np.ndarray  # [Nz][H][W] float64
    phase: np.ndarray  # [Nz][H][W] float64 (radian, = sigma * V)
    probe: np.ndarray  # [M][N][N] complex128
    pos: np.ndarray  # [Ntot][2] float64, top-left corner of each patch (pixels)
    tilt: np.ndarray  # [Ntot][2] float64 (radian)

    @property
    def Ntot(self) -> int:
        return self.pos.shape[0]


def mode_powers(M: int) -> np.ndarray:
    """First mode carries 0.6 of the dose, the rest decay geometrically by 1/2."""
    if M == 1:
        return np.ones(1)
    rest = 0.5 ** np.arange(M - 1)
    rest = 0.4 * rest / rest.sum()
    return np.concatenate([[0.6], rest])


def make_probe(N: int, M: int, dx: float, kV: float = 200.0, alpha_mrad: float = 20.0,
               defocus_A: float = 50.0, dose: float = 1e5, seed: int = 1236) -> np.ndarray:
    """Mixed-state STEM probe, [M][N][N] complex128, centred in the window.

    Base mode: inverse FFT of a hard aperture |k| <= alpha/lambda with a defocus
    aberration exp(-i pi lambda df |k|^2).  Further modes: the base mode times
    low-order monomials y^a x^b, Gram-Schmidt orthonormalised, each scaled to
    sqrt(power_k * dose) so the total intensity equals the dose.  The seed adds a
    tiny random perturbation to the monomial coefficients so modes are generic.
    """
    lam = electron_wavelength_A(kV)
    k = np.fft.fftfreq(N, d=dx)
    k0, k1 = np.meshgrid(k, k, indexing="ij")
    kk = k0 ** 2 + k1 ** 2
    aperture = (np.sqrt(kk) <= alpha_mrad * 1e-3 / lam).astype(np.float64)
    chi = np.exp(-1j * np.pi * lam * defocus_A * kk)
    base = np.fft.fftshift(np.fft.ifft2(aperture * chi))
    r = (np.arange(N) - N / 2) * dx
    y, x = np.meshgrid(r, r, indexing="ij")
    rng = np.random.default_rng(seed)
    monos = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2), (0, 3),
             (4, 0), (3, 1), (2, 2), (1, 3), (0, 4)]
    if M > len(monos):
        raise ValueError("at most %d probe modes" % len(monos))
    modes = []
    for a, b in monos[:M]:
        c = 1.0 + 0.05 * (rng.standard_normal() + 1j * rng.standard_normal())
        v = base * (y ** a) * (x ** b) * c
        for u in modes:
            v = v - np.vdot(u, v) * u
        v = v / np.linalg.norm(v)
        modes.append(v)
    p = mode_powers(M)
    return np.stack([np.sqrt(p[m] * dose) * modes[m] for m in range(M)])


def _gaussian_atoms(H, W, dx, centres_A, sigma_A, peak):
    """Sum of isotropic Gaussians of height `peak` at the given centres (angstrom)."""
    out = np.zeros((H, W))
    rad = int(math.ceil(5 * sigma_A / dx))
    for (cy, cx) in centres_A:
        iy, ix = int(round(cy / dx)), int(round(cx / dx))
        y0, y1 = max(iy - rad, 0), min(iy + rad + 1, H)
        x0, x1 = max(ix - rad, 0), min(ix + rad + 1, W)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = np.arange(y0, y1)[:, None] * dx - cy
        xx = np.arange(x0, x1)[None, :] * dx - cx
        out[y0:y1, x0:x1] += peak * np.exp(-(yy ** 2 + xx ** 2) / (2 * sigma_A ** 2))
    return out


def make_object_2d(H: int, W: int, dx: float, lattice_A: float = 3.0, jitter_A: float = 0.1,
                   sigma_A: float = 0.4, peak: float = 0.3, seed: int = 1234):
    """Single-slice object: Gaussian atoms on a jittered hexagonal lattice.

    Returns (amp [1][H][W] = 1, phase [1][H][W]).
    """
    rng = np.random.default_rng(seed)
    a = lattice_A
    centres = []
    ny = int(H * dx / (a * math.sqrt(3) / 2)) + 2
    nx = int(W * dx / a) + 2
    for i in range(-1, ny):
        for j in range(-1, nx):
            cy = i * a * math.sqrt(3) / 2
            cx = j * a + (a / 2 if i % 2 else 0.0)
            centres.append((cy + rng.uniform(-jitter_A, jitter_A),
                            cx + rng.uniform(-jitter_A, jitter_A)))
    phase = _gaussian_atoms(H, W, dx, centres, sigma_A, peak)[None]
    return np.ones_like(phase), phase


def make_object_3d(Nz: int, H: int, W: int, dx: float, density_per_A2: float = 0.1,
                   sigma_A: float = 0.4, peak: float = 0.3, seed: int = 1234):
    """Multislice object: per slice, atoms uniformly at random with the given areal density.

    Returns (amp [Nz][H][W] = 1, phase [Nz][H][W]).
    """
    rng = np.random.default_rng(seed)
    area = H * dx * W * dx
    phase = np.zeros((Nz, H, W))
    for s in range(Nz):
        n = rng.poisson(density_per_A2 * area)
        cy = rng.uniform(0, H * dx, n)
        cx = rng.uniform(0, W * dx, n)
        phase[s] = _gaussian_atoms(H, W, dx, list(zip(cy, cx)), sigma_A, peak)
    return np.ones_like(phase), phase


def make_scan(n0: int, n1: int, step_px: float, N: int, H: int, W: int,
              jitter_px: float = 0.3, seed: int = 1235) -> np.ndarray:
    """Raster scan of n0 x n1 patch corners, centred in the object, with uniform jitter.

    Returns pos [n0*n1][2] float64 = top-left corner (row, col) of each N x N patch.
    """
    rng = np.random.default_rng(seed)
    ext0 = (n0 - 1) * step_px + N
    ext1 = (n1 - 1) * step_px + N
    o0 = (H - ext0) / 2.0
    o1 = (W - ext1) / 2.0
    g0, g1 = np.meshgrid(np.arange(n0) * step_px + o0, np.arange(n1) * step_px + o1, indexing="ij")
    pos = np.stack([g0.ravel(), g1.ravel()], axis=1)
    pos = pos + rng.uniform(-jitter_px, jitter_px, pos.shape)
    r = np.round(pos)
    if (r.min() < 0) or (r[:, 0].max() + N > H) or (r[:, 1].max() + N > W):
        raise ValueError("scan does not fit in the object")
    return pos


def flat_object(Nz: int, H: int, W: int, seed: int = 1234):
    """Default start: amplitude 1, phase uniform in [0, 1e-8] (Sec. "Preprocessing and initialization")."""
    rng = np.random.default_rng(seed)
    return np.ones((Nz, H, W)), rng.uniform(0.0, 1e-8, (Nz, H, W))


def poisson_counts(I: np.ndarray, seed: int = 1237) -> np.ndarray:
    """Poisson noise on expected counts (the measured patterns of a simulated dataset)."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.maximum(I, 0.0)).astype(np.float64)


def vacuum_patterns(probe: np.ndarray, n: int, seed: int = 1237) -> np.ndarray:
    """n Poisson-noisy copies of the probe's bright-field disc, DC-centred, [n][N][N].

    Used only where a realistic-looking measured pattern is needed at a size the
    oracle cannot simulate in seconds (throughput runs); parity tests simulate
    their patterns with the oracle instead.
    """
    N = probe.shape[-1]
    disc = np.zeros((N, N))
    for P in probe:
        disc += np.abs(np.fft.fftshift(np.fft.fft2(P, norm="ortho"))) ** 2
    rng = np.random.default_rng(seed)
    out = np.empty((n, N, N), dtype=np.float32)
    for i in range(0, n, 64):  # chunks keep the integer draws small
        k = min(64, n - i)
        out[i:i + k] = rng.poisson(np.broadcast_to(disc, (k, N, N)))
    return out


# ---------------------------------------------------------------------------------------------
# Named workloads.  C1..C3 are the configurations the library is measured on; `small` cases
# span several tiles with ragged object sizes and still let the FP64 oracle finish in seconds.
# ---------------------------------------------------------------------------------------------

def workload(name: str, **over) -> Workload:
    kV = 200.0
    lam = electron_wavelength_A(kV)
    dx = 0.1
    if name == "c1":  # 2D ptychography, 64x64 probe, 1 mode, 16x16 scan, object 128^2
        N, M, Nz, H, W, dz = 64, 1, 1, 128, 128, 1.0
        amp, phase = make_object_2d(H, W, dx)
        pos = make_scan(16, 16, 4, N, H, W)
        tilt = np.zeros_like(pos)
    elif name == "c4":  # the single-slice physics of c1 with a 128x128 window: object 192^2
        N, M, Nz, H, W, dz = 128, 1, 1, 192, 192, 1.0
        amp, phase = make_object_2d(H, W, dx)
        pos = make_scan(16, 16, 4, N, H, W)
        tilt = np.zeros_like(pos)
    elif name == "c2":  # multislice: 128x128, 6 modes, 8 slices of 512^2, 64x64 scan
        N, M, Nz, H, W, dz = 128, 6, 8, 512, 512, 2.0
        amp, phase = make_object_3d(Nz, H, W, dx)
        pos = make_scan(64, 64, 4, N, H, W)
        tilt = np.tile(np.array([0.5e-3, -0.3e-3]), (pos.shape[0], 1))
    elif name == "c3":  # scale: 256x256, 12 modes, 20 slices of 1024^2, 128x128 scan
        N, M, Nz, H, W, dz = 256, 12, 20, 1024, 1024, 2.0
        amp, phase = make_object_3d(Nz, H, W, dx)
        pos = make_scan(128, 128, 4, N, H, W)
        tilt = np.tile(np.array([0.5e-3, -0.3e-3]), (pos.shape[0], 1))
    elif name == "paper":  # shaped like the paper's twisted-bilayer reconstruction: 12 modes, 6 slices
        N, M, Nz, H, W, dz = 128, 12, 6, 614, 614, 2.0
        amp, phase = make_object_3d(Nz, H, W, dx)
        pos = make_scan(128, 128, 3.8, N, H, W)
        tilt = np.tile(np.array([0.5e-3, -0.3e-3]), (pos.shape[0], 1))
    elif name == "small":  # ragged multislice case for parity tests
        N = over.pop("N", 64)
        M = over.pop("M", 3)
        Nz = over.pop("Nz", 3)
        n0, n1 = over.pop("scan", (3, 4))
        step = over.pop("step", 5)
        H = (n0 - 1) * step + N + over.pop("pad0", 7)
        W = (n1 - 1) * step + N + over.pop("pad1", 10)
        dz = over.pop("dz", 2.0)
        amp, phase = make_object_3d(Nz, H, W, dx, seed=over.pop("seed", 1234))
        rng = np.random.default_rng(99)
        amp = amp * (1.0 + 0.05 * rng.standard_normal(amp.shape))
        pos = make_scan(n0, n1, step, N, H, W)
        rng = np.random.default_rng(98)
        tilt = np.stack([0.5e-3 + 0.3e-3 * rng.standard_normal(pos.shape[0]),
                         -0.3e-3 + 0.3e-3 * rng.standard_normal(pos.shape[0])], axis=1)
    else:
        raise KeyError(name)
    probe = make_probe(N, M, dx, kV=kV, dose=over.pop("dose", 1e5))
    if over:
        raise TypeError("unused overrides: %s" % sorted(over))
    return Workload(N=N, M=M, Nz=Nz, H=H, W=W, dx=dx, lam=lam, dz=dz, amp=amp, phase=phase,
                    probe=probe, pos=pos, tilt=tilt)
