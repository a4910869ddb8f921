"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a brute-force sum, a closed form of
continuous Fourier optics, an identity of the model, a hand-computed example, or a
finite difference of the oracle's own loss (which checks its hand-written adjoint).
"""
import json
import os

import numpy as np
import pytest

from oracle import ptycho as O
from paper_2505_07814_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _brute_dft2(x, sign=-1):
    N0, N1 = x.shape
    out = np.zeros_like(x, dtype=np.complex128)
    for k0 in range(N0):
        for k1 in range(N1):
            acc = 0j
            for r0 in range(N0):
                for r1 in range(N1):
                    acc += x[r0, r1] * np.exp(sign * 2j * np.pi * (k0 * r0 / N0 + k1 * r1 / N1))
            out[k0, k1] = acc
    return out


@pytest.mark.parametrize("N", [8, 16])
def test_dft_matches_bruteforce(N):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    ref = _brute_dft2(x)
    assert np.max(np.abs(O.dft2(x) - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(O.idft2(ref) - x)) <= 1e-12 * np.max(np.abs(x))
    # orthonormal far field = DFT / N
    assert np.max(np.abs(O.far_field(x) - ref / N)) <= 1e-12 * np.max(np.abs(ref))


def test_far_field_parseval():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))
    a, b = np.sum(np.abs(O.far_field(x)) ** 2), np.sum(np.abs(x) ** 2)
    assert abs(a - b) <= 1e-13 * b


def test_propagator_unitary_and_semigroup():
    N, dx, lam = 64, 0.1, 0.0251
    th = (3e-3, -2e-3)
    M1 = O.propagator(N, dx, lam, 1.3, th)
    M2 = O.propagator(N, dx, lam, 2.2, th)
    M3 = O.propagator(N, dx, lam, 3.5, th)
    assert np.max(np.abs(np.abs(M1) - 1)) < 1e-14
    assert np.max(np.abs(M1 * M2 - M3)) < 1e-12
    rng = np.random.default_rng(2)
    psi = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    out = O.idft2(M1 * O.dft2(psi))
    assert abs(np.linalg.norm(out) - np.linalg.norm(psi)) < 1e-12 * np.linalg.norm(psi)


@pytest.mark.parametrize("theta", [(0.0, 0.0), (1e-2, -0.6e-2)])
def test_propagator_gaussian_closed_form(theta):
    """Fresnel propagation of exp(-pi r^2 / a) over dz with tilt theta has the closed form
    a/(a + i lam dz) exp(-pi |r + dz tan(theta)|^2 / (a + i lam dz)) (continuous Fourier optics:
    FT of exp(-pi r^2/a) is a exp(-pi a k^2); the tilt term exp(2 pi i dz k.tan(theta)) translates
    by -dz tan(theta)).  Pins the sign and scale of both terms of Eq. 4 and the frequency grid."""
    N, dx, lam, dz, a = 128, 0.1, 0.0251, 50.0, 1.0
    r = (np.arange(N) - N // 2) * dx
    y, x = np.meshgrid(r, r, indexing="ij")
    psi0 = np.exp(-np.pi * (y ** 2 + x ** 2) / a)
    out = O.idft2(O.propagator(N, dx, lam, dz, theta) * O.dft2(psi0))
    q = a + 1j * lam * dz
    s0, s1 = dz * np.tan(theta[0]), dz * np.tan(theta[1])
    ref = a / q * np.exp(-np.pi * ((y + s0) ** 2 + (x + s1) ** 2) / q)
    assert np.max(np.abs(out - ref)) < 1e-10


def test_shift_operator_integer_is_roll():
    rng = np.random.default_rng(3)
    P = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    out = O.shift_operator(P, np.array([2.0, -3.0]))
    assert np.max(np.abs(out - np.roll(P, (2, -3), axis=(0, 1)))) < 1e-12


def test_crop_index_rounding():
    r, dr = O.crop_index([2.5, 3.5])
    assert tuple(r) == (2, 4)  # half to even
    r, dr = O.crop_index([7.3, -0.2 + 5])
    assert tuple(r) == (7, 5) and np.allclose(dr, [0.3, -0.2])


def _small_problem(N=16, M=2, Nz=3, n_pos=3, seed=0, H=27, W=30, loss=O.POISSON, global_tilt=False):
    rng = np.random.default_rng(seed)
    geom = O.Geometry(N=N, M=M, Nz=Nz, H=H, W=W, dx=0.2, lam=0.0251, loss=loss,
                      global_tilt=global_tilt)
    amp = 1.0 + 0.1 * rng.standard_normal((Nz, H, W))
    phase = 0.3 * rng.standard_normal((Nz, H, W))
    probe = (rng.standard_normal((M, N, N)) + 1j * rng.standard_normal((M, N, N))) * 3.0
    pos = np.stack([rng.uniform(0.7, H - N - 0.7, n_pos), rng.uniform(0.7, W - N - 0.7, n_pos)], 1)
    # keep clear of the round() discontinuity at .5
    frac = pos - np.floor(pos)
    pos = np.where(np.abs(frac - 0.5) < 0.05, pos + 0.1, pos)
    tilt = rng.normal(0, 1e-2, (2,) if global_tilt else (n_pos, 2))
    dz = 3.0
    # measured data from a different object, plus noise
    amp_t = 1.0 + 0.1 * rng.standard_normal((Nz, H, W))
    phase_t = 0.3 * rng.standard_normal((Nz, H, W))
    I_t = O.model_patterns(geom, amp_t, phase_t, probe, pos, tilt, dz, range(n_pos))
    I_meas = np.maximum(I_t + 0.5 * rng.standard_normal(I_t.shape), 0.0)
    return geom, amp, phase, probe, pos, tilt, dz, I_meas


def _loss(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx):
    I = O.model_patterns(geom, amp, phase, probe, pos, tilt, dz, idx)
    return O.loss_value(geom, I, np.stack([I_meas[j] for j in idx]))


@pytest.mark.parametrize("loss", [O.POISSON, O.GAUSSIAN])
@pytest.mark.parametrize("global_tilt", [False, True])
def test_gradients_match_central_differences(loss, global_tilt):
    """Directional central differences of the oracle's own loss for every gradient kind."""
    geom, amp, phase, probe, pos, tilt, dz, I_meas = _small_problem(loss=loss, global_tilt=global_tilt)
    idx = [2, 0, 1]
    g = O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx)
    assert np.isclose(g.loss, _loss(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx), rtol=1e-13)
    rng = np.random.default_rng(7)
    args = dict(amp=amp, phase=phase, probe=probe, pos=pos, tilt=tilt, dz=dz)
    steps = dict(amp=1e-5, phase=1e-5, probe=1e-5, pos=1e-5, tilt=1e-6, dz=1e-5)
    for name, h in steps.items():
        x = args[name]
        if name == "dz":
            d = 1.0
        elif name == "probe":
            d = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
        else:
            d = rng.standard_normal(np.shape(x))
        gx = getattr(g, name)
        if name == "probe":
            analytic = np.sum(np.real(np.conj(gx) * d))
        else:
            analytic = np.sum(gx * d)
        plus, minus = dict(args), dict(args)
        plus[name] = x + h * d
        minus[name] = x - h * d
        fd = (_loss(geom, I_meas=I_meas, idx=idx, **plus) - _loss(geom, I_meas=I_meas, idx=idx, **minus)) / (2 * h)
        assert abs(fd - analytic) <= 1e-6 * abs(analytic) + 1e-12, (name, fd, analytic)


def test_gradient_single_entries_central_differences():
    """Entry-wise checks (catches errors a random direction could average out)."""
    geom, amp, phase, probe, pos, tilt, dz, I_meas = _small_problem(seed=5)
    idx = [0, 1, 2]
    g = O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx)
    h = 1e-6

    def fd(name, index, dval=1.0):
        a = dict(amp=amp.copy(), phase=phase.copy(), probe=probe.copy(), pos=pos.copy(),
                 tilt=tilt.copy(), dz=dz)
        b = dict(amp=amp.copy(), phase=phase.copy(), probe=probe.copy(), pos=pos.copy(),
                 tilt=tilt.copy(), dz=dz)
        a[name][index] += h * dval
        b[name][index] -= h * dval
        return (_loss(geom, I_meas=I_meas, idx=idx, **a) - _loss(geom, I_meas=I_meas, idx=idx, **b)) / (2 * h)

    r0, _ = O.crop_index(pos[1])
    for name in ["amp", "phase"]:
        index = (1, int(r0[0]) + 5, int(r0[1]) + 7)
        assert np.isclose(fd(name, index), getattr(g, name)[index], rtol=1e-6, atol=1e-12)
    # untouched pixel has zero gradient
    assert g.amp[0, geom.H - 1, 0] == 0.0 or geom.H - 1 < int(min(pos[:, 0])) + geom.N
    for index in [(0, 3, 4), (1, 8, 2)]:
        re = fd("probe", index, 1.0)
        im = fd("probe", index, 1j)
        assert np.isclose(re, g.probe[index].real, rtol=1e-6, atol=1e-12)
        assert np.isclose(im, g.probe[index].imag, rtol=1e-6, atol=1e-12)
    for index in [(0, 0), (2, 1)]:
        assert np.isclose(fd("pos", index), g.pos[index], rtol=1e-6, atol=1e-12)
        assert np.isclose(fd("tilt", index), g.tilt[index], rtol=1e-6, atol=1e-12)


def test_dz_zero_is_product_of_transmissions():
    geom, amp, phase, probe, pos, tilt, dz, _ = _small_problem(Nz=4)
    T = O.transmission(amp, phase)
    r, dr = O.crop_index(pos[1])
    Oj = O.object_patch(T, r, geom.N)
    Pj = O.shift_operator(probe[0], dr)
    Mj = O.propagator(geom.N, geom.dx, geom.lam, 0.0, tilt[1])
    ref = Pj * Oj[0] * Oj[1] * Oj[2] * Oj[3]
    assert np.max(np.abs(O.exit_wave(Pj, Oj, Mj) - ref)) < 1e-12 * np.max(np.abs(ref))


def test_crop_places_patch():
    """A single bright pixel of the object lands at (y - r0, x - r1) of the exit wave (Nz = 1)."""
    N, H, W = 16, 40, 40
    phase = np.zeros((1, H, W))
    phase[0, 20, 23] = 0.7
    T = O.transmission(np.ones_like(phase), phase)
    r, _ = O.crop_index([12.2, 9.6])
    Oj = O.object_patch(T, r, N)
    psi = O.exit_wave(np.ones((N, N)), Oj, np.ones((N, N)))
    ang = np.angle(psi)
    assert np.unravel_index(np.argmax(ang), ang.shape) == (20 - 12, 23 - 10)
    with pytest.raises(IndexError):
        O.object_patch(T, np.array([30, 0]), N)


def test_vacuum_object_invariants():
    """amp 1, phase 0: I_j = sum_m |F_ortho P_m|^2 for every position, and the loss does not
    depend on positions, tilts or dz (|F[S P]| = |F P|, propagation is a pure k-space phase)."""
    geom, amp, phase, probe, pos, tilt, dz, I_meas = _small_problem(Nz=3)
    amp = np.ones_like(amp)
    phase = np.zeros_like(phase)
    idx = [0, 1, 2]
    g = O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx)
    ref = np.fft.fftshift(sum(np.abs(np.fft.fft2(P, norm="ortho")) ** 2 for P in probe))
    for b in range(3):
        assert np.max(np.abs(g.I_model[b] - ref)) < 1e-10 * ref.max()
    scale = np.max(np.abs(g.phase))
    assert scale > 0
    assert np.max(np.abs(g.pos)) < 1e-10 * scale
    assert np.max(np.abs(g.tilt)) < 1e-10 * scale
    assert abs(g.dz) < 1e-10 * scale


def test_pure_phase_conserves_mode_power():
    geom, amp, phase, probe, pos, tilt, dz, _ = _small_problem(Nz=3)
    I = O.model_patterns(geom, np.ones_like(amp), phase, probe, pos, tilt, dz, [0, 1, 2])
    total = sum(np.sum(np.abs(P) ** 2) for P in probe)
    for b in range(3):
        assert abs(I[b].sum() - total) < 1e-12 * total


def test_mode_sum_is_linear():
    geom, amp, phase, probe, pos, tilt, dz, _ = _small_problem(M=3)
    I = O.model_patterns(geom, amp, phase, probe, pos, tilt, dz, [0, 1])
    g1 = O.Geometry(**{**geom.__dict__, "M": 1})
    parts = sum(O.model_patterns(g1, amp, phase, probe[m:m + 1], pos, tilt, dz, [0, 1]) for m in range(3))
    assert np.max(np.abs(I - parts)) < 1e-12 * np.max(I)


def test_loss_golden_values():
    d = json.load(open(os.path.join(GOLDEN, "loss_toy.json")))
    g = O.Geometry(N=2, M=1, Nz=1, H=2, W=2, dx=1.0, lam=1.0, loss=O.GAUSSIAN)
    c = d["gaussian_p05"]
    Im, Id = np.array(c["I_model"], float)[None], np.array(c["I_meas"], float)[None]
    assert np.isclose(O.loss_value(g, Im, Id), c["loss"], rtol=1e-14)
    assert np.allclose(O.loss_grad_I(g, Im, Id)[0], c["dLdI"], rtol=1e-13, atol=1e-16)
    g = O.Geometry(N=2, M=1, Nz=1, H=2, W=2, dx=1.0, lam=1.0, loss=O.POISSON, eps=0.0)
    c = d["poisson_p1_eps0"]
    Im, Id = np.array(c["I_model"], float)[None], np.array(c["I_meas"], float)[None]
    assert np.isclose(O.loss_value(g, Im, Id), c["loss"], rtol=1e-14)
    assert np.allclose(O.loss_grad_I(g, Im, Id)[0], c["dLdI"], rtol=1e-13)
    # the default eps = 1e-6 moves the values only at the 1e-6 level
    g.eps = 1e-6
    assert np.isclose(O.loss_value(g, Im, Id), c["loss"], rtol=1e-5)


def test_gaussian_loss_zero_at_truth():
    geom, amp, phase, probe, pos, tilt, dz, _ = _small_problem(loss=O.GAUSSIAN)
    I = O.model_patterns(geom, amp, phase, probe, pos, tilt, dz, [0, 1, 2])
    g = O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I, [0, 1, 2])
    assert g.loss == 0.0
    for a in (g.amp, g.phase, g.probe, g.pos, g.tilt):
        assert np.max(np.abs(a)) == 0.0
    assert g.dz == 0.0


def test_gaussian_grad_guard_at_zero_intensity():
    g = O.Geometry(N=2, M=1, Nz=1, H=2, W=2, dx=1.0, lam=1.0, loss=O.GAUSSIAN)
    Im = np.array([[[0.0, 1.0], [4.0, 9.0]]])
    Id = np.array([[[1.0, 1.0], [1.0, 1.0]]])
    d = O.loss_grad_I(g, Im, Id)
    assert d[0, 0, 0] == 0.0 and np.all(np.isfinite(d))


def test_wavelength_and_parameter_count_golden():
    c = json.load(open(os.path.join(GOLDEN, "constants.json")))
    w = c["electron_wavelength"]
    assert abs(synth.electron_wavelength_A(w["kV"]) - w["lambda_A"]) < w["abs_tol_A"]
    p = c["parameter_count"]
    obj = 2 * p["Nz"] * p["H"] * p["W"]  # amplitude + phase arrays
    probe = 2 * p["M"] * p["N"] ** 2  # complex
    positions = 2 * p["Ntot"]
    assert (obj, probe, positions) == (p["object"], p["probe"], p["positions"])
    assert obj + probe + positions == p["total"]
    assert p["N"] ** 4 == p["measurements"]


def test_synthetic_probe_dose_and_orthogonality():
    P = synth.make_probe(64, 4, 0.1, dose=1e5)
    G = np.einsum("mij,nij->mn", P.conj(), P)
    assert abs(np.trace(G).real - 1e5) < 1e-6 * 1e5
    off = G - np.diag(np.diag(G))
    assert np.max(np.abs(off)) < 1e-9 * 1e5
    assert np.allclose(np.diag(G).real / 1e5, synth.mode_powers(4))
