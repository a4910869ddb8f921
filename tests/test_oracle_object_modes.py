"""Pins of the oracle's mixed-state object (Eq. 2 with K object modes): the incoherent mode sum,
reduction to one mode, symmetry under relabelling the modes, and central differences of every
gradient through the whole forward model."""
import dataclasses

import numpy as np
import pytest

from oracle import ptycho as O
from tests.test_oracle import _small_problem


def _two_modes(loss=O.POISSON, **kw):
    geom, amp, phase, probe, pos, tilt, dz, I_meas = _small_problem(loss=loss, **kw)
    rng = np.random.default_rng(21)
    amp2 = np.stack([amp, 0.6 * amp * (1.0 + 0.05 * rng.standard_normal(amp.shape))])
    phase2 = np.stack([phase, 0.5 * phase + 0.1 * rng.standard_normal(phase.shape)])
    return dataclasses.replace(geom, K=2), amp2, phase2, probe, pos, tilt, dz, I_meas


def test_mode_sum_is_incoherent():
    g2, amp, phase, probe, pos, tilt, dz, _ = _two_modes()
    g1 = dataclasses.replace(g2, K=1)
    idx = [0, 1, 2]
    I2 = O.model_patterns(g2, amp, phase, probe, pos, tilt, dz, idx)
    parts = [O.model_patterns(g1, amp[n], phase[n], probe, pos, tilt, dz, idx) for n in range(2)]
    np.testing.assert_allclose(I2, parts[0] + parts[1], rtol=1e-13)
    # K identical modes: K times one mode
    same = O.model_patterns(g2, np.stack([amp[0]] * 2), np.stack([phase[0]] * 2), probe, pos, tilt, dz, idx)
    np.testing.assert_allclose(same, 2.0 * parts[0], rtol=1e-13)
    # one mode given as [1][Nz][H][W] is the plain object
    np.testing.assert_array_equal(O.model_patterns(g1, amp[:1], phase[:1], probe, pos, tilt, dz, idx), parts[0])


def test_relabelling_modes_permutes_gradients():
    g, amp, phase, probe, pos, tilt, dz, I_meas = _two_modes()
    a = O.loss_and_grad(g, amp, phase, probe, pos, tilt, dz, I_meas, [2, 0])
    b = O.loss_and_grad(g, amp[::-1].copy(), phase[::-1].copy(), probe, pos, tilt, dz, I_meas, [2, 0])
    assert np.isclose(a.loss, b.loss, rtol=1e-13)
    np.testing.assert_allclose(b.amp, a.amp[::-1], rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(b.phase, a.phase[::-1], rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(b.probe, a.probe, rtol=1e-11, atol=1e-15)
    assert a.amp.shape == amp.shape


def _total(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx):
    I = O.model_patterns(geom, amp, phase, probe, pos, tilt, dz, idx)
    Im = np.stack([I_meas[j] for j in idx])
    corners = [tuple(O.crop_index(pos[j])[0]) for j in idx]
    return (O.loss_value(geom, I, Im) + geom.w_pacbed * O.pacbed_value(geom, I, Im) +
            geom.w_sparse * O.sparse_value(geom, phase, corners))


@pytest.mark.parametrize("loss,w_pacbed,w_sparse", [(O.POISSON, 0.0, 0.0), (O.GAUSSIAN, 0.0, 0.0),
                                                    (O.POISSON, 0.3, 0.1)])
def test_object_mode_gradients_central_differences(loss, w_pacbed, w_sparse):
    geom, amp, phase, probe, pos, tilt, dz, I_meas = _two_modes(loss=loss)
    geom = dataclasses.replace(geom, w_pacbed=w_pacbed, w_sparse=w_sparse)
    idx = [1, 2, 0]
    g = O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx)
    assert np.isclose(g.loss, _total(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx), rtol=1e-13)
    rng = np.random.default_rng(9)
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
        analytic = np.sum(np.real(np.conj(gx) * d)) if name == "probe" else np.sum(gx * d)
        plus, minus = dict(args), dict(args)
        plus[name] = x + h * d
        minus[name] = x - h * d
        fd = (_total(geom, I_meas=I_meas, idx=idx, **plus) - _total(geom, I_meas=I_meas, idx=idx, **minus)) / (2 * h)
        assert abs(fd - analytic) <= 1e-6 * abs(analytic) + 1e-12, (name, fd, analytic)
