"""Pins of the PACBED and sparsity terms of the oracle's total loss (Eq. 7-9): closed forms and
central differences, alone and through the whole forward model."""
import dataclasses

import numpy as np
import pytest

from oracle import ptycho as O
from tests.test_oracle import _small_problem


def _geom(**kw):
    return O.Geometry(N=8, M=1, Nz=2, H=20, W=20, dx=0.2, lam=0.0251, **kw)


def test_pacbed_closed_forms():
    rng = np.random.default_rng(0)
    I = rng.uniform(0.5, 5.0, (4, 8, 8))
    g = _geom(p_pacbed=1.0)
    assert O.pacbed_value(g, I, I) == 0.0
    assert not O.pacbed_grad_I(g, I, I).any()
    # only the batch means enter: permuting or reshuffling mass between patterns changes nothing
    J = I[::-1].copy()
    J[0] += 1.0
    J[1] -= 1.0
    Im = rng.uniform(0.5, 5.0, (4, 8, 8))
    assert np.isclose(O.pacbed_value(g, I, Im), O.pacbed_value(g, J, Im), rtol=1e-13)
    # one pattern, p = 1, model = c * measurement: |c - 1| sqrt(<I^2>) / <I>
    c = 1.7
    assert np.isclose(O.pacbed_value(g, c * I[:1], I[:1]),
                      abs(c - 1) * np.sqrt(np.mean(I[0] ** 2)) / np.mean(I[0]), rtol=1e-13)


@pytest.mark.parametrize("p", [0.5, 1.0])
def test_pacbed_gradient_central_differences(p):
    rng = np.random.default_rng(1)
    I = rng.uniform(0.5, 5.0, (3, 8, 8))
    Im = rng.uniform(0.5, 5.0, (3, 8, 8))
    g = _geom(p_pacbed=p)
    G = O.pacbed_grad_I(g, I, Im)
    D = rng.standard_normal(I.shape)
    h = 1e-6
    fd = (O.pacbed_value(g, I + h * D, Im) - O.pacbed_value(g, I - h * D, Im)) / (2 * h)
    assert abs(fd - np.sum(G * D)) <= 1e-7 * abs(fd)


def test_sparse_closed_forms():
    g = _geom(p_sparse=1.0)
    phase = np.zeros((2, 20, 20))
    phase[:, 2:10, 3:11] = -0.4  # the patch at corner (2, 3)
    corners = [(2, 3), (2, 3)]
    assert np.isclose(O.sparse_value(g, phase, corners), 0.4)
    G = O.sparse_grad_phase(g, phase, corners)
    n = 2 * 2 * 64  # two positions x two slices x 8 x 8
    np.testing.assert_allclose(G[:, 2:10, 3:11], -2.0 / n)  # reached twice, sign -1, 1/n each
    assert not G[:, :2].any() and not G[:, 10:].any()
    # p = 2: the RMS
    g2 = _geom(p_sparse=2.0)
    rng = np.random.default_rng(2)
    ph = rng.standard_normal((2, 20, 20))
    v = np.concatenate([ph[:, 1:9, 4:12].ravel(), ph[:, 6:14, 0:8].ravel()])
    assert np.isclose(O.sparse_value(g2, ph, [(1, 4), (6, 0)]), np.sqrt(np.mean(v ** 2)), rtol=1e-13)


@pytest.mark.parametrize("p", [1.0, 2.0, 0.7])
def test_sparse_gradient_central_differences(p):
    g = _geom(p_sparse=p)
    rng = np.random.default_rng(3)
    ph = rng.standard_normal((2, 20, 20))
    corners = [(1, 4), (6, 0), (3, 3)]
    G = O.sparse_grad_phase(g, ph, corners)
    D = rng.standard_normal(ph.shape)
    h = 1e-7
    fd = (O.sparse_value(g, ph + h * D, corners) - O.sparse_value(g, ph - h * D, corners)) / (2 * h)
    assert abs(fd - np.sum(G * D)) <= 1e-6 * abs(fd)


def _total_loss(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx):
    """The total loss from its definitions: Eq. 5/6 + w_pacbed Eq. 7 + w_sparse Eq. 8."""
    I = O.model_patterns(geom, amp, phase, probe, pos, tilt, dz, idx)
    Im = np.stack([I_meas[j] for j in idx])
    corners = [tuple(O.crop_index(pos[j])[0]) for j in idx]
    return (O.loss_value(geom, I, Im) + geom.w_pacbed * O.pacbed_value(geom, I, Im) +
            geom.w_sparse * O.sparse_value(geom, phase, corners))


@pytest.mark.parametrize("loss", [O.POISSON, O.GAUSSIAN])
def test_total_loss_gradients_central_differences(loss):
    geom, amp, phase, probe, pos, tilt, dz, I_meas = _small_problem(loss=loss)
    geom = dataclasses.replace(geom, w_pacbed=0.3, w_sparse=0.1)
    idx = [2, 0, 1]
    g = O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx)
    assert np.isclose(g.loss, _total_loss(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx), rtol=1e-13)
    rng = np.random.default_rng(8)
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
        fd = (_total_loss(geom, I_meas=I_meas, idx=idx, **plus) -
              _total_loss(geom, I_meas=I_meas, idx=idx, **minus)) / (2 * h)
        assert abs(fd - analytic) <= 1e-6 * abs(analytic) + 1e-12, (name, fd, analytic)
