"""Pins of the oracle's split-batch reading (R11): a batch split into parts (data-parallel ranks or
accumulated sub-batches) against the whole batch's loss (Eq. 5/6) and gradient."""
import dataclasses

import numpy as np
import pytest

from oracle import ptycho as O
from tests.test_oracle import _small_problem

PARTS = [(0, 2), (2, 3), (3, 5)]


def _grads(prob, idx, part=None):
    geom, amp, phase, probe, pos, tilt, dz, I_meas = prob
    return O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx, part=part)


@pytest.mark.parametrize("loss", [O.POISSON, O.GAUSSIAN])
@pytest.mark.parametrize("global_tilt", [False, True])
def test_parts_add_up_to_the_whole_batch(loss, global_tilt):
    """Shares of the loss and part gradients add up to the whole batch's (linearity of the adjoint
    in dL/dI); a part computed against its own patterns only would not."""
    prob = _small_problem(n_pos=5, loss=loss, global_tilt=global_tilt, seed=3)
    idx = [4, 1, 0, 3, 2]
    whole = _grads(prob, idx)
    parts = [_grads(prob, idx, part=p) for p in PARTS]
    assert np.isclose(sum(p.loss for p in parts), whole.loss, rtol=1e-12, atol=0)
    for name in ("amp", "phase", "probe", "pos", "tilt"):
        tot = sum(getattr(p, name) for p in parts)
        ref = getattr(whole, name)
        assert np.linalg.norm((tot - ref).ravel()) <= 1e-12 * np.linalg.norm(ref.ravel()), name
    assert np.isclose(sum(p.dz for p in parts), whole.dz, rtol=1e-11)
    # a part normalised by its own patterns (the plain call on the sub-batch) differs
    geom, amp, phase, probe, pos, tilt, dz, I_meas = prob
    own = O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx[0:2])
    assert not np.allclose(own.amp, parts[0].amp, rtol=1e-3)
    # position gradients of a part are zero outside its own positions
    assert not parts[0].pos[[idx[k] for k in range(2, 5)]].any()


@pytest.mark.parametrize("loss", [O.POISSON, O.GAUSSIAN])
def test_part_gradient_is_the_whole_loss_through_that_part(loss):
    """Directional central differences of the whole batch's loss in which only the part's patterns
    see the perturbed parameters (the definition of a part's gradient)."""
    prob = _small_problem(n_pos=4, loss=loss, seed=5)
    geom, amp, phase, probe, pos, tilt, dz, I_meas = prob
    idx = [0, 1, 2, 3]
    a, b = 1, 3
    I0 = O.model_patterns(geom, amp, phase, probe, pos, tilt, dz, idx)
    Im = np.stack([I_meas[j] for j in idx])

    def L(amp_, phase_, probe_):
        I = I0.copy()
        I[a:b] = O.model_patterns(geom, amp_, phase_, probe_, pos, tilt, dz, idx[a:b])
        return O.loss_value(geom, I, Im)

    g = _grads(prob, idx, part=(a, b))
    rng = np.random.default_rng(9)
    h = 1e-6
    for name in ("amp", "phase", "probe"):
        d = rng.standard_normal(np.shape({"amp": amp, "phase": phase, "probe": probe}[name]))
        if name == "probe":
            d = d + 1j * rng.standard_normal(d.shape)
        args_p = dict(amp_=amp, phase_=phase, probe_=probe)
        args_m = dict(args_p)
        args_p[name + "_"] = args_p[name + "_"] + h * d
        args_m[name + "_"] = args_m[name + "_"] - h * d
        fd = (L(**args_p) - L(**args_m)) / (2 * h)
        G = getattr(g, name)
        an = np.sum(np.real(np.conj(G) * d)) if name == "probe" else np.sum(G * d)
        assert abs(fd - an) <= 1e-6 * abs(fd), (name, fd, an)


def test_whole_part_is_the_plain_call():
    prob = _small_problem(n_pos=3, loss=O.GAUSSIAN, seed=7)
    idx = [2, 0, 1]
    a = _grads(prob, idx)
    b = _grads(prob, idx, part=(0, 3))
    assert np.isclose(a.loss, b.loss, rtol=1e-13)
    np.testing.assert_allclose(a.amp, b.amp, rtol=0, atol=1e-15 * np.abs(a.amp).max())


def test_split_terms_are_refused():
    prob = list(_small_problem(n_pos=2, seed=1))
    prob[0] = dataclasses.replace(prob[0], w_pacbed=0.1)
    with pytest.raises(ValueError):
        _grads(prob, [0, 1], part=(0, 1))
