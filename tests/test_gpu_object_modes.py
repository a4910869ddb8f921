"""Mixed-state object (pty_geom.obj_modes = K, Eq. 2) through the C ABI against the FP64 oracle.

Waves run as (position, probe mode, object mode) triples: every path that indexes waves or the
object is covered (forward, adjoint, recompute, the four-CTA clusters at N = 256, the split-precision
GEMM form, the sparsity and PACBED terms, the constraints applied per mode, the Adam step).
Tolerances as the single-mode parity tests: FP32 intensities and loss <= 1e-5 relative L2,
gradients <= 1e-4; the three-piece bf16 split form <= 1e-4 / 1e-3.
"""
import dataclasses

import numpy as np
import pytest

from oracle import constraints as KC
from oracle import ptycho as O
from tests.cases import f32, make_case, oracle_grads, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRADS = ("amp", "phase", "probe", "pos", "tilt", "dz")


def _modes(case, K, seed=40):
    """K object modes: the case's object and K - 1 weaker, perturbed copies (float32-exact)."""
    rng = np.random.default_rng(seed)
    amps, phases = [case.amp], [case.phase]
    for n in range(1, K):
        amps.append(f32(case.amp * (0.7 - 0.1 * n) * (1.0 + 0.03 * rng.standard_normal(case.amp.shape))))
        phases.append(f32(case.phase * (0.5 + 0.2 * n) + 0.02 * rng.standard_normal(case.phase.shape)))
    return dataclasses.replace(case, geom=dataclasses.replace(case.geom, K=K), amp=np.stack(amps),
                               phase=np.stack(phases))


def _gpu(case, grads=GRADS, **geo):
    from paper_2505_07814_gb300.ptycho import Geometry, Params, Ptycho
    g = case.geom
    geom = Geometry(N=g.N, M=g.M, Nz=g.Nz, H=g.H, W=g.W, Ntot=case.Ntot, dx=g.dx, lam=g.lam, loss=g.loss,
                    eps=g.eps, grads=tuple(grads), global_tilt=g.global_tilt, obj_modes=g.K,
                    w_pacbed=g.w_pacbed, w_sparse=g.w_sparse, **geo)
    dev = torch.device("cuda")
    t32 = dict(dtype=torch.float32, device=dev)
    params = Params(amp=torch.tensor(case.amp, **t32), phase=torch.tensor(case.phase, **t32),
                    probe=torch.tensor(case.probe, dtype=torch.complex64, device=dev),
                    pos=torch.tensor(case.pos, **t32), tilt=torch.tensor(case.tilt, **t32),
                    dz=torch.tensor([case.dz], **t32))
    return Ptycho(geom, case.Ntot, device=dev), params, torch.tensor(case.I_meas, **t32)


def _np(t):
    return t.detach().cpu().numpy()


def _check(case, idx, tol_i=1e-5, tol_g=1e-4, **geo):
    pt, params, I_meas = _gpu(case, **geo)
    I_model = torch.empty((len(idx), case.geom.N, case.geom.N), dtype=torch.float32, device="cuda")
    loss, grads = pt.loss_grad(params, idx, I_meas, I_model=I_model)
    torch.cuda.synchronize()
    assert pt.status() == 0
    ref = oracle_grads(case, idx)
    assert rel_l2(_np(I_model), ref.I_model) <= tol_i
    assert abs(loss.item() - ref.loss) <= tol_i * abs(ref.loss)
    for name in GRADS:
        got = _np(getattr(grads, name))
        err = rel_l2(got[0] if name == "dz" else got, getattr(ref, name))
        assert err <= tol_g, (name, err)
    I_fwd = pt.forward(params, idx)
    torch.cuda.synchronize()
    assert rel_l2(_np(I_fwd), ref.I_model) <= tol_i


@pytest.mark.parametrize("loss", [O.POISSON, O.GAUSSIAN])
def test_two_object_modes_n64(loss):
    case = _modes(make_case(N=64, M=2, Nz=3, scan=(3, 4), loss=loss), 2)
    _check(case, [5, 0, 11, 3, 7, 1, 2, 9, 4, 10, 6, 8])


def test_three_object_modes_n128_recompute():
    case = _modes(make_case(N=128, M=1, Nz=3, scan=(2, 2), seed=2), 3)
    _check(case, [3, 1, 0, 2], ckpt_stride=2)


def test_object_modes_n256_cluster():
    case = _modes(make_case(N=256, M=1, Nz=2, scan=(2, 2), seed=12, step=9), 2)
    _check(case, [2, 0, 3, 1])


def test_object_modes_split_bf16x3():
    case = _modes(make_case(N=64, M=2, Nz=2, scan=(2, 3), seed=3), 2)
    _check(case, [0, 4, 2, 1, 5, 3], tol_i=1e-4, tol_g=1e-3, fft="bf16x3")


def test_object_modes_with_pacbed_and_sparsity():
    case = _modes(make_case(N=64, M=2, Nz=2, scan=(3, 3), seed=4), 2)
    case = dataclasses.replace(case, geom=dataclasses.replace(case.geom, w_pacbed=0.3, w_sparse=0.1))
    _check(case, [8, 0, 4, 2, 6, 1])


def test_identical_modes_double_the_patterns():
    """K identical object modes: every pattern is exactly K times the single-mode pattern (Eq. 2)."""
    base = make_case(N=64, M=2, Nz=2, scan=(2, 3), seed=5)
    idx = [0, 1, 2, 3, 4, 5]
    pt1, p1, _ = _gpu(base)
    I1 = _np(pt1.forward(p1, idx))
    two = dataclasses.replace(base, geom=dataclasses.replace(base.geom, K=2), amp=np.stack([base.amp] * 2),
                              phase=np.stack([base.phase] * 2))
    pt2, p2, _ = _gpu(two)
    I2 = _np(pt2.forward(p2, idx))
    torch.cuda.synchronize()
    assert rel_l2(I2, 2.0 * I1) <= 1e-6


def test_constraints_apply_per_mode():
    from paper_2505_07814_gb300.ptycho import constrain
    case = _modes(make_case(N=64, M=1, Nz=4, scan=(2, 2), seed=6), 2)
    pt, params, _ = _gpu(case)
    constrain(pt, params, phase_positivity=1.0, rz_sigma=1.0, kz_beta=1.0, kz_alpha=0.02, kz_relax=0.8)
    torch.cuda.synchronize()
    for n in range(2):
        ra, rp = KC.constrain(case.amp[n], case.phase[n], 1.0, 1.0, 1.0, kz_beta=1.0, kz_alpha=0.02, kz_relax=0.8,
                              dx=case.geom.dx, dz=case.dz)
        np.testing.assert_allclose(_np(params.amp)[n], ra, rtol=1e-5, atol=2e-5)
        np.testing.assert_allclose(_np(params.phase)[n], rp, rtol=1e-5, atol=2e-5)


def test_adam_step_updates_every_mode():
    from paper_2505_07814_gb300.ptycho import Adam, step
    case = _modes(make_case(N=64, M=1, Nz=2, scan=(2, 2), seed=7), 2)
    pt, params, I_meas = _gpu(case)
    before = _np(params.amp).copy()
    adam = Adam(params, lr={"amp": 1e-3, "phase": 1e-3, "probe": 0.0, "pos": 0.0, "tilt": 0.0, "dz": 0.0})
    grads = params.zeros_like()
    step(pt, params, grads, adam, [0, 1, 2, 3], I_meas)
    torch.cuda.synchronize()
    assert pt.status() == 0
    moved = np.abs(_np(params.amp) - before)
    assert moved[0].max() > 0 and moved[1].max() > 0
    ref = oracle_grads(case, [0, 1, 2, 3])
    # the first Adam step moves every touched entry by lr * sign(gradient)
    # (away from |g| ~ eps = 1e-8, where the step is smaller, and from entries FP32 cannot resolve)
    touched = np.abs(ref.amp) > max(1e-5, 1e-4 * np.abs(ref.amp).max())
    np.testing.assert_allclose(((_np(params.amp) - before) / -1e-3)[touched], np.sign(ref.amp[touched]), atol=2e-3)
