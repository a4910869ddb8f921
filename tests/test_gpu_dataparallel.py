"""A batch split into parts through the C ABI (pty_loss_stats, pty_loss_grad_part): the parts'
statistics summed and handed back reproduce the whole batch's loss and gradients, and each part
matches the FP64 oracle's part (reading R11: the whole batch's dL/dI, adjoint over the part)."""
import numpy as np
import pytest

from oracle import ptycho as O
from tests.cases import make_case, rel_l2
from tests.test_gpu_parity import TOL_G, TOL_I, _gpu, _np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ("amp", "phase", "probe", "pos", "tilt", "dz")


def _err(got, exp, name):
    if name == "dz":
        got = got[0]
    return rel_l2(got, exp)


@pytest.mark.parametrize("loss", [O.POISSON, O.GAUSSIAN])
@pytest.mark.parametrize("N", [64, 128])
def test_two_parts_with_accumulate_equal_the_whole_batch(loss, N):
    case = make_case(N=N, M=2, Nz=3, scan=(2, 3), loss=loss, seed=21)
    idx = [4, 0, 5, 2, 1, 3]
    parts = [idx[:2], idx[2:]]
    pt, params, I_meas = _gpu(case)
    # the whole batch in one call
    loss_w, g_w = pt.loss_grad(params, idx, I_meas)
    loss_w = loss_w.item()
    g_w = {n: _np(getattr(g_w, n)) for n in NAMES}
    # each part's statistics, summed (what an all-reduce does across ranks)
    stats = sum(pt.loss_stats(params, p, I_meas).clone() for p in parts)
    grads = params.zeros_like()
    shares = []
    for k, p in enumerate(parts):
        lk, grads = pt.loss_grad(params, p, I_meas, grads=grads, accumulate=k > 0, whole_stats=stats)
        shares.append(lk.item())
    torch.cuda.synchronize()
    assert pt.status() == 0
    assert abs(sum(shares) - loss_w) <= TOL_I * abs(loss_w)
    for n in NAMES:
        err = rel_l2(_np(getattr(grads, n)), g_w[n])
        assert err <= TOL_I * 10, (n, err)  # the same sums in another atomic order
    # each part against the oracle's part of the same whole batch
    for a, b in ((0, 2), (2, 6)):
        pt2, params2, I_meas2 = _gpu(case)
        lk, gk = pt2.loss_grad(params2, idx[a:b], I_meas2, whole_stats=stats)
        torch.cuda.synchronize()
        ref = O.loss_and_grad(case.geom, case.amp, case.phase, case.probe, case.pos, case.tilt, case.dz,
                              case.I_meas, idx, part=(a, b))
        assert abs(lk.item() - ref.loss) <= TOL_I * abs(ref.loss)
        for n in NAMES:
            err = _err(_np(getattr(gk, n)), getattr(ref, n), n)
            assert err <= TOL_G, (a, b, n, err)


@pytest.mark.parametrize("loss", [O.POISSON, O.GAUSSIAN])
def test_statistics_of_a_batch(loss):
    case = make_case(N=64, M=2, Nz=2, scan=(2, 2), loss=loss, seed=22)
    idx = [3, 1, 2]
    pt, params, I_meas = _gpu(case)
    st = _np(pt.loss_stats(params, idx, I_meas))
    I = O.model_patterns(case.geom, case.amp, case.phase, case.probe, case.pos, case.tilt, case.dz, idx)
    Id = np.stack([case.I_meas[j] for j in idx])
    p = case.geom.power
    S = np.sum(O._pow(Id, p))
    assert abs(st[0] - S) <= 1e-6 * S
    assert st[2] == I.size
    if loss == O.GAUSSIAN:
        Q = np.sum((O._pow(I, p) - O._pow(Id, p)) ** 2)
        assert abs(st[1] - Q) <= 1e-4 * Q
    else:
        assert st[1] == 0.0
    # empty part: zeros
    st0 = _np(pt.loss_stats(params, [], I_meas))
    assert not st0.any()


def test_part_call_refuses_batch_wide_terms():
    from paper_2505_07814_gb300 import _lib
    from paper_2505_07814_gb300.ptycho import Geometry, Ptycho
    case = make_case(N=64, M=1, Nz=1, scan=(1, 2), seed=23)
    pt, params, I_meas = _gpu(case)
    g = case.geom
    geom = Geometry(N=g.N, M=g.M, Nz=g.Nz, H=g.H, W=g.W, Ntot=case.Ntot, dx=g.dx, lam=g.lam, w_pacbed=0.2)
    pt2 = Ptycho(geom, 2)
    stats = torch.ones(3, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.PtyError) as e:
        pt2.loss_grad(params, [0, 1], I_meas, whole_stats=stats)
    assert e.value.code == _lib.PTY_EINVAL
