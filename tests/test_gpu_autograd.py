"""Adjoint behind torch.autograd, the checkpoint / recompute plan, GPU finite differences, Adam.

* pty_loss_grad with ckpt_stride K > 1 (segments re-run from stored spectra) gives the oracle's
  gradients like K = 1;
* the autograd function (pty_forward_save + pty_backward) with a loss written in torch gives the
  same gradients as pty_loss_grad for that loss;
* central differences of the GPU forward model (h = 1e-3) agree with the GPU gradient;
* pty_step's Adam update equals torch.optim.Adam fed the same gradients.
"""
import numpy as np
import pytest

from oracle import ptycho as O
from tests.cases import make_case, oracle_grads, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_G = 1e-4
NAMES = ("amp", "phase", "probe", "pos", "tilt", "dz")


def _setup(case, **geom_kw):
    from paper_2505_07814_gb300.ptycho import Geometry, Params, Ptycho
    g = case.geom
    geom = Geometry(N=g.N, M=g.M, Nz=g.Nz, H=g.H, W=g.W, Ntot=case.Ntot, dx=g.dx, lam=g.lam, loss=g.loss,
                    global_tilt=g.global_tilt, **geom_kw)
    dev = torch.device("cuda")
    f32 = dict(dtype=torch.float32, device=dev)
    params = Params(amp=torch.tensor(case.amp, **f32), phase=torch.tensor(case.phase, **f32),
                    probe=torch.tensor(case.probe, dtype=torch.complex64, device=dev),
                    pos=torch.tensor(case.pos, **f32), tilt=torch.tensor(case.tilt, **f32),
                    dz=torch.tensor([case.dz], **f32))
    return Ptycho(geom, case.Ntot, device=dev), params, torch.tensor(case.I_meas, **f32)


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("N,M,Nz,scan,K", [(64, 2, 5, (2, 3), 2), (64, 2, 5, (2, 3), 3), (64, 2, 5, (2, 3), 5),
                                           (128, 2, 8, (2, 2), 3), (256, 2, 5, (2, 1), 2)])
def test_recompute_plan_matches_oracle(N, M, Nz, scan, K):
    case = make_case(N=N, M=M, Nz=Nz, scan=scan, seed=30 + K)
    idx = list(range(case.Ntot))[::-1]
    ref = oracle_grads(case, idx)
    pt, params, I_meas = _setup(case, ckpt_stride=K)
    loss, grads = pt.loss_grad(params, idx, I_meas)
    torch.cuda.synchronize()
    assert pt.status() == 0
    assert abs(loss.item() - ref.loss) <= 1e-5 * abs(ref.loss)
    for n in NAMES:
        got = _np(getattr(grads, n))
        err = rel_l2(got[0] if n == "dz" else got, getattr(ref, n))
        assert err <= TOL_G, (n, err)


def _torch_poisson(I, I_meas_b, eps=1e-6):
    I = I.to(torch.float64)
    d = I_meas_b.to(torch.float64)
    return -torch.mean(d * torch.log(I + eps) - I) / torch.mean(d)


@pytest.mark.parametrize("K", [1, 2])
def test_autograd_function_matches_loss_grad(K):
    from paper_2505_07814_gb300.ptycho import forward_model
    case = make_case(N=64, M=3, Nz=4, scan=(2, 3), seed=40 + K)
    idx = [3, 0, 5, 1]
    pt, params, I_meas = _setup(case, ckpt_stride=K)
    loss_ref, g_ref = pt.loss_grad(params, idx, I_meas)
    loss_ref = loss_ref.item()
    g_ref = {n: _np(getattr(g_ref, n)).copy() for n in NAMES}
    leaves = {n: getattr(params, n).clone().requires_grad_(True) for n in NAMES}
    from paper_2505_07814_gb300.ptycho import Params
    p = Params(**leaves)
    I = forward_model(pt, p, idx)
    loss = _torch_poisson(I, I_meas[torch.tensor(idx, device="cuda")])
    loss.backward()
    assert abs(loss.item() - loss_ref) <= 1e-5 * abs(loss_ref)
    for n in NAMES:
        err = rel_l2(_np(leaves[n].grad), g_ref[n])
        assert err <= TOL_G, (n, err)
    # backward without a matching forward on this workspace is refused
    I2 = forward_model(pt, p, idx)
    pt.forward_save(params, idx)  # another forward on the same workspace
    with pytest.raises(RuntimeError):
        _torch_poisson(I2, I_meas[torch.tensor(idx, device="cuda")]).backward()


def test_gpu_central_differences():
    """h = 1e-3 central differences of the GPU forward (loss in FP64 on the host) against the GPU
    gradient: single entries of the probe, positions, tilts and dz; random directions over the whole
    object arrays (one object pixel moves an FP32 loss by less than its rounding)."""
    case = make_case(N=64, M=2, Nz=3, scan=(2, 2), seed=50)
    idx = [0, 1, 2, 3]
    pt, params, I_meas = _setup(case)
    Im = _np(I_meas)[idx].astype(np.float64)
    g = O.Geometry(N=case.geom.N, M=case.geom.M, Nz=case.geom.Nz, H=case.geom.H, W=case.geom.W, dx=case.geom.dx,
                   lam=case.geom.lam)

    def loss_at(prm):
        I = _np(pt.forward(prm, idx)).astype(np.float64)
        return O.loss_value(g, I, Im)

    def shifted(name, delta):
        q = params.zeros_like()
        for n in NAMES:
            getattr(q, n).copy_(getattr(params, n))
        getattr(q, name).add_(delta)
        return q

    _, grads = pt.loss_grad(params, idx, I_meas)
    h = 1e-3
    rng = np.random.default_rng(51)
    checks = []
    for name in ("amp", "phase", "probe"):
        x = getattr(params, name)
        if name == "probe":  # direction scaled to the probe's size
            d = torch.tensor(rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape),
                             dtype=torch.complex64, device="cuda") * x.abs().mean()
        else:
            d = torch.tensor(rng.standard_normal(x.shape), dtype=torch.float32, device="cuda")
        fd = (loss_at(shifted(name, h * d)) - loss_at(shifted(name, -h * d))) / (2 * h)
        gd = getattr(grads, name) * d.conj() if name == "probe" else getattr(grads, name) * d
        checks.append((name, fd, float(gd.real.sum() if name == "probe" else gd.sum())))
    entries = {"pos": [(0, 0), (3, 1), (2, 0)], "tilt": [(1, 0), (2, 1)], "dz": [(0,)]}
    for name, es in entries.items():
        scale = 0.1 if name == "tilt" else 1.0  # tilt step 1e-4 rad: smaller steps drown in FP32 rounding
        for e in es:
            d = torch.zeros_like(getattr(params, name))
            d[e] = h * scale
            fd = (loss_at(shifted(name, d)) - loss_at(shifted(name, -d))) / (2 * h * scale)
            checks.append(((name, e), fd, float(_np(getattr(grads, name))[e])))
    for what, fd, an in checks:
        assert abs(fd - an) <= 1e-2 * abs(an) + 1e-7, (what, fd, an)


def test_adam_step_matches_torch_adam():
    from paper_2505_07814_gb300.ptycho import Adam, step
    case = make_case(N=64, M=2, Nz=3, scan=(2, 2), seed=60)
    idx = [2, 0, 3]
    pt, params, I_meas = _setup(case)
    lr = {"amp": 1e-3, "phase": 2e-3, "probe": 0.5, "pos": 1e-2, "tilt": 1e-5, "dz": 1e-2}
    # reference: torch.optim.Adam on copies, fed the gradients pty_step itself computed (a second
    # gradient call would differ in the last bits through the order of the float atomics, and Adam's
    # first steps turn that into sign-sized differences where a gradient is near zero)
    ref = {n: getattr(params, n).clone().requires_grad_(True) for n in NAMES}
    opt = torch.optim.Adam([{"params": [ref[n]], "lr": lr[n]} for n in NAMES], betas=(0.9, 0.999), eps=1e-8)
    adam = Adam(params, lr, betas=(0.9, 0.999), eps=1e-8)
    grads = params.zeros_like()
    for it in range(3):
        loss = step(pt, params, grads, adam, idx, I_meas)
        torch.cuda.synchronize()
        for n in NAMES:
            ref[n].grad = getattr(grads, n).clone()
        opt.step()
        torch.cuda.synchronize()
        for n in NAMES:
            a, b = _np(getattr(params, n)), _np(ref[n])
            assert np.allclose(a, b, rtol=2e-5, atol=1e-6 * max(1.0, np.abs(b).max())), (it, n)
