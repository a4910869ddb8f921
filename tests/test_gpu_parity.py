"""CUDA path (through the C ABI) against the FP64 oracle on seeded inputs.

Tolerances: FP32 intensities and loss to relative L2 <= 1e-5, gradients to relative L2 <= 1e-4
(the object and probe gradients are summed with float atomics, so their last bits depend on the
order in which CTAs finish).
"""
import numpy as np
import pytest

from oracle import ptycho as O
from tests.cases import make_case, oracle_grads, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_I = 1e-5
TOL_G = 1e-4


def _gpu(case, grads=("amp", "phase", "probe", "pos", "tilt", "dz"), max_batch=None):
    from paper_2505_07814_gb300.ptycho import Geometry, Params, Ptycho
    g = case.geom
    geom = Geometry(N=g.N, M=g.M, Nz=g.Nz, H=g.H, W=g.W, Ntot=case.Ntot, dx=g.dx, lam=g.lam, loss=g.loss,
                    eps=g.eps, grads=tuple(grads), global_tilt=g.global_tilt)
    dev = torch.device("cuda")
    f32 = dict(dtype=torch.float32, device=dev)
    params = Params(amp=torch.tensor(case.amp, **f32), phase=torch.tensor(case.phase, **f32),
                    probe=torch.tensor(case.probe, dtype=torch.complex64, device=dev),
                    pos=torch.tensor(case.pos, **f32), tilt=torch.tensor(case.tilt, **f32),
                    dz=torch.tensor([case.dz], **f32))
    pt = Ptycho(geom, max_batch or case.Ntot, device=dev)
    I_meas = torch.tensor(case.I_meas, **f32)
    return pt, params, I_meas


def _np(t):
    return t.detach().cpu().numpy()


def _check_all(case, idx, grads_names=("amp", "phase", "probe", "pos", "tilt", "dz")):
    pt, params, I_meas = _gpu(case, grads_names)
    B = len(idx)
    I_model = torch.empty((B, case.geom.N, case.geom.N), dtype=torch.float32, device="cuda")
    loss, grads = pt.loss_grad(params, idx, I_meas, I_model=I_model)
    torch.cuda.synchronize()
    assert pt.status() == 0
    ref = oracle_grads(case, idx)
    assert rel_l2(_np(I_model), ref.I_model) <= TOL_I
    assert abs(loss.item() - ref.loss) <= TOL_I * abs(ref.loss)
    for name in grads_names:
        got = _np(getattr(grads, name))
        exp = getattr(ref, name)
        if name == "dz":
            got = got[0]
        err = rel_l2(got, exp)
        assert err <= TOL_G, (name, err)
    # forward-only entry point agrees with the modelled patterns of the gradient call
    I_fwd = pt.forward(params, idx)
    torch.cuda.synchronize()
    assert rel_l2(_np(I_fwd), ref.I_model) <= TOL_I
    return pt, params, I_meas, ref


@pytest.mark.parametrize("loss", [O.POISSON, O.GAUSSIAN])
def test_multislice_multimode_n64(loss):
    case = make_case(N=64, M=3, Nz=3, scan=(3, 4), loss=loss)
    _check_all(case, [5, 0, 11, 3, 7, 1, 2, 9, 4, 10, 6, 8])


def test_multislice_n128():
    case = make_case(N=128, M=2, Nz=3, scan=(2, 3), seed=1)
    _check_all(case, [0, 1, 2, 3, 4, 5])


def test_multislice_n256_cluster():
    """256 x 256 windows: each wave spread over a four-CTA cluster."""
    case = make_case(N=256, M=3, Nz=3, scan=(2, 2), seed=12, step=9)
    _check_all(case, [2, 0, 3, 1])


@pytest.mark.parametrize("loss", [O.GAUSSIAN])
def test_n256_gaussian_global_tilt(loss):
    case = make_case(N=256, M=2, Nz=2, scan=(1, 3), seed=13, loss=loss, global_tilt=True)
    _check_all(case, [1, 2, 0])


def test_single_slice_single_mode_n64():
    """The 2D ptychography shape (1 mode, 1 slice): no propagation, dz/tilt gradients are 0."""
    case = make_case(N=64, M=1, Nz=1, scan=(4, 4), seed=2)
    _check_all(case, list(range(16)))


def test_adjoint_wave_order_full_and_ragged_groups():
    """40 positions: the adjoint takes its waves in groups of 32 positions (modes outermost inside a
    group), so this batch has one full group and a ragged group of 8; every gradient must still be
    the oracle's."""
    case = make_case(N=64, M=3, Nz=2, scan=(5, 8), seed=21, step=4)
    idx = list(range(40))
    idx = idx[7:] + idx[:7]
    _check_all(case, idx)


def test_global_tilt_and_ragged_batch():
    case = make_case(N=64, M=2, Nz=4, scan=(3, 3), global_tilt=True, seed=3)
    _check_all(case, [8, 2, 5, 0, 7])  # B = 5: partial batch of a 9-position scan


def test_six_modes_eight_slices_n128():
    """The multislice workload's mode / slice counts at a reduced scan."""
    case = make_case(N=128, M=6, Nz=8, scan=(2, 2), seed=4)
    _check_all(case, [3, 1, 0, 2])


def test_repeated_index_and_accumulate():
    case = make_case(N=64, M=2, Nz=2, scan=(2, 3), seed=5)
    pt, params, I_meas = _gpu(case)
    # batch with a repeated position: its gradient contributions add
    idx = [1, 4, 1]
    loss, grads = pt.loss_grad(params, idx, I_meas)
    ref = oracle_grads(case, idx)
    assert abs(loss.item() - ref.loss) <= TOL_I * abs(ref.loss)
    for name in ("amp", "phase", "probe", "pos", "tilt"):
        assert rel_l2(_np(getattr(grads, name)), getattr(ref, name)) <= TOL_G, name
    # accumulate = 1 adds a second batch's gradient onto the first
    first = [0, 2]
    second = [3, 5]
    loss, g = pt.loss_grad(params, first, I_meas)
    loss, g = pt.loss_grad(params, second, I_meas, grads=g, accumulate=True)
    r1, r2 = oracle_grads(case, first), oracle_grads(case, second)
    for name in ("amp", "phase", "probe", "pos", "tilt"):
        assert rel_l2(_np(getattr(g, name)), getattr(r1, name) + getattr(r2, name)) <= TOL_G, name
    assert abs(_np(g.dz)[0] - (r1.dz + r2.dz)) <= TOL_G * (abs(r1.dz) + abs(r2.dz))


def test_empty_batch():
    case = make_case(N=64, M=1, Nz=2, scan=(2, 2), seed=6)
    pt, params, I_meas = _gpu(case)
    grads = params.zeros_like()
    for t in (grads.amp, grads.phase, grads.pos, grads.tilt, grads.dz):
        t.fill_(7.0)
    grads.probe.fill_(7.0)
    loss, grads = pt.loss_grad(params, [], I_meas, grads=grads)
    torch.cuda.synchronize()
    assert loss.item() == 0.0
    for t in (grads.amp, grads.phase, grads.probe, grads.pos, grads.tilt, grads.dz):
        assert torch.count_nonzero(t).item() == 0
    assert pt.forward(params, []).shape == (0, 64, 64)


def test_patch_outside_object_sets_status_and_stays_in_bounds():
    case = make_case(N=64, M=1, Nz=1, scan=(2, 2), seed=7)
    pt, params, I_meas = _gpu(case)
    params.pos[1, 0] = case.geom.H  # patch would start at the last row
    pt.forward(params, [0, 1])
    assert pt.status() & 2  # PTY_EBOUNDS
    params.pos[1, 0] = float("nan")
    pt.forward(params, [1])
    assert pt.status() & 2
    params.pos[1, 0] = float(case.pos[1, 0])
    pt.forward(params, [0, 1])
    assert pt.status() == 0


@pytest.mark.parametrize("N", [64, 128])
def test_gradient_mask_subsets(N):
    """Only the requested gradients are computed; the others are untouched (may be absent).  At
    N = 128 the mask also decides which once-read blocks the adjoint bulk-copies into shared memory
    (checkpoints for the object gradient, spectra for dz / tilt, none for probe and positions)."""
    case = make_case(N=N, M=2, Nz=3, scan=(2, 2), seed=8)
    idx = [0, 1, 2, 3]
    ref = oracle_grads(case, idx)
    for names in (("phase",), ("probe", "pos"), ("tilt", "dz"), ("amp", "dz")):
        pt, params, I_meas = _gpu(case, names)
        grads = params.zeros_like()
        for t in (grads.amp, grads.phase, grads.pos, grads.tilt, grads.dz):
            t.fill_(3.0)
        grads.probe.fill_(3.0)
        loss, grads = pt.loss_grad(params, idx, I_meas, grads=grads)
        torch.cuda.synchronize()
        assert pt.status() == 0, names
        for name in ("amp", "phase", "probe", "pos", "tilt", "dz"):
            got = _np(getattr(grads, name))
            if name in names:
                exp = getattr(ref, name)
                assert rel_l2(got[0] if name == "dz" else got, exp) <= TOL_G, (names, name)
            else:
                assert np.all(got == 3.0), (names, name)


def test_deterministic_intensities_and_loss():
    case = make_case(N=64, M=3, Nz=3, scan=(3, 3), seed=9)
    pt, params, I_meas = _gpu(case)
    idx = list(range(9))
    I1 = pt.forward(params, idx).clone()
    I2 = pt.forward(params, idx).clone()
    assert torch.equal(I1, I2)
    l1 = pt.loss_grad(params, idx, I_meas)[0].item()
    l2 = pt.loss_grad(params, idx, I_meas)[0].item()
    assert l1 == l2


def test_batch_index_outside_scan_is_flagged():
    case = make_case(N=64, M=1, Nz=1, scan=(2, 2), seed=10)
    pt, params, I_meas = _gpu(case)
    pt.loss_grad(params, [0, case.Ntot], I_meas)
    assert pt.status() & 2
    pt.loss_grad(params, [0, -1], I_meas)
    assert pt.status() & 2
    pt.loss_grad(params, [0, 1], I_meas)
    assert pt.status() == 0
