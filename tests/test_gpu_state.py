"""Resume of a reconstruction from a checkpoint file: three Adam iterations (pty_step), a save, a
reload into a fresh problem on the device, three more iterations give the same loss trajectory and
parameters as six iterations run straight through.  The object and probe gradients are summed
with float atomics, so two runs differ in their last bits; losses are compared to 1e-6 and the
parameter arrays to 1e-5 in relative L2."""
import numpy as np
import pytest

from tests.cases import make_case, rel_l2
from tests.test_gpu_parity import _gpu, _np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ("amp", "phase", "probe", "pos", "tilt", "dz")
LR = {"amp": 1e-4, "phase": 2e-4, "probe": 1e-2, "pos": 1e-3, "tilt": 1e-6, "dz": 1e-3}


def _run(pt, params, adam, I_meas, batches):
    from paper_2505_07814_gb300.ptycho import step
    grads = params.zeros_like()
    losses = []
    for idx in batches:
        losses.append(step(pt, params, grads, adam, idx, I_meas).item())
    torch.cuda.synchronize()
    assert pt.status() == 0
    return losses


def test_resume_continues_the_trajectory(tmp_path):
    from paper_2505_07814_gb300 import state
    from paper_2505_07814_gb300.ptycho import Adam, Ptycho
    case = make_case(N=64, M=2, Nz=3, scan=(2, 3), seed=41)
    batches = [[0, 1, 2], [3, 4, 5], [5, 2, 0], [1, 4, 3], [0, 5, 2], [4, 1, 3]]
    # straight through
    pt, params, I_meas = _gpu(case)
    adam = Adam(params, LR)
    straight = _run(pt, params, adam, I_meas, batches)
    final = {n: _np(getattr(params, n)).copy() for n in NAMES}
    # three iterations, save, reload into a new problem, three more
    pt2, params2, _ = _gpu(case)
    adam2 = Adam(params2, LR)
    first = _run(pt2, params2, adam2, I_meas, batches[:3])
    path = str(tmp_path / "rec.pt")
    state.save(path, pt2.geom, params2, adam2, iteration=3)
    del pt2, params2, adam2
    geom3, params3, adam3, it, _ = state.load(path, device="cuda")
    assert it == 3 and adam3.t == 3
    pt3 = Ptycho(geom3, case.Ntot, device="cuda")
    second = _run(pt3, params3, adam3, I_meas, batches[3:])
    resumed = first + second
    np.testing.assert_allclose(resumed, straight, rtol=1e-6)
    for n in NAMES:
        assert rel_l2(_np(getattr(params3, n)), final[n]) <= 1e-5, n
    assert adam3.t == 6
