"""pty_constrain (relaxed depth blur and phase positivity) against the constraint oracle."""
import numpy as np
import pytest

from oracle import constraints as K

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(Nz, H, W, seed=0):
    from paper_2505_07814_gb300.ptycho import Geometry, Params, Ptycho
    rng = np.random.default_rng(seed)
    amp = (1.0 + 0.1 * rng.standard_normal((Nz, H, W))).astype(np.float32)
    phase = (0.3 * rng.standard_normal((Nz, H, W))).astype(np.float32)
    geom = Geometry(N=64, M=1, Nz=Nz, H=H, W=W, Ntot=1, dx=0.1, lam=0.025, grads=("amp", "phase"))
    f = dict(dtype=torch.float32, device="cuda")
    params = Params(amp=torch.tensor(amp, **f), phase=torch.tensor(phase, **f),
                    probe=torch.zeros((1, 64, 64), dtype=torch.complex64, device="cuda"),
                    pos=torch.zeros((1, 2), **f), tilt=torch.zeros((1, 2), **f), dz=torch.ones(1, **f))
    return Ptycho(geom, 1), params, amp.astype(np.float64), phase.astype(np.float64)


# 70 x 90 takes the float4 path over 12 full tiles and a ragged one; 71 x 90 (plane not a multiple
# of 4) the scalar path; Nz = 128 the largest depth, with more than 48 KB of shared memory per CTA.
@pytest.mark.parametrize("Nz,H,W,pos,sigma,relax", [(7, 70, 90, 1.0, 1.3, 0.6), (20, 70, 90, 0.5, 2.0, 1.0),
                                                   (8, 70, 90, 1.0, 0.0, 1.0), (1, 70, 90, 1.0, 1.0, 1.0),
                                                   (5, 70, 90, 0.0, 0.7, 0.3), (6, 71, 90, 1.0, 1.1, 0.8),
                                                   (3, 71, 90, 0.7, 0.0, 1.0), (128, 70, 90, 1.0, 3.0, 1.0),
                                                   (40, 65, 66, 0.0, 30.0, 1.0)])
def test_constrain_matches_oracle(Nz, H, W, pos, sigma, relax):
    from paper_2505_07814_gb300.ptycho import constrain
    pt, params, amp, phase = _setup(Nz, H, W)
    constrain(pt, params, phase_positivity=pos, rz_sigma=sigma, rz_relax=relax)
    torch.cuda.synchronize()
    ra, rp = K.constrain(amp, phase, pos, sigma, relax)
    np.testing.assert_allclose(params.amp.cpu().numpy(), ra, rtol=2e-6, atol=2e-7)
    np.testing.assert_allclose(params.phase.cpu().numpy(), rp, rtol=2e-6, atol=2e-7)
    if pos == 1.0:
        assert float(params.phase.min()) >= 0.0


def test_constrain_rejects_bad_arguments():
    from paper_2505_07814_gb300 import _lib
    from paper_2505_07814_gb300.ptycho import constrain
    pt, params, _, _ = _setup(3, 64, 64)
    for kw in (dict(phase_positivity=1.5), dict(rz_relax=-0.1), dict(rz_sigma=float("nan"))):
        with pytest.raises(_lib.PtyError):
            constrain(pt, params, **kw)
    pt2, params2, _, _ = _setup(129, 64, 64)
    with pytest.raises(_lib.PtyError):
        constrain(pt2, params2, rz_sigma=1.0)
    constrain(pt2, params2, phase_positivity=1.0)  # the clip alone has no slice limit
