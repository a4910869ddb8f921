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


def _with_dz(params, dz):
    params.dz.fill_(dz)
    return params


# 64 x 64 takes the radix-2 line transforms; 70 and 96 (not powers of two) the direct DFT; 512 x 512
# the object of the multislice workload.
@pytest.mark.parametrize("Nz,H,W,beta,alpha,relax", [(8, 64, 64, 1.0, 0.01, 1.0), (5, 70, 96, 0.5, 0.0, 0.7),
                                                    (3, 128, 80, 2.0, 0.05, 1.0), (1, 64, 72, 1.0, 0.02, 1.0),
                                                    (8, 512, 512, 1.0, 0.01, 1.0)])
def test_kz_filter_matches_oracle(Nz, H, W, beta, alpha, relax):
    from paper_2505_07814_gb300.ptycho import constrain
    pt, params, amp, phase = _setup(Nz, H, W, seed=Nz + H)
    dz = 2.0
    _with_dz(params, dz)
    constrain(pt, params, kz_beta=beta, kz_alpha=alpha, kz_relax=relax)
    torch.cuda.synchronize()
    dx = pt.geom.dx
    ra = K.kz_filter(amp, dx, dz, beta, alpha, relax)
    rp = K.kz_filter(phase, dx, dz, beta, alpha, relax)
    for got, ref in ((params.amp, ra), (params.phase, rp)):
        g = got.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(g - ref) <= 2e-6 * np.linalg.norm(ref), np.linalg.norm(g - ref) / np.linalg.norm(ref)
        assert np.abs(g - ref).max() <= 2e-5


def test_all_object_constraints_in_order():
    from paper_2505_07814_gb300.ptycho import constrain
    pt, params, amp, phase = _setup(6, 64, 70, seed=11)
    _with_dz(params, 1.5)
    constrain(pt, params, phase_positivity=1.0, rz_sigma=1.0, rz_relax=0.8, kz_beta=1.0, kz_alpha=0.02,
              kz_relax=0.9)
    torch.cuda.synchronize()
    ra, rp = K.constrain(amp, phase, 1.0, 1.0, 0.8, kz_beta=1.0, kz_alpha=0.02, kz_relax=0.9, dx=pt.geom.dx, dz=1.5)
    np.testing.assert_allclose(params.amp.cpu().numpy(), ra, rtol=1e-5, atol=2e-5)
    np.testing.assert_allclose(params.phase.cpu().numpy(), rp, rtol=1e-5, atol=2e-5)
    assert float(params.phase.min()) >= 0.0


def _probe_setup(M, N, seed, mix=True):
    from paper_2505_07814_gb300.ptycho import Geometry, Params, Ptycho
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((M, N, N)) + 1j * rng.standard_normal((M, N, N))
    if mix:  # modes of unequal power
        P *= (0.7 ** np.arange(M))[:, None, None]
    P = P.astype(np.complex64)
    geom = Geometry(N=N, M=M, Nz=1, H=N, W=N, Ntot=1, dx=0.1, lam=0.025)
    f = dict(dtype=torch.float32, device="cuda")
    params = Params(amp=torch.ones((1, N, N), **f), phase=torch.zeros((1, N, N), **f),
                    probe=torch.tensor(P, device="cuda"), pos=torch.zeros((1, 2), **f), tilt=torch.zeros((1, 2), **f),
                    dz=torch.ones(1, **f))
    return Ptycho(geom, 1), params, P.astype(np.complex128)


@pytest.mark.parametrize("M,N", [(6, 64), (12, 128), (32, 64), (3, 256), (1, 64)])
def test_orthogonalize_probe_matches_oracle(M, N):
    from paper_2505_07814_gb300.ptycho import constrain
    pt, params, P = _probe_setup(M, N, seed=M * N)
    constrain(pt, params, orthogonalize_probe=True)
    torch.cuda.synchronize()
    Q = params.probe.cpu().numpy().astype(np.complex128)
    R, lam = K.orthogonalize_probe(P)
    np.testing.assert_allclose(np.sum(np.abs(Q) ** 2, axis=(1, 2)), lam, rtol=1e-5)
    for k in range(M):
        assert np.linalg.norm(Q[k] - R[k]) <= 1e-5 * np.linalg.norm(R[k]), k
    # the amplitude and phase are untouched
    assert float(params.amp.min()) == 1.0 and float(params.phase.abs().max()) == 0.0


def test_orthogonalize_degenerate_powers():
    """Equal powers: the eigenvectors are not unique; the result must still be orthogonal, keep the
    density matrix and the powers."""
    from paper_2505_07814_gb300.ptycho import constrain
    pt, params, P = _probe_setup(4, 64, seed=5, mix=False)
    A = P.reshape(4, -1)
    Qr, _ = np.linalg.qr(A.T)  # orthonormal modes of equal power
    P2 = (Qr.T * 3.0).reshape(P.shape).astype(np.complex64)
    params.probe.copy_(torch.tensor(P2, device="cuda"))
    constrain(pt, params, orthogonalize_probe=True)
    torch.cuda.synchronize()
    B = params.probe.cpu().numpy().astype(np.complex128).reshape(4, -1)
    A2 = P2.astype(np.complex128).reshape(4, -1)
    np.testing.assert_allclose(B @ B.conj().T, 9.0 * np.eye(4), atol=1e-4)
    np.testing.assert_allclose(B.conj().T @ B, A2.conj().T @ A2, atol=1e-5)


def test_constrain_rejects_unsupported_sizes():
    from paper_2505_07814_gb300 import _lib
    from paper_2505_07814_gb300.ptycho import constrain
    pt, params, _ = _probe_setup(33, 64, seed=1)
    with pytest.raises(_lib.PtyError):
        constrain(pt, params, orthogonalize_probe=True)
    pt, params, _, _ = _setup(1, 64, 8200)
    with pytest.raises(_lib.PtyError):
        constrain(pt, params, kz_beta=1.0, kz_relax=1.0)
    for kw in (dict(kz_beta=-1.0, kz_relax=1.0), dict(kz_beta=1.0, kz_relax=1.5), dict(kz_alpha=float("inf"))):
        with pytest.raises(_lib.PtyError):
            constrain(pt, params, **kw)
