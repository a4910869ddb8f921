"""FP64 CPU oracle for mixed-state multislice ptychography: forward model, loss, adjoint.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only the
tests, the smoke check and the CPU-baseline leg of the throughput script call it.
It shares no code with the CUDA path.

It evaluates, in complex128 and one scan position / one probe mode at a time,
exactly what the paper's forward model defines (PtyRAD, arXiv 2505.07814):

* Eq. 1  I_j = f(P, O, rho_j, theta_j, dz)                         -> `model_patterns`
* Eq. 2  incoherent sum over probe modes of |F[psi_j^(m)]|^2       -> `model_patterns`
* Sec. "Physical model": integer crop of the object patch at
  round(rho_j) and the sub-pixel shift operator S_dr acting on the
  probe, dr = rho_j - round(rho_j)                                    -> `crop_index`, `shift_operator`
* Eq. 3  multislice exit wave, propagator between slices           -> `exit_wave`
* Eq. 4  adaptive Fresnel propagator with local tilt               -> `propagator`
* Eq. 5, 6  Gaussian / Poisson negative log-likelihood losses      -> `loss_value`, `loss_grad_I`
* the PACBED and sparsity terms of the weighted total loss
  (Sec. "Loss functions", Eq. 7-9)                                 -> `pacbed_*`, `sparse_*`
* the derivative of the loss with respect to all six parameters
  (object amplitude and phase, probe, positions, tilts, dz),
  written out by hand as the adjoint of each step                  -> `loss_and_grad`

Readings where the paper is silent (each also listed in the design notes):
  R1  the shift operator moves the probe (Fig. 1 caption), ramp exp(-2 pi i k.dr);
  R2  Nz - 1 propagations: none after the last slice (Eq. 3);
  R3  propagation uses the unnormalised DFT F with F^-1 = (1/N^2) conj-DFT; the far field uses the
      orthonormal DFT; patterns are stored DC-centred (fftshift);
  R4  round() is half-to-even; rho is the patch's top-left corner; a patch outside the object is an
      error, never a wrap;
  R5  Eq. 4 is used as printed: no band-limit mask; theta in radian through tan();
  R6  <.>_{D,B} is the mean over detector pixels and batch; the denominator <I_meas^p> is a constant
      of the batch; eps = 1e-6 sits inside the log, added to I_model^p;
  R7  where I_model = 0 and p < 1, dI^p/dI is taken as 0;
  R8  complex gradients follow dL/dRe + i dL/dIm; amp/phase gradients are real;
  R9  K object modes (Eq. 2): the pattern sums |F[psi]|^2 over every (probe mode, object mode)
      pair, with no weights between the object modes; the paper's reconstructions use K = 1;
  R10 total loss = (Eq. 5 or 6) + w_pacbed L_PACBED + w_sparse L_sparse (the weights of Eq. 9 with
      the chosen likelihood at weight 1); L_PACBED raises the batch-mean patterns to p_pacbed
      (default 0.5) and normalises by <I_meas^p_pacbed>_{D,B}; L_sparse averages |phase|^p_sparse
      (default 1) over every slice of every batch position's N x N patch (a pixel reached by two
      positions counts twice); sign(0) = 0 and |x|^(p - 1) = 0 at x = 0 for p < 1;
  R11 a batch split into parts (data-parallel ranks, accumulated sub-batches): a part's gradient is
      the adjoint, over that part's patterns only, of dL/dI of the whole batch's loss; a part's
      loss is its share of the whole batch's loss: the Poisson sum over its pixels divided by the
      whole batch's sum of I_meas^p, or for Gaussian the whole loss times the part's fraction of
      the whole batch's squared residuals.  The shares add up to the loss and the parts' gradients
      to the whole batch's gradient.

Array conventions: row-major, axis 0 = rows, axis 1 = columns; k_a = fftfreq(N, dx) in 1/angstrom;
positions and tilts are (axis-0, axis-1) pairs; the probe is [M][N][N]; the object amplitude and
phase are [Nz][H][W] (one object mode) or [K][Nz][H][W]; measured patterns are [Ntot][N][N],
DC-centred.
"""
from __future__ import annotations

import dataclasses

import numpy as np

POISSON = "poisson"
GAUSSIAN = "gaussian"


@dataclasses.dataclass
class Geometry:
    N: int
    M: int
    Nz: int
    H: int
    W: int
    dx: float  # angstrom per pixel
    lam: float  # electron wavelength, angstrom
    loss: str = POISSON
    p: float | None = None  # exponent on the patterns; default 1 (Poisson) / 0.5 (Gaussian)
    eps: float = 1e-6
    global_tilt: bool = False  # one tilt for all positions instead of one per position
    w_pacbed: float = 0.0  # weight of the PACBED term (reading R10)
    p_pacbed: float | None = None  # its exponent, default 0.5
    w_sparse: float = 0.0  # weight of the phase sparsity term
    p_sparse: float | None = None  # its exponent, default 1
    K: int = 1  # object modes (reading R9)

    @property
    def power(self) -> float:
        if self.p is not None:
            return float(self.p)
        return 1.0 if self.loss == POISSON else 0.5


# ----------------------------------------------------------------------------------------------
# Fourier transforms (numpy's pocketfft, forward sign -2 pi i)
# ----------------------------------------------------------------------------------------------

def dft2(x):
    """Unnormalised forward DFT: sum_r x(r) exp(-2 pi i k.r / N)."""
    return np.fft.fft2(x)


def idft2(x):
    """Inverse of dft2 (carries 1/N^2)."""
    return np.fft.ifft2(x)


def far_field(psi):
    """Orthonormal DFT, so that sum |F psi|^2 = sum |psi|^2 (reading R3)."""
    return np.fft.fft2(psi, norm="ortho")


def freqs(N, dx):
    """(k0, k1) grids of spatial frequency in 1/angstrom, unshifted DFT order."""
    k = np.fft.fftfreq(N, d=dx)
    return np.meshgrid(k, k, indexing="ij")


# ----------------------------------------------------------------------------------------------
# Forward model steps
# ----------------------------------------------------------------------------------------------

def crop_index(rho):
    """Integer patch corner round(rho) and the sub-pixel remainder dr = rho - round(rho)."""
    rho = np.asarray(rho, dtype=np.float64)
    r = np.round(rho)  # half-to-even
    return r.astype(np.int64), rho - r


def shift_ramp(N, dr):
    """exp(-2 pi i (f0 dr0 + f1 dr1)) with f in cycles per pixel: translates by +dr pixels."""
    f = np.fft.fftfreq(N)
    f0, f1 = np.meshgrid(f, f, indexing="ij")
    return np.exp(-2j * np.pi * (f0 * dr[0] + f1 * dr[1]))


def shift_operator(P, dr):
    """S_dr P = F^-1[F[P] . ramp(dr)]  (Sec. "Physical model", sub-pixel shift of the probe)."""
    return idft2(dft2(P) * shift_ramp(P.shape[-1], dr))


def propagator(N, dx, lam, dz, theta):
    """Eq. 4: M(k) = exp[-i pi lam |k|^2 dz + 2 pi i dz (k0 tan th0 + k1 tan th1)]."""
    k0, k1 = freqs(N, dx)
    return np.exp(-1j * np.pi * lam * (k0 ** 2 + k1 ** 2) * dz
                  + 2j * np.pi * dz * (k0 * np.tan(theta[0]) + k1 * np.tan(theta[1])))


def transmission(amp, phase):
    """Object function from its two real parameter arrays: amp . exp(i phase)."""
    return amp * np.exp(1j * phase)


def object_patch(T, r, N):
    """O_j: the N x N window of every slice whose top-left corner is r (reading R4)."""
    Nz, H, W = T.shape
    if r[0] < 0 or r[1] < 0 or r[0] + N > H or r[1] + N > W:
        raise IndexError("object patch at %s lies outside the %dx%d object" % (tuple(r), H, W))
    return T[:, r[0]:r[0] + N, r[1]:r[1] + N]


def exit_wave(Pj, Oj, Mj):
    """Eq. 3: psi = O_Nz . F^-1[M F[ ... F^-1[M F[O_1 Pj]] ... ]], propagation between slices only."""
    psi = Oj[0] * Pj
    for s in range(1, Oj.shape[0]):
        psi = Oj[s] * idft2(Mj * dft2(psi))
    return psi


def tilt_of(geom, tilt, j):
    return np.asarray(tilt if geom.global_tilt else tilt[j], dtype=np.float64).reshape(2)


def object_modes(geom, x):
    """The object array as [K][Nz][H][W] (a single mode may be passed as [Nz][H][W])."""
    x = np.asarray(x)
    return x.reshape((geom.K, geom.Nz) + x.shape[-2:])


def model_patterns(geom, amp, phase, probe, pos, tilt, dz, idx):
    """Eq. 1-2 for the scan positions idx: I_j = fftshift(sum_m sum_n |F_ortho[psi_j^(m)(n)]|^2),
    [B][N][N] (probe modes m, object modes n)."""
    N = geom.N
    T = transmission(object_modes(geom, amp), object_modes(geom, phase))
    out = np.zeros((len(idx), N, N))
    for b, j in enumerate(idx):
        r, dr = crop_index(pos[j])
        Mj = propagator(N, geom.dx, geom.lam, dz, tilt_of(geom, tilt, j))
        I = np.zeros((N, N))
        for m in range(geom.M):
            Pj = shift_operator(probe[m], dr)
            for n in range(geom.K):
                I += np.abs(far_field(exit_wave(Pj, object_patch(T[n], r, N), Mj))) ** 2
        out[b] = np.fft.fftshift(I)
    return out


# ----------------------------------------------------------------------------------------------
# Loss (Eq. 5, 6) and its derivative with respect to the modelled intensity
# ----------------------------------------------------------------------------------------------

def _pow(I, p):
    return I if p == 1.0 else np.power(np.maximum(I, 0.0), p)


def _dpow(I, p):
    """d(I^p)/dI, 0 where I = 0 and p < 1 (reading R7)."""
    if p == 1.0:
        return np.ones_like(I)
    out = np.zeros_like(I)
    nz = I > 0
    out[nz] = p * np.power(I[nz], p - 1.0)
    return out


def loss_value(geom, I_model, I_meas):
    """L over one batch; I arrays [B][N][N].  Means over detector and batch (reading R6)."""
    p = geom.power
    Im, Id = _pow(I_model, p), _pow(I_meas, p)
    if geom.loss == GAUSSIAN:  # Eq. 5
        return np.sqrt(np.mean((Im - Id) ** 2)) / np.mean(Id)
    if geom.loss == POISSON:  # Eq. 6
        return -np.mean(Id * np.log(Im + geom.eps) - Im) / np.mean(Id)
    raise ValueError(geom.loss)


def loss_grad_I(geom, I_model, I_meas):
    """dL/dI_model, same shape as I_model."""
    p = geom.power
    Im, Id = _pow(I_model, p), _pow(I_meas, p)
    D = I_model.size
    dp = _dpow(I_model, p)
    if geom.loss == GAUSSIAN:
        mse = np.mean((Im - Id) ** 2)
        if mse == 0.0:
            return np.zeros_like(I_model)
        # d/dIm sqrt(mean((Im-Id)^2)) = (Im-Id) / (D sqrt(mse))
        return (Im - Id) / (D * np.sqrt(mse)) / np.mean(Id) * dp
    if geom.loss == POISSON:
        return -(Id / (Im + geom.eps) - 1.0) / D / np.mean(Id) * dp
    raise ValueError(geom.loss)


def loss_share(geom, I_model, I_meas, a, b):
    """The share of patterns a..b-1 in the loss of the whole batch I_model (reading R11)."""
    p = geom.power
    Im, Id = _pow(I_model, p), _pow(I_meas, p)
    if geom.loss == GAUSSIAN:
        r2 = (Im - Id) ** 2
        total = np.sum(r2)
        return 0.0 if total == 0.0 else loss_value(geom, I_model, I_meas) * np.sum(r2[a:b]) / total
    if geom.loss == POISSON:
        return -np.sum(Id[a:b] * np.log(Im[a:b] + geom.eps) - Im[a:b]) / np.sum(Id)
    raise ValueError(geom.loss)


def pacbed_value(geom, I_model, I_meas):
    """L_PACBED: the batch-mean patterns (position-averaged CBED) compared like Eq. 5."""
    p = 0.5 if geom.p_pacbed is None else float(geom.p_pacbed)
    d = _pow(I_model.mean(axis=0), p) - _pow(I_meas.mean(axis=0), p)
    return np.sqrt(np.mean(d ** 2)) / np.mean(_pow(I_meas, p))


def pacbed_grad_I(geom, I_model, I_meas):
    """dL_PACBED / dI_model: the same for every pattern of the batch (each enters the mean 1/B)."""
    p = 0.5 if geom.p_pacbed is None else float(geom.p_pacbed)
    B = I_model.shape[0]
    A = I_model.mean(axis=0)
    d = _pow(A, p) - _pow(I_meas.mean(axis=0), p)
    ms = np.mean(d ** 2)
    if ms == 0.0:
        return np.zeros_like(I_model)
    g = d / (d.size * np.sqrt(ms)) / np.mean(_pow(I_meas, p)) * _dpow(A, p) / B
    return np.broadcast_to(g, I_model.shape).copy()


def _patches(phase, corners, N):
    """Every position's N x N window of every slice (of every object mode, when phase is 4D)."""
    ph = np.asarray(phase, dtype=np.float64)
    return [ph[..., r0:r0 + N, r1:r1 + N] for r0, r1 in corners]


def sparse_value(geom, phase, corners):
    """L_sparse = <|phase|^p>^(1/p) over the batch's patches (reading R10)."""
    p = 1.0 if geom.p_sparse is None else float(geom.p_sparse)
    v = np.concatenate([np.abs(x).ravel() for x in _patches(phase, corners, geom.N)])
    return float(np.mean(v ** p) ** (1.0 / p))


def sparse_grad_phase(geom, phase, corners):
    p = 1.0 if geom.p_sparse is None else float(geom.p_sparse)
    N = geom.N
    pats = _patches(phase, corners, N)
    n = sum(x.size for x in pats)
    S = sum(float(np.sum(np.abs(x) ** p)) for x in pats)
    g = np.zeros(np.shape(phase))
    if S == 0.0:
        return g
    scale = (S / n) ** (1.0 / p - 1.0) / n
    for (r0, r1), x in zip(corners, pats):
        a = np.abs(x)
        w = np.zeros_like(a)
        nz = a > 0
        w[nz] = a[nz] ** (p - 1.0)
        g[..., r0:r0 + N, r1:r1 + N] += scale * w * np.sign(x)
    return g


# ----------------------------------------------------------------------------------------------
# Loss and gradients of all six parameters (hand-written adjoint of every step above)
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Gradients:
    loss: float
    I_model: np.ndarray  # [B][N][N] DC-centred
    amp: np.ndarray  # shape of the amp argument
    phase: np.ndarray  # shape of the phase argument
    probe: np.ndarray  # [M][N][N] complex, dL/dRe + i dL/dIm
    pos: np.ndarray  # [Ntot][2]
    tilt: np.ndarray  # [Ntot][2] (or [2] with global tilt)
    dz: float


def loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx, part=None):
    """Loss of the batch idx and the exact gradient of every parameter.

    I_meas is indexed by scan position ([Ntot][N][N], DC-centred).  Gradient arrays cover the
    whole parameter (zeros where the batch does not reach).  part = (a, b): the loss share and
    the gradient of patterns idx[a:b] only, within the whole batch idx (reading R11); the PACBED
    and sparsity terms are not split.
    """
    if part is not None and (geom.w_pacbed or geom.w_sparse):
        raise ValueError("the PACBED and sparsity terms are not split into parts")
    N, M, Nz, K = geom.N, geom.M, geom.Nz, geom.K
    idx = list(idx)
    B = len(idx)
    amp_shape = np.shape(amp)
    amp, phase = object_modes(geom, amp), object_modes(geom, phase)
    T = transmission(amp, phase)  # [K][Nz][H][W]
    k0, k1 = freqs(N, geom.dx)
    f = np.fft.fftfreq(N)
    f0, f1 = np.meshgrid(f, f, indexing="ij")

    # ---------------- forward, keeping what the adjoint needs ----------------
    Phat = np.stack([dft2(probe[m]) for m in range(M)])
    records = []
    I_model = np.zeros((B, N, N))
    for b, j in enumerate(idx):
        r, dr = crop_index(pos[j])
        th = tilt_of(geom, tilt, j)
        Mj = propagator(N, geom.dx, geom.lam, dz, th)
        R = shift_ramp(N, dr)
        per_mode = []  # [(m, n)] for probe mode m, object mode n
        I = np.zeros((N, N))
        for m in range(M):
            for n in range(K):
                Oj = object_patch(T[n], r, N)
                psi = idft2(Phat[m] * R)  # shifted probe P_j
                psi_in, vhat = [], []
                for s in range(Nz):
                    psi_in.append(psi)
                    u = Oj[s] * psi
                    if s < Nz - 1:
                        vhat.append(Mj * dft2(u))
                        psi = idft2(vhat[-1])
                    else:
                        psi = u
                Psi = far_field(psi)
                I += np.abs(Psi) ** 2
                per_mode.append((m, n, psi_in, vhat, Psi))
        I_model[b] = np.fft.fftshift(I)
        records.append((j, r, dr, th, Mj, R, per_mode))

    Imeas_b = np.stack([np.asarray(I_meas[j], dtype=np.float64) for j in idx])
    loss = loss_value(geom, I_model, Imeas_b)
    dLdI = loss_grad_I(geom, I_model, Imeas_b)
    if geom.w_pacbed:
        loss += geom.w_pacbed * pacbed_value(geom, I_model, Imeas_b)
        dLdI = dLdI + geom.w_pacbed * pacbed_grad_I(geom, I_model, Imeas_b)
    lo, hi = (0, B) if part is None else part
    if part is not None:
        loss = loss_share(geom, I_model, Imeas_b, lo, hi)

    # ---------------- adjoint ----------------
    gT = np.zeros_like(T)
    g_probe_hat = np.zeros((M, N, N), dtype=np.complex128)
    g_pos = np.zeros_like(np.asarray(pos, dtype=np.float64))
    g_tilt = np.zeros_like(np.asarray(tilt, dtype=np.float64))
    g_dz = 0.0
    for b, (j, r, dr, th, Mj, R, per_mode) in enumerate(records):
        if not lo <= b < hi:
            continue
        w = np.fft.ifftshift(dLdI[b])  # back to DFT order
        # dM/d(dz) / M and dM/d(theta_a) / M
        c_dz = 1j * (-np.pi * geom.lam * (k0 ** 2 + k1 ** 2)
                     + 2 * np.pi * (k0 * np.tan(th[0]) + k1 * np.tan(th[1])))
        c_t0 = 2j * np.pi * dz * k0 / np.cos(th[0]) ** 2
        c_t1 = 2j * np.pi * dz * k1 / np.cos(th[1]) ** 2
        gth = np.zeros(2)
        for m, n, psi_in, vhat, Psi in per_mode:
            Oj = object_patch(T[n], r, N)
            # I = |Psi|^2 -> g_Psi = 2 dL/dI Psi ; Psi = F_ortho psi -> g_psi = F_ortho^H g_Psi
            g = np.fft.ifft2(2.0 * w * Psi, norm="ortho")
            for s in range(Nz - 1, -1, -1):
                # u_s = O_s psi_in_s
                gT[n, s, r[0]:r[0] + N, r[1]:r[1] + N] += np.conj(psi_in[s]) * g
                g = np.conj(Oj[s]) * g
                if s > 0:
                    # psi_in_s = F^-1[vhat], F^-1 = (1/N^2) F^H  ->  g_vhat = F[g] / N^2
                    g_v = dft2(g) / N ** 2
                    v = vhat[s - 1]
                    g_dz += np.real(np.sum(np.conj(g_v) * c_dz * v))
                    gth[0] += np.real(np.sum(np.conj(g_v) * c_t0 * v))
                    gth[1] += np.real(np.sum(np.conj(g_v) * c_t1 * v))
                    # vhat = M F[u_{s-1}]  ->  g_u = F^H [conj(M) g_v] = N^2 F^-1[conj(M) g_v]
                    g = N ** 2 * idft2(np.conj(Mj) * g_v)
            # g is now dL/dP_j ; P_j = F^-1[Phat R]
            g_PR = dft2(g) / N ** 2
            g_probe_hat[m] += np.conj(R) * g_PR
            PR = Phat[m] * R
            g_pos[j, 0] += np.real(np.sum(np.conj(g_PR) * (-2j * np.pi * f0) * PR))
            g_pos[j, 1] += np.real(np.sum(np.conj(g_PR) * (-2j * np.pi * f1) * PR))
        if geom.global_tilt:
            g_tilt += gth
        else:
            g_tilt[j] += gth

    # Phat = F[P] -> g_P = F^H g_Phat = N^2 F^-1[g_Phat]
    g_probe = np.stack([N ** 2 * idft2(g_probe_hat[m]) for m in range(M)])
    # T = amp e^{i phase}:  dL/damp = Re(conj(e^{i phase}) gT),  dL/dphase = Re(conj(i T) gT)
    g_amp = np.real(np.conj(np.exp(1j * phase)) * gT)
    g_phase = np.real(np.conj(1j * T) * gT)
    if geom.w_sparse:
        corners = [tuple(crop_index(pos[j])[0]) for j in idx]
        loss += geom.w_sparse * sparse_value(geom, phase, corners)
        g_phase = g_phase + geom.w_sparse * sparse_grad_phase(geom, phase, corners)
    g_amp, g_phase = g_amp.reshape(amp_shape), g_phase.reshape(amp_shape)
    return Gradients(loss=float(loss), I_model=I_model, amp=g_amp, phase=g_phase, probe=g_probe,
                     pos=g_pos, tilt=g_tilt, dz=float(g_dz))
