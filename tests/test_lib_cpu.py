"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a, loads, exports
every function include/*.h declares, and rejects bad arguments before launching anything."""
import ctypes
import os
import re

import pytest

from paper_2505_07814_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pty_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert set(declared) == set(_lib.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_missing_library_fails_loudly(tmp_path):
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(RuntimeError):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved


def _geom(**kw):
    g = dict(N=64, M=2, Nz=3, H=100, W=110, Ntot=12, dx=0.1, lambda_=0.0251, loss=0, p=0.0, eps=1e-6,
             grad_mask=63, global_tilt=0, ckpt_stride=0, fft_impl=0)
    g.update(kw)
    return _lib.pty_geom(**g)


def test_workspace_size_and_validation(lib):
    n = lib.pty_workspace_size(ctypes.byref(_geom()), 8)
    # at least the checkpoints: B*M*Nz*N^2 complex64
    assert n >= 8 * 2 * 3 * 64 * 64 * 8
    assert lib.pty_workspace_size(ctypes.byref(_geom(grad_mask=_lib.PTY_GRAD_PROBE)), 8) < n
    for bad in (dict(N=32), dict(N=96), dict(N=512), dict(N=256, H=200), dict(M=0), dict(Nz=0), dict(H=63), dict(loss=7), dict(dx=0.0),
                dict(grad_mask=64), dict(ckpt_stride=-1), dict(fft_impl=4), dict(fft_impl=-1),
                dict(N=256, H=300, W=300, fft_impl=1)):
        assert lib.pty_workspace_size(ctypes.byref(_geom(**bad)), 8) == 0, bad
        assert lib.pty_last_error()
    assert lib.pty_supported_sizes() == (1 << 6) | (1 << 7) | (1 << 8)


def test_split_dft_workspace(lib):
    """The split-precision DFT modes keep every slice's checkpoint and add two wave buffers."""
    full = lib.pty_workspace_size(ctypes.byref(_geom(Nz=12, ckpt_stride=1)), 16)
    for impl in (_lib.PTY_FFT_SPLIT_BF16, _lib.PTY_FFT_SPLIT_FP16, _lib.PTY_FFT_SPLIT3_BF16):
        for K in (1, 4):
            n = lib.pty_workspace_size(ctypes.byref(_geom(Nz=12, ckpt_stride=K, fft_impl=impl)), 16)
            wave = 16 * 2 * 64 * 64 * 8  # one complex64 buffer of every wave
            pieces = 3 if impl == _lib.PTY_FFT_SPLIT3_BF16 else 2
            extra = 2 * wave + 2 * wave * pieces // 2  # wave + transposed buffer, two split operands
            assert full + extra <= n <= full + extra + 8192
        assert lib.pty_workspace_size(ctypes.byref(_geom(N=128, H=200, W=200, fft_impl=impl)), 4) > 0


def test_bad_arguments_rejected_before_launch(lib):
    g = _geom()
    fake = ctypes.c_void_p(0x10000)  # never dereferenced: validation fails first
    null = None
    # unsupported N
    rc = lib.pty_forward(ctypes.byref(_geom(N=32)), 1, fake, fake, fake, fake, fake, fake, fake, fake, fake, 1 << 30,
                         null)
    assert rc == _lib.PTY_EINVAL and "N = 32" in lib.pty_last_error().decode()
    # null parameter
    rc = lib.pty_forward(ctypes.byref(g), 1, fake, null, fake, fake, fake, fake, fake, fake, fake, 1 << 30, null)
    assert rc == _lib.PTY_EINVAL
    # workspace too small
    rc = lib.pty_forward(ctypes.byref(g), 4, fake, fake, fake, fake, fake, fake, fake, fake, fake, 1024, null)
    assert rc == _lib.PTY_EWORKSPACE and "workspace" in lib.pty_last_error().decode()
    # negative batch
    rc = lib.pty_loss_grad(ctypes.byref(g), -1, fake, fake, fake, fake, fake, fake, fake, fake, fake, null, fake,
                           fake, fake, fake, fake, fake, 0, fake, 1 << 30, null)
    assert rc == _lib.PTY_EINVAL
    # requested gradient without an output array
    ws = ctypes.c_void_p(0x100000)
    rc = lib.pty_loss_grad(ctypes.byref(g), 2, fake, fake, fake, fake, fake, fake, fake, fake, fake, null, null,
                           fake, fake, fake, fake, fake, 0, ws, 1 << 40, null)
    assert rc == _lib.PTY_EINVAL and "g_amp" in lib.pty_last_error().decode()
    # misaligned probe
    rc = lib.pty_forward(ctypes.byref(g), 1, fake, fake, fake, ctypes.c_void_p(0x10004), fake, fake, fake, fake,
                         ws, 1 << 40, null)
    assert rc == _lib.PTY_EINVAL
    # Adam with a step count of 0
    a = _lib.pty_adam()
    rc = lib.pty_adam_update(ctypes.byref(g), fake, fake, fake, fake, fake, fake, fake, fake, fake, fake, fake, fake,
                             ctypes.byref(a), 0, null)
    assert rc == _lib.PTY_EINVAL


def test_recompute_plan_shrinks_the_workspace(lib):
    """ckpt_stride K > 1 keeps one spectrum per K slices plus one K-slice segment instead of every slice."""
    full = lib.pty_workspace_size(ctypes.byref(_geom(Nz=12, ckpt_stride=1)), 16)
    k3 = lib.pty_workspace_size(ctypes.byref(_geom(Nz=12, ckpt_stride=3)), 16)
    k12 = lib.pty_workspace_size(ctypes.byref(_geom(Nz=12, ckpt_stride=12)), 16)
    wave = 16 * 2 * 64 * 64 * 8
    assert full - k3 >= wave * ((2 * 12 - 1) - (12 // 3 - 1 + 2 * 3 + 1)) - (1 << 16)
    assert k3 < full and k3 < k12  # K = Nz replays everything but needs Nz-slot segment buffers
    # without object, dz or tilt gradients nothing is recorded, whatever the stride
    g = _geom(Nz=12, ckpt_stride=3, grad_mask=_lib.PTY_GRAD_PROBE | _lib.PTY_GRAD_POS)
    g1 = _geom(Nz=12, ckpt_stride=1, grad_mask=_lib.PTY_GRAD_PROBE | _lib.PTY_GRAD_POS)
    assert lib.pty_workspace_size(ctypes.byref(g), 16) == lib.pty_workspace_size(ctypes.byref(g1), 16)


def test_object_modes_scale_the_workspace(lib):
    """Per-wave arrays and the object-sized transmission / gradient grow with the object modes."""
    n1 = lib.pty_workspace_size(ctypes.byref(_geom()), 8)
    n3 = lib.pty_workspace_size(ctypes.byref(_geom(obj_modes=3)), 8)
    assert n3 > 2.5 * n1
    assert lib.pty_workspace_size(ctypes.byref(_geom(obj_modes=0)), 8) == n1  # 0 means one mode
    for bad in (-1, 65):
        assert lib.pty_workspace_size(ctypes.byref(_geom(obj_modes=bad)), 8) == 0
        assert b"obj_modes" in lib.pty_last_error()


def _constraints(**kw):
    c = _lib.pty_constraints()
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def test_constrain_workspace_size(lib):
    g = _geom(Nz=3, H=100, W=70, M=5)
    assert lib.pty_constrain_workspace_size(ctypes.byref(g), ctypes.byref(_constraints(rz_sigma=1.0, rz_relax=1.0))) == 0
    kz = lib.pty_constrain_workspace_size(ctypes.byref(g), ctypes.byref(_constraints(kz_beta=1.0, kz_relax=1.0)))
    assert kz == (8 * 3 * 100 * 70 + 255) // 256 * 256  # one complex volume
    # beta = alpha = 0 or relaxation 0: the filter is the identity and is skipped
    assert lib.pty_constrain_workspace_size(ctypes.byref(g), ctypes.byref(_constraints(kz_relax=1.0))) == 0
    assert lib.pty_constrain_workspace_size(ctypes.byref(g), ctypes.byref(_constraints(kz_beta=1.0))) == 0
    ortho = lib.pty_constrain_workspace_size(ctypes.byref(g), ctypes.byref(_constraints(probe_orthogonalize=1)))
    assert 0 < ortho < 64 * 1024
    assert lib.pty_constrain_workspace_size(ctypes.byref(_geom(M=1)), ctypes.byref(_constraints(probe_orthogonalize=1))) == 0


def test_constrain_rejects_bad_arguments_before_launch(lib):
    buf = (ctypes.c_float * 16)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    cases = [
        (_geom(), _constraints(phase_positivity=1.5)),
        (_geom(), _constraints(rz_sigma=1.0, rz_relax=-0.1)),
        (_geom(), _constraints(rz_sigma=float("nan"), rz_relax=1.0)),
        (_geom(), _constraints(kz_beta=-1.0, kz_relax=1.0)),
        (_geom(), _constraints(kz_beta=1.0, kz_relax=2.0)),
        (_geom(Nz=129), _constraints(rz_sigma=1.0, rz_relax=1.0)),
        (_geom(W=8200), _constraints(kz_beta=1.0, kz_relax=1.0)),
        (_geom(M=33), _constraints(probe_orthogonalize=1)),
    ]
    for g, c in cases:
        assert lib.pty_constrain(ctypes.byref(g), p, p, p, p, ctypes.byref(c), None, 0, None) == _lib.PTY_EINVAL
        assert lib.pty_last_error()
    # the k_z filter needs dz and a workspace; orthogonalisation needs the probe
    g = _geom()
    c = _constraints(kz_beta=1.0, kz_relax=1.0)
    assert lib.pty_constrain(ctypes.byref(g), p, p, p, None, ctypes.byref(c), None, 0, None) == _lib.PTY_EINVAL
    assert lib.pty_constrain(ctypes.byref(g), p, p, p, p, ctypes.byref(c), None, 0, None) == _lib.PTY_EINVAL
    c = _constraints(probe_orthogonalize=1)
    assert lib.pty_constrain(ctypes.byref(g), p, p, None, p, ctypes.byref(c), None, 0, None) == _lib.PTY_EINVAL


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference: the oracle timed on the host, one JSON line with the contract keys."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "c1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def _plan(lib, g, B, budget):
    k, n = ctypes.c_int(0), ctypes.c_size_t(0)
    rc = lib.pty_plan_ckpt(ctypes.byref(g), B, budget, ctypes.byref(k), ctypes.byref(n))
    return rc, k.value, n.value


@pytest.mark.parametrize("Nz,N,M,B", [(20, 64, 3, 5), (8, 128, 6, 4), (7, 64, 1, 3)])
def test_checkpoint_plan_from_a_budget(lib, Nz, N, M, B):
    """The memory plan against the record's byte count B*M*N^2*8*blocks, blocks = 2 Nz - 1 for
    K = 1 and ceil(Nz/K) - 1 + 2K + 1 for K > 1 (anchors, segment waves and spectra, handed-over
    adjoint wave): K = 1 when it fits, else the largest K < Nz that fits and saves memory."""
    g = _geom(N=N, M=M, Nz=Nz, H=N + 40, W=N + 50)
    wave = B * M * N * N * 8
    blocks = {1: 2 * Nz - 1}
    for K in range(2, Nz):
        blocks[K] = -(-Nz // K) - 1 + 2 * K + 1
    ws = {K: lib.pty_workspace_size(ctypes.byref(_geom(N=N, M=M, Nz=Nz, H=N + 40, W=N + 50, ckpt_stride=K)), B)
          for K in blocks}
    for K in blocks:  # the workspace differs from K = 1's by exactly the record's blocks
        assert ws[1] - ws[K] == wave * (blocks[1] - blocks[K]), K
    # a budget that holds K = 1
    assert _plan(lib, g, B, ws[1]) == (_lib.PTY_OK, 1, ws[1])
    # every budget between the smallest plan and K = 1: the largest fitting K of smaller record
    for budget in sorted(set(ws.values())):
        if budget >= ws[1]:
            continue
        rc, k, n = _plan(lib, g, B, budget)
        expect = max(K for K in blocks if K > 1 and ws[K] <= budget)
        assert (rc, k, n) == (_lib.PTY_OK, expect, ws[expect]), budget
    # below the smallest plan: refused, with the smallest workspace in the message
    rc, k, n = _plan(lib, g, B, min(ws.values()) - 1)
    assert rc == _lib.PTY_EWORKSPACE and str(min(ws.values())) in lib.pty_last_error().decode()
    # the split-precision modes keep every checkpoint: K = 1 or nothing
    gs = _geom(N=N, M=M, Nz=Nz, H=N + 40, W=N + 50, fft_impl=1)
    full = lib.pty_workspace_size(ctypes.byref(gs), B)
    assert _plan(lib, gs, B, full)[:2] == (_lib.PTY_OK, 1)
    assert _plan(lib, gs, B, full - 1)[0] == _lib.PTY_EWORKSPACE
