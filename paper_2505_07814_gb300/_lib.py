"""ctypes binding of libpty.so (include/pty.h): same names, argument marshalling only.

Every array argument is a raw device address (int) or None; sizes are ints.  Nothing here
computes any part of the model.  Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpty.so")

PTY_OK = 0
PTY_EINVAL = 1
PTY_EBOUNDS = 2
PTY_EWORKSPACE = 4
PTY_ECUDA = 8
PTY_ETIMEOUT = 16
PTY_ENONFINITE = 32

PTY_LOSS_POISSON = 0
PTY_LOSS_GAUSSIAN = 1

PTY_GRAD_AMP = 1
PTY_GRAD_PHASE = 2
PTY_GRAD_PROBE = 4
PTY_GRAD_POS = 8
PTY_GRAD_TILT = 16
PTY_GRAD_DZ = 32
PTY_GRAD_ALL = 63
PTY_FFT_FP32, PTY_FFT_SPLIT_BF16, PTY_FFT_SPLIT_FP16, PTY_FFT_SPLIT3_BF16 = 0, 1, 2, 3

# Every symbol include/pty.h declares (checked by the CPU test suite).
EXPORTS = ("pty_workspace_size", "pty_forward", "pty_loss_grad", "pty_adam_update", "pty_step",
           "pty_status", "pty_last_error", "pty_supported_sizes", "pty_launch_count", "pty_profile_enable",
           "pty_profile_read", "pty_loss_grad_noalloc", "pty_forward_save", "pty_backward",
           "pty_cnn_param_count", "pty_cnn_workspace_size", "pty_cnn_forward", "pty_cnn_loss_grad", "pty_cnn_adam",
           "pty_cnn_train_step", "pty_cnn_targets", "pty_cnn_stitch", "pty_cnn_stitch_finish", "pty_cnn_read_state", "pty_constrain",
           "pty_constrain_workspace_size", "pty_loss_stats", "pty_loss_grad_part", "pty_set_wait_limit",
           "pty_plan_ckpt", "pty_fma_probe")
PROF_STAGES = ("prepare_object", "probe_spectrum", "forward", "loss", "loss_finalize", "adjoint", "object_grad",
               "probe_grad", "scalar_grad")


class pty_geom(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("Nz", ctypes.c_int), ("H", ctypes.c_int),
                ("W", ctypes.c_int), ("Ntot", ctypes.c_int), ("dx", ctypes.c_float),
                ("lambda_", ctypes.c_float), ("loss", ctypes.c_int), ("p", ctypes.c_float),
                ("eps", ctypes.c_float), ("grad_mask", ctypes.c_int), ("global_tilt", ctypes.c_int),
                ("ckpt_stride", ctypes.c_int), ("fft_impl", ctypes.c_int), ("w_pacbed", ctypes.c_float),
                ("p_pacbed", ctypes.c_float), ("w_sparse", ctypes.c_float), ("p_sparse", ctypes.c_float),
                ("obj_modes", ctypes.c_int)]


class pty_adam(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("m_amp", "v_amp", "m_phase", "v_phase", "m_probe", "v_probe",
                                               "m_pos", "v_pos", "m_tilt", "v_tilt", "m_dz", "v_dz")] + \
               [(n, ctypes.c_float) for n in ("lr_amp", "lr_phase", "lr_probe", "lr_pos", "lr_tilt", "lr_dz",
                                              "beta1", "beta2", "eps")]


class pty_constraints(ctypes.Structure):
    _fields_ = [("phase_positivity", ctypes.c_float), ("rz_sigma", ctypes.c_float), ("rz_relax", ctypes.c_float),
                ("kz_beta", ctypes.c_float), ("kz_alpha", ctypes.c_float), ("kz_relax", ctypes.c_float),
                ("probe_orthogonalize", ctypes.c_int)]


class PtyError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("pty error %d: %s" % (code, msg))
        self.code = code


_lib = None
P = ctypes.c_void_p
I = ctypes.c_int
SZ = ctypes.c_size_t


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpty.so (once).  Raises if it is missing: there is no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libpty.so is not built (%s); run paper_2505_07814_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    G = ctypes.POINTER(pty_geom)
    A = ctypes.POINTER(pty_adam)
    lib.pty_workspace_size.argtypes = [G, I]
    lib.pty_workspace_size.restype = SZ
    lib.pty_forward.argtypes = [G, I, P, P, P, P, P, P, P, P, P, SZ, P]
    lib.pty_forward.restype = I
    lib.pty_loss_grad.argtypes = [G, I, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, I, P, SZ, P]
    lib.pty_loss_grad.restype = I
    lib.pty_loss_stats.argtypes = [G, I, P, P, P, P, P, P, P, P, P, P, SZ, P]
    lib.pty_loss_stats.restype = I
    lib.pty_loss_grad_part.argtypes = [G, I, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, I, P, SZ, P]
    lib.pty_loss_grad_part.restype = I
    lib.pty_forward_save.argtypes = [G, I, P, P, P, P, P, P, P, P, P, SZ, P]
    lib.pty_forward_save.restype = I
    lib.pty_backward.argtypes = [G, I, P, P, P, P, P, P, P, P, P, P, P, P, P, P, I, P, SZ, P]
    lib.pty_backward.restype = I
    lib.pty_adam_update.argtypes = [G, P, P, P, P, P, P, P, P, P, P, P, P, A, I, P]
    lib.pty_adam_update.restype = I
    lib.pty_step.argtypes = [G, I, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, A, I, P, SZ, P]
    lib.pty_step.restype = I
    lib.pty_status.argtypes = [P, P]
    lib.pty_status.restype = I
    lib.pty_last_error.argtypes = []
    lib.pty_last_error.restype = ctypes.c_char_p
    lib.pty_supported_sizes.argtypes = []
    lib.pty_supported_sizes.restype = I
    lib.pty_loss_grad_noalloc.argtypes = [G, I, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, I, P, P]
    lib.pty_loss_grad_noalloc.restype = I
    lib.pty_launch_count.argtypes = []
    lib.pty_launch_count.restype = ctypes.c_longlong
    lib.pty_profile_enable.argtypes = [I]
    lib.pty_profile_enable.restype = I
    lib.pty_profile_read.argtypes = [ctypes.POINTER(ctypes.c_double), I]
    lib.pty_profile_read.restype = I
    lib.pty_plan_ckpt.argtypes = [G, I, SZ, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)]
    lib.pty_plan_ckpt.restype = I
    lib.pty_fma_probe.argtypes = [P, I, I, P]
    lib.pty_fma_probe.restype = I
    lib.pty_set_wait_limit.argtypes = [ctypes.c_longlong]
    lib.pty_set_wait_limit.restype = I
    F = ctypes.c_float
    lib.pty_cnn_param_count.argtypes = []
    lib.pty_cnn_param_count.restype = SZ
    lib.pty_cnn_workspace_size.argtypes = [I, I]
    lib.pty_cnn_workspace_size.restype = SZ
    lib.pty_cnn_forward.argtypes = [I, I, P, P, F, P, P, SZ, P]
    lib.pty_cnn_forward.restype = I
    lib.pty_cnn_loss_grad.argtypes = [I, I, P, P, P, F, P, P, P, P, SZ, P]
    lib.pty_cnn_loss_grad.restype = I
    lib.pty_cnn_adam.argtypes = [P, P, P, P, I, F, F, F, F, P]
    lib.pty_cnn_adam.restype = I
    lib.pty_cnn_train_step.argtypes = [I, I, P, P, P, P, I, F, P, P, F, P, P, SZ, P]
    lib.pty_cnn_train_step.restype = I
    lib.pty_cnn_targets.argtypes = [I, I, I, I, P, P, P, P, I, P, P]
    lib.pty_cnn_targets.restype = I
    lib.pty_cnn_stitch.argtypes = [I, I, I, P, P, P, I, P, P, P, P]
    lib.pty_cnn_stitch.restype = I
    lib.pty_cnn_stitch_finish.argtypes = [I, I, I, P, P, P, P, P]
    lib.pty_cnn_stitch_finish.restype = I
    lib.pty_cnn_read_state.argtypes = [I, I, P, SZ, I, I, P, P]
    lib.pty_cnn_read_state.restype = I
    lib.pty_constrain.argtypes = [G, P, P, P, P, ctypes.POINTER(pty_constraints), P, SZ, P]
    lib.pty_constrain.restype = I
    lib.pty_constrain_workspace_size.argtypes = [G, ctypes.POINTER(pty_constraints)]
    lib.pty_constrain_workspace_size.restype = SZ
    _lib = lib
    return lib


def _check(rc: int):
    if rc != PTY_OK:
        raise PtyError(rc, load().pty_last_error().decode())


def pty_workspace_size(geom: pty_geom, B: int) -> int:
    n = load().pty_workspace_size(ctypes.byref(geom), B)
    if n == 0:
        raise PtyError(PTY_EINVAL, load().pty_last_error().decode())
    return n


def pty_forward(geom, B, idx, amp, phase, probe, pos, tilt, dz, I_model, ws, ws_bytes, stream):
    _check(load().pty_forward(ctypes.byref(geom), B, idx, amp, phase, probe, pos, tilt, dz, I_model, ws,
                              ws_bytes, stream))


def pty_loss_grad(geom, B, idx, amp, phase, probe, pos, tilt, dz, I_meas, loss, I_model, g_amp, g_phase,
                  g_probe, g_pos, g_tilt, g_dz, accumulate, ws, ws_bytes, stream):
    _check(load().pty_loss_grad(ctypes.byref(geom), B, idx, amp, phase, probe, pos, tilt, dz, I_meas, loss,
                                I_model, g_amp, g_phase, g_probe, g_pos, g_tilt, g_dz, int(accumulate), ws,
                                ws_bytes, stream))


def pty_plan_ckpt(geom, B: int, budget_bytes: int) -> tuple[int, int]:
    """(ckpt_stride, workspace bytes) of the adjoint memory plan that fits budget_bytes."""
    k, n = ctypes.c_int(0), ctypes.c_size_t(0)
    _check(load().pty_plan_ckpt(ctypes.byref(geom), B, budget_bytes, ctypes.byref(k), ctypes.byref(n)))
    return k.value, n.value


def pty_loss_stats(geom, B, idx, amp, phase, probe, pos, tilt, dz, I_meas, stats, ws, ws_bytes, stream):
    _check(load().pty_loss_stats(ctypes.byref(geom), B, idx, amp, phase, probe, pos, tilt, dz, I_meas, stats, ws,
                                 ws_bytes, stream))


def pty_loss_grad_part(geom, B, idx, amp, phase, probe, pos, tilt, dz, I_meas, whole_stats, loss, I_model, g_amp,
                       g_phase, g_probe, g_pos, g_tilt, g_dz, accumulate, ws, ws_bytes, stream):
    _check(load().pty_loss_grad_part(ctypes.byref(geom), B, idx, amp, phase, probe, pos, tilt, dz, I_meas,
                                     whole_stats, loss, I_model, g_amp, g_phase, g_probe, g_pos, g_tilt, g_dz,
                                     int(accumulate), ws, ws_bytes, stream))


def pty_forward_save(geom, B, idx, amp, phase, probe, pos, tilt, dz, I_model, ws, ws_bytes, stream):
    _check(load().pty_forward_save(ctypes.byref(geom), B, idx, amp, phase, probe, pos, tilt, dz, I_model, ws,
                                   ws_bytes, stream))


def pty_backward(geom, B, idx, amp, phase, probe, pos, tilt, dz, dL_dI, g_amp, g_phase, g_probe, g_pos, g_tilt,
                 g_dz, accumulate, ws, ws_bytes, stream):
    _check(load().pty_backward(ctypes.byref(geom), B, idx, amp, phase, probe, pos, tilt, dz, dL_dI, g_amp, g_phase,
                               g_probe, g_pos, g_tilt, g_dz, int(accumulate), ws, ws_bytes, stream))


def pty_adam_update(geom, amp, phase, probe, pos, tilt, dz, g_amp, g_phase, g_probe, g_pos, g_tilt, g_dz,
                    adam: pty_adam, step, stream):
    _check(load().pty_adam_update(ctypes.byref(geom), amp, phase, probe, pos, tilt, dz, g_amp, g_phase, g_probe,
                                  g_pos, g_tilt, g_dz, ctypes.byref(adam), step, stream))


def pty_step(geom, B, idx, amp, phase, probe, pos, tilt, dz, I_meas, loss, g_amp, g_phase, g_probe, g_pos,
             g_tilt, g_dz, adam: pty_adam, step, ws, ws_bytes, stream):
    _check(load().pty_step(ctypes.byref(geom), B, idx, amp, phase, probe, pos, tilt, dz, I_meas, loss, g_amp,
                           g_phase, g_probe, g_pos, g_tilt, g_dz, ctypes.byref(adam), step, ws, ws_bytes, stream))


def pty_status(ws, stream) -> int:
    return load().pty_status(ws, stream)


def pty_last_error() -> str:
    return load().pty_last_error().decode()


def pty_supported_sizes() -> int:
    return load().pty_supported_sizes()


def pty_launch_count() -> int:
    return load().pty_launch_count()


def pty_profile_enable(on: bool):
    _check(load().pty_profile_enable(int(on)))


def pty_profile_read() -> tuple[int, dict]:
    """(number of recorded calls, {stage name: summed device milliseconds})."""
    buf = (ctypes.c_double * len(PROF_STAGES))()
    n = load().pty_profile_read(buf, len(PROF_STAGES))
    if n < 0:
        raise PtyError(PTY_ECUDA, "profile read failed")
    return n, {name: buf[k] for k, name in enumerate(PROF_STAGES)}


def pty_fma_probe(sink, blocks: int, iters: int, stream):
    _check(load().pty_fma_probe(sink, blocks, iters, stream))


def pty_set_wait_limit(polls: int):
    _check(load().pty_set_wait_limit(int(polls)))


def pty_loss_grad_noalloc(geom, B, idx, amp, phase, probe, pos, tilt, dz, I_meas, loss, I_model, g_amp, g_phase,
                          g_probe, g_pos, g_tilt, g_dz, accumulate, status, stream):
    _check(load().pty_loss_grad_noalloc(ctypes.byref(geom), B, idx, amp, phase, probe, pos, tilt, dz, I_meas, loss,
                                        I_model, g_amp, g_phase, g_probe, g_pos, g_tilt, g_dz, int(accumulate),
                                        status, stream))


# ---- learned initialiser (include/pty_cnn.h) ----
def pty_cnn_param_count() -> int:
    return load().pty_cnn_param_count()


def pty_cnn_workspace_size(S: int, B: int) -> int:
    n = load().pty_cnn_workspace_size(S, B)
    if n == 0:
        raise PtyError(PTY_EINVAL, load().pty_last_error().decode())
    return n


def pty_cnn_forward(S, B, params, I, s_in, pred, ws, ws_bytes, stream):
    _check(load().pty_cnn_forward(S, B, params, I, s_in, pred, ws, ws_bytes, stream))


def pty_cnn_loss_grad(S, B, params, I, Y, s_in, loss, grad, pred, ws, ws_bytes, stream):
    _check(load().pty_cnn_loss_grad(S, B, params, I, Y, s_in, loss, grad, pred, ws, ws_bytes, stream))


def pty_cnn_adam(params, m, v, grad, step, lr, beta1, beta2, eps, stream):
    _check(load().pty_cnn_adam(params, m, v, grad, step, lr, beta1, beta2, eps, stream))


def pty_cnn_train_step(S, B, params, m, v, grad, step, lr, I, Y, s_in, loss, ws, ws_bytes, stream):
    _check(load().pty_cnn_train_step(S, B, params, m, v, grad, step, lr, I, Y, s_in, loss, ws, ws_bytes, stream))


def pty_cnn_targets(S, Nz, H, W, amp, phase, pos, idx, B, Y, stream):
    _check(load().pty_cnn_targets(S, Nz, H, W, amp, phase, pos, idx, B, Y, stream))


def pty_cnn_stitch(S, H, W, pred, pos, idx, B, weight, num, den, stream):
    _check(load().pty_cnn_stitch(S, H, W, pred, pos, idx, B, weight, num, den, stream))


def pty_cnn_stitch_finish(Nz, H, W, num, den, amp, phase, stream):
    _check(load().pty_cnn_stitch_finish(Nz, H, W, num, den, amp, phase, stream))


def pty_cnn_read_state(S, B, ws, ws_bytes, layer, what, out, stream):
    _check(load().pty_cnn_read_state(S, B, ws, ws_bytes, layer, what, out, stream))


def pty_constrain_workspace_size(geom, c: pty_constraints) -> int:
    return load().pty_constrain_workspace_size(ctypes.byref(geom), ctypes.byref(c))


def pty_constrain(geom, amp, phase, probe, dz, c: pty_constraints, ws, ws_bytes: int, stream):
    _check(load().pty_constrain(ctypes.byref(geom), amp, phase, probe, dz, ctypes.byref(c), ws, ws_bytes, stream))
