/* pty_cnn.h -- C ABI of the learned initialiser: a small convolutional encoder-decoder that maps a
 * log-scaled S x S diffraction pattern to the (S/2) x (S/2) object patch under the centre of the
 * probe window (depth-summed phase and log-amplitude), trained on pairs that the forward model of
 * pty.h generates, and the stitching of its predictions into an initial object.
 *
 * The paper has no counterpart: it starts every reconstruction from a flat object (amplitude 1,
 * phase U[0, 1e-8], Sec. "Preprocessing and initialization") and mentions learned direct solvers
 * only as related work.  That flat start stays the fallback; this network only replaces it.
 *
 * Network (channels last, 3x3 convolutions with zero padding 1, bf16 weights and activations,
 * FP32 accumulation, FP32 biases):
 *   input   bf16(s_in * log(1 + I))                                   S x S x 1
 *   1       conv stride 2, 1 -> 48, ReLU                               S/2
 *   2       conv stride 2, 48 -> 96, ReLU                              S/4
 *   3       conv stride 2, 96 -> 192, ReLU                             S/8
 *   4       conv stride 2, 192 -> 384, ReLU                            S/16
 *   5       nearest upsampling x2, conv 384 -> 256, ReLU               S/8
 *   6       nearest upsampling x4, conv 256 -> 2 (linear, FP32 out)    S/2
 *   loss    mean squared error against the targets
 * Layers 1-5 run as implicit GEMMs on the tensor cores (bf16 operands); layer 6 (two output
 * channels) sums each tap's channel products once per low-resolution pixel on the CUDA cores.
 *
 * Parameters: one flat FP32 vector, layer after layer: weights [OC][3][3][IC] then biases [OC]
 * (pty_cnn_param_count() floats).  Patterns [B][S][S] FP32, DC-centred; predictions and targets
 * [B][S/2][S/2][2] FP32 (channel 0: sum over slices of the phase, 1: sum of log-amplitude).
 * All pointers are device pointers unless stated; arrays must be 16-byte aligned.  Calls are
 * asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream) and return PTY_OK or a
 * PTY_* code from pty.h with the reason in pty_last_error(); arguments are checked before any
 * launch.  S must be a multiple of 16 between 16 and 512.  The workspace starts with a status word
 * that pty_status() (pty.h) reads: PTY_ETIMEOUT if a tensor-core pipeline wait gave up (the
 * outputs of that call are then invalid). */
#ifndef PTY_CNN_H
#define PTY_CNN_H

#include <stddef.h>
#include <stdint.h>

#include "pty.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Number of FP32 parameters (weights and biases of the six layers). */
size_t pty_cnn_param_count(void);

/* Workspace bytes for batches of up to B patterns of S x S (0 and pty_last_error() if S or B is
 * invalid).  The workspace holds the bf16 weights, every layer's activations and their gradients;
 * it is the caller's and may be reused by calls that do not overlap on the GPU. */
size_t pty_cnn_workspace_size(int S, int B);

/* Predictions pred[B][S/2][S/2][2] for patterns I[B][S][S] with input scale s_in. */
int pty_cnn_forward(int S, int B, const float* params, const float* I, float s_in, float* pred, void* ws,
                    size_t ws_bytes, void* stream);

/* Loss mean((pred - Y)^2) over the batch into *loss (device double) and its gradient with respect
 * to the parameters into grad (device, pty_cnn_param_count() floats, overwritten).  Y[B][S/2][S/2][2].
 * pred may be NULL; otherwise the forward's predictions are also written there. */
int pty_cnn_loss_grad(int S, int B, const float* params, const float* I, const float* Y, float s_in, double* loss,
                      float* grad, float* pred, void* ws, size_t ws_bytes, void* stream);

/* One Adam step (PyTorch's bias-corrected Adam, step >= 1) on the flat parameter vector with
 * moment arrays m, v (zeroed by the caller before step 1). */
int pty_cnn_adam(float* params, float* m, float* v, const float* grad, int step, float lr, float beta1, float beta2,
                 float eps, void* stream);

/* pty_cnn_loss_grad followed by pty_cnn_adam; grad is scratch of pty_cnn_param_count() floats. */
int pty_cnn_train_step(int S, int B, float* params, float* m, float* v, float* grad, int step, float lr,
                       const float* I, const float* Y, float s_in, double* loss, void* ws, size_t ws_bytes,
                       void* stream);

/* Training targets for scan positions idx[B] of an object amp, phase [Nz][H][W]: the central
 * (S/2) x (S/2) of each S x S probe window (corner round(pos), half to even, clamped into the
 * object) of the depth-summed phase and log-amplitude, written to Y[B][S/2][S/2][2]. */
int pty_cnn_targets(int S, int Nz, int H, int W, const float* amp, const float* phase, const float* pos,
                    const int32_t* idx, int B, float* Y, void* stream);

/* Stitching: for scan positions idx[B] with predictions pred[B][S/2][S/2][2], adds weight * pred
 * into num[H][W][2] and weight into den[H][W] at the centre of each window (float atomics; the
 * caller zeroes num and den before the first batch).  weight[S/2][S/2] is typically the probe
 * intensity there. */
int pty_cnn_stitch(int S, int H, int W, const float* pred, const float* pos, const int32_t* idx, int B,
                   const float* weight, float* num, float* den, void* stream);

/* Initial object from the stitched sums: phase = (num0 / den) / Nz and amp = exp((num1 / den) / Nz)
 * in every slice; pixels with den = 0 get the flat start (amp 1, phase 0). */
int pty_cnn_stitch_finish(int Nz, int H, int W, const float* num, const float* den, float* amp, float* phase,
                          void* stream);

/* Copy, converted to FP32, what the last pty_cnn_forward / pty_cnn_loss_grad call on this workspace
 * left in it for layer `layer` (1..6): what = 0, the stored activation a_layer (layers 1..5,
 * [B][h][h][C], after bias, ReLU and bf16 rounding); what = 1, the bf16 gradient dL/dz_layer that
 * fed that layer's weight and input gradients (layers 1..6).  S and B must be those of that call.
 * For inspecting and testing the layers one at a time. */
int pty_cnn_read_state(int S, int B, const void* ws, size_t ws_bytes, int layer, int what, float* out,
                       void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PTY_CNN_H */
