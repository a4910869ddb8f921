// pty_internal.h -- validated problem description and workspace layout shared by the launchers.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "pty.h"

namespace pty {

// Workspace carve-up (all pieces 256-byte aligned).  k-space arrays use the FFT's digit-ordered
// layout: element p1 * N + p0 holds frequency (kbin(p0), kbin(p1)) along (axis 0, axis 1).
struct Workspace {
  int* status;     // [1]   device status bits
  float2* T;       // [Ko][Nz][H][W]  transmission amp * exp(i phase)
  float2* Phat;    // [M][N*N]        probe spectra F[P_m] (k-space layout)
  float2* ckpt;     // [B][M][Nz][N*N] wave entering each slice (natural layout); recompute mode:
                    // [B][M][K][N*N], the current segment's entering waves
  float2* vhat;     // [B][M][Nz-1][N*N] propagated spectra / N^2 (k-space), for dz/tilt gradients;
                    // recompute mode: [B][M][K][N*N], slot j = spectrum entering slice s0 + j
  float2* anchors;  // recompute mode: [B][M][nseg-1][N*N] spectrum entering slices K, 2K, ...
  float2* gstate;   // recompute mode: [B][M][N*N] adjoint wave handed between segments
  float2* Psi;     // [B][M][N*N]     far-field waves (k-space)
  float* Imode;    // [B][M][N*N]     per-mode far-field intensity (k-space)
  float* u;        // [B][N*N]        dL/dI before the batch normaliser (k-space)
  double* lpart;   // [B][2]          per-pattern loss sums
  double* scal;    // [4]             {dL/dI normaliser, loss, -, -}
  float2* gT;      // [Ko][Nz][H][W]  dL/dT accumulator
  float2* gPhat;   // [M][N*N]        probe-spectrum gradient accumulator (k-space)
  double* spart;   // [B][M][5]       per-wave {pos0, pos1, tilt0, tilt1, dz} gradient partials
  // split-precision DFT modes only
  float2* wave;    // [B][M][N*N]     current wave of every (position, mode)
  float2* tmp;     // [B][M][N*N]     half-transformed waves (transposed per wave)
  float* gscal;    // [4]             fp16 batch scaling: {max |x| bits, scale, -, -}
  // extra loss terms (when their weights are non-zero)
  float* pac;      // [3][N*N]        sum over the batch of I_model, of I_meas (k-space), PACBED dL/dI
  double* pacpart; // [B]             per-pattern sums of I_meas^p_pacbed
  double* sppart;  // [152*8]         partial sums of c |phase|^p_sparse (sparsity term)
  int* cover;      // [H][W+1]        patch coverage count c of the batch (sparsity term)
  void* pieces0;   // [B][M][N][pieces][2N] 16-bit split operands of the tensor-core GEMMs
  void* pieces1;   // (the same, for the second GEMM of a 2D transform)
};

// MODE_FORWARD: patterns only.  MODE_FORWARD_SAVE: patterns, keeping in the workspace what a later
// MODE_BACKWARD needs.  MODE_GRAD: loss and gradients in one pass.  MODE_BACKWARD: gradients for a
// caller-supplied dL/dI, after a MODE_FORWARD_SAVE pass on the same workspace.
// MODE_STATS: the loss statistics of the batch only (pty_loss_stats).
enum Mode { MODE_FORWARD = 0, MODE_GRAD = 1, MODE_FORWARD_SAVE = 2, MODE_BACKWARD = 3, MODE_STATS = 4 };

struct Problem {
  int N, M, Nz, H, W, Ntot, B;
  int Ko;  // object modes (>= 1); waves are ordered (position, probe mode, object mode)
  float dx, lam;
  int loss;
  float p, eps;
  int grad_mask, global_tilt, accumulate, mode;
  int kstride;  // slices per recompute segment (1: every slice's checkpoint is stored)
  int fft_impl;  // PTY_FFT_*
  float w_pac, p_pac, w_sp, p_sp;  // extra loss terms (weights 0 = off), exponents resolved
  const int32_t* idx;
  const float *amp, *phase, *pos, *tilt, *dz;
  const float2* probe;
  const float* I_meas;
  const float* dldi;  // MODE_BACKWARD: dL/dI [B][N][N], DC-centred
  double* loss_out;
  // Statistics of the whole batch when this call holds one part of it (pty_loss_grad_part), or
  // nullptr: {sum of I_meas^p, sum of the Gaussian squared residuals, detector pixels x patterns}.
  const double* whole;
  double* stats_out;  // MODE_STATS: this call's part of those three sums
  float* I_model;
  float *g_amp, *g_phase, *g_pos, *g_tilt, *g_dz;
  float2* g_probe;
  Workspace ws;
  cudaStream_t stream;
};

// Slices per recompute segment a pass will use (see pty_geom.ckpt_stride).
int effective_stride(const pty_geom& g);

// Byte offsets of the workspace pieces; returns the total size.  base may be NULL (size query).
size_t layout_workspace(const pty_geom& g, int B, int mode, char* base, Workspace* out);

// One pass of the hot path for FFT size N (instantiated in pty_n<N>.cu).  Returns a PTY_* code.
template <int N>
int run_pipeline(const Problem& pb);
// The same pass with split-precision DFT-GEMMs (P = PTY_FFT_SPLIT_BF16 or _FP16; N = 64, 128).
template <int N, int P>
int run_pipeline_gemm(const Problem& pb);

void set_error(const char* fmt, ...);
// Current poll limit of the tensor-core GEMM's pipeline waits (pty_set_wait_limit).
long stage_wait_limit();
// Checks the fields of a geometry every entry point shares; PTY_OK or PTY_EINVAL (message set).
int validate_geom(const pty_geom* g);

inline bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

#define REQUIRE(cond, ...)     \
  do {                         \
    if (!(cond)) {             \
      set_error(__VA_ARGS__);  \
      return PTY_EINVAL;       \
    }                          \
  } while (0)

// Diagnostics: launch counter and optional per-stage event timing (pty_profile_*).
void note_launch();
void prof_begin(cudaStream_t st);     // start of a pipeline call
void prof_mark(int stage, cudaStream_t st);  // after the kernel of `stage`

}  // namespace pty
