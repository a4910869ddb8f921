// pty_api.cu -- the C ABI declared in include/pty.h: host-side validation, workspace layout,
// dispatch on the window size N, and the Adam update.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "pty_internal.h"

namespace pty {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

// ---------------------------------------------------------------------------------------------
// Diagnostics
// ---------------------------------------------------------------------------------------------
static long long g_launches = 0;
static const int kProfCalls = 256;
static bool g_prof_on = false;
static int g_prof_calls = 0;
static cudaEvent_t g_prof_ev[kProfCalls][PTY_PROF_STAGES + 1];
static bool g_prof_have[kProfCalls][PTY_PROF_STAGES + 1];
static bool g_prof_created = false;

void note_launch() { __atomic_add_fetch(&g_launches, 1, __ATOMIC_RELAXED); }

void prof_begin(cudaStream_t st) {
  if (!g_prof_on || g_prof_calls >= kProfCalls) return;
  for (int k = 0; k <= PTY_PROF_STAGES; ++k) g_prof_have[g_prof_calls][k] = false;
  cudaEventRecord(g_prof_ev[g_prof_calls][0], st);
  g_prof_have[g_prof_calls][0] = true;
  ++g_prof_calls;
}

void prof_mark(int stage, cudaStream_t st) {
  if (!g_prof_on || g_prof_calls == 0 || g_prof_calls > kProfCalls) return;
  const int c = g_prof_calls - 1;
  cudaEventRecord(g_prof_ev[c][stage + 1], st);
  g_prof_have[c][stage + 1] = true;
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Poll limit of the tensor-core GEMM's pipeline waits (pty_set_wait_limit).
static long g_stage_spin = -1;
long stage_wait_limit() { return g_stage_spin >= 0 ? g_stage_spin : (long)PTY_WAIT_POLLS_DEFAULT; }

// Slices per recompute segment actually used: 1 (checkpoint every slice) unless the caller asked for
// a stride and some gradient needs the forward waves.
int effective_stride(const pty_geom& g) {
  const bool needs = (g.grad_mask & (PTY_GRAD_AMP | PTY_GRAD_PHASE)) ||
                     ((g.grad_mask & (PTY_GRAD_DZ | PTY_GRAD_TILT)) && g.Nz > 1);
  if (!needs || g.ckpt_stride <= 1 || g.fft_impl != PTY_FFT_FP32) return 1;
  return g.ckpt_stride < g.Nz ? g.ckpt_stride : g.Nz;
}

size_t layout_workspace(const pty_geom& g, int B, int mode, char* base, Workspace* out) {
  const size_t NN = (size_t)g.N * g.N;
  const size_t Ko = g.obj_modes > 1 ? (size_t)g.obj_modes : 1;
  const size_t nobj = Ko * g.Nz * g.H * g.W;
  const size_t waves = (size_t)B * g.M * Ko;
  const bool grad = mode != MODE_FORWARD && mode != MODE_STATS;
  const bool want_obj = grad && (g.grad_mask & (PTY_GRAD_AMP | PTY_GRAD_PHASE));
  const bool want_prop = grad && (g.grad_mask & (PTY_GRAD_DZ | PTY_GRAD_TILT)) && g.Nz > 1;
  const bool want_probe = grad && (g.grad_mask & PTY_GRAD_PROBE);
  const int K = effective_stride(g);
  const int nseg = (g.Nz + K - 1) / K;
  size_t off = 0;
  Workspace w;
  memset(&w, 0, sizeof(w));
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  w.status = (int*)take(sizeof(int) * 64);
  w.scal = (double*)take(sizeof(double) * 4);
  w.T = (float2*)take(sizeof(float2) * nobj);
  w.Phat = (float2*)take(sizeof(float2) * g.M * NN);
  w.Imode = (float*)take(sizeof(float) * waves * NN);
  if (mode == MODE_STATS) {
    w.u = (float*)take(sizeof(float) * (size_t)B * NN);
    w.lpart = (double*)take(sizeof(double) * 2 * (size_t)(B > 0 ? B : 1));
  }
  if (grad) {
    if (K == 1) {
      if (want_obj) w.ckpt = (float2*)take(sizeof(float2) * waves * g.Nz * NN);
      if (want_prop) w.vhat = (float2*)take(sizeof(float2) * waves * (g.Nz - 1) * NN);
    } else {
      if (nseg > 1) w.anchors = (float2*)take(sizeof(float2) * waves * (nseg - 1) * NN);
      if (want_obj) w.ckpt = (float2*)take(sizeof(float2) * waves * K * NN);
      if (want_prop) w.vhat = (float2*)take(sizeof(float2) * waves * K * NN);
      w.gstate = (float2*)take(sizeof(float2) * waves * NN);
    }
    w.Psi = (float2*)take(sizeof(float2) * waves * NN);
    w.u = (float*)take(sizeof(float) * (size_t)B * NN);
    w.lpart = (double*)take(sizeof(double) * 2 * (size_t)(B > 0 ? B : 1));
    if (want_obj) w.gT = (float2*)take(sizeof(float2) * nobj);
    if (want_probe) w.gPhat = (float2*)take(sizeof(float2) * g.M * NN);
    w.spart = (double*)take(sizeof(double) * 5 * (waves > 0 ? waves : 1));
    if (g.w_pacbed > 0.f) {
      w.pac = (float*)take(sizeof(float) * 3 * NN);
      w.pacpart = (double*)take(sizeof(double) * (size_t)(B > 0 ? B : 1));
    }
    if (g.w_sparse > 0.f) {
      w.sppart = (double*)take(sizeof(double) * 152 * 8);
      w.cover = (int*)take(sizeof(int) * (size_t)g.H * (g.W + 1));
    }
  }
  if (g.fft_impl != PTY_FFT_FP32) {
    w.wave = (float2*)take(sizeof(float2) * waves * NN);
    w.tmp = (float2*)take(sizeof(float2) * waves * NN);
    w.gscal = (float*)take(sizeof(float) * 4);
    const size_t pieces = g.fft_impl == PTY_FFT_SPLIT3_BF16 ? 3 : 2;
    w.pieces0 = take(2 * pieces * 2 * waves * NN);
    w.pieces1 = take(2 * pieces * 2 * waves * NN);
  }
  if (out) *out = w;
  return off;
}

static bool supported_N(int N) { return N == 64 || N == 128 || N == 256; }

int validate_geom(const pty_geom* g) {
  if (!g) {
    set_error("geometry is NULL");
    return PTY_EINVAL;
  }
  if (!supported_N(g->N)) {
    set_error("N = %d is not supported (64, 128 or 256)", g->N);
    return PTY_EINVAL;
  }
  if (g->M < 1 || g->Nz < 1 || g->H < g->N || g->W < g->N || g->Ntot < 0) {
    set_error("bad shape: M=%d Nz=%d H=%d W=%d Ntot=%d (need M,Nz >= 1, H,W >= N)", g->M, g->Nz, g->H, g->W,
              g->Ntot);
    return PTY_EINVAL;
  }
  if (!(g->dx > 0.f) || !(g->lambda > 0.f) || !isfinite(g->dx) || !isfinite(g->lambda)) {
    set_error("dx and lambda must be positive and finite");
    return PTY_EINVAL;
  }
  if (g->loss != PTY_LOSS_POISSON && g->loss != PTY_LOSS_GAUSSIAN) {
    set_error("unknown loss kind %d", g->loss);
    return PTY_EINVAL;
  }
  if ((g->grad_mask & ~PTY_GRAD_ALL) != 0) {
    set_error("unknown bits in grad_mask 0x%x", g->grad_mask);
    return PTY_EINVAL;
  }
  if (g->fft_impl < PTY_FFT_FP32 || g->fft_impl > PTY_FFT_SPLIT3_BF16) {
    set_error("unknown fft_impl %d", g->fft_impl);
    return PTY_EINVAL;
  }
  if (g->fft_impl != PTY_FFT_FP32 && g->N != 64 && g->N != 128) {
    set_error("split-precision DFTs support N = 64 and 128, not %d", g->N);
    return PTY_EINVAL;
  }
  if (!(g->w_pacbed >= 0.f) || !(g->w_sparse >= 0.f) || !isfinite(g->w_pacbed) || !isfinite(g->w_sparse) ||
      !isfinite(g->p_pacbed) || !isfinite(g->p_sparse)) {
    set_error("w_pacbed, w_sparse must be finite and >= 0, p_pacbed, p_sparse finite");
    return PTY_EINVAL;
  }
  if (g->ckpt_stride < 0) {
    set_error("ckpt_stride %d < 0", g->ckpt_stride);
    return PTY_EINVAL;
  }
  if (g->obj_modes < 0 || g->obj_modes > 64) {
    set_error("obj_modes = %d outside 0 .. 64", g->obj_modes);
    return PTY_EINVAL;
  }
  if ((double)(g->obj_modes > 1 ? g->obj_modes : 1) * g->Nz * g->H * g->W > 4.0e9) {
    set_error("object too large");
    return PTY_EINVAL;
  }
  return PTY_OK;
}


static int prepare(const pty_geom* g, int B, int mode, const int32_t* idx, const float* amp, const float* phase,
                   const float* probe, const float* pos, const float* tilt, const float* dz, void* ws,
                   size_t ws_bytes, void* stream, Problem* pb) {
  int rc = validate_geom(g);
  if (rc) return rc;
  REQUIRE(B >= 0, "batch size %d < 0", B);
  REQUIRE((double)B * g->M * (g->obj_modes > 1 ? g->obj_modes : 1) < 2.0e9, "batch too large");
  REQUIRE(amp && phase && probe && pos && tilt && dz, "a parameter pointer is NULL");
  REQUIRE(B == 0 || idx, "idx is NULL");
  REQUIRE(B == 0 || g->Ntot >= 1, "a non-empty batch needs Ntot >= 1");
  REQUIRE(ws, "workspace is NULL");
  REQUIRE(aligned(probe, 8) && aligned(ws, 256), "probe must be 8-byte and workspace 256-byte aligned");
  REQUIRE(aligned(amp, 4) && aligned(phase, 4) && aligned(pos, 4) && aligned(tilt, 4) && aligned(dz, 4),
          "float arrays must be 4-byte aligned");
  const size_t need = layout_workspace(*g, B, mode, nullptr, nullptr);
  if (ws_bytes < need) {
    set_error("workspace has %zu bytes, %zu needed", ws_bytes, need);
    return PTY_EWORKSPACE;
  }
  memset(pb, 0, sizeof(*pb));
  pb->N = g->N;
  pb->M = g->M;
  pb->Ko = g->obj_modes > 1 ? g->obj_modes : 1;
  pb->Nz = g->Nz;
  pb->H = g->H;
  pb->W = g->W;
  pb->Ntot = g->Ntot;
  pb->B = B;
  pb->dx = g->dx;
  pb->lam = g->lambda;
  pb->loss = g->loss;
  pb->p = g->p > 0.f ? g->p : (g->loss == PTY_LOSS_POISSON ? 1.0f : 0.5f);
  pb->eps = g->eps;
  pb->grad_mask = g->grad_mask;
  pb->global_tilt = g->global_tilt ? 1 : 0;
  pb->mode = mode;
  pb->kstride = effective_stride(*g);
  pb->fft_impl = g->fft_impl;
  pb->w_pac = g->w_pacbed;
  pb->p_pac = g->p_pacbed > 0.f ? g->p_pacbed : 0.5f;
  pb->w_sp = g->w_sparse;
  pb->p_sp = g->p_sparse > 0.f ? g->p_sparse : 1.0f;
  pb->idx = idx;
  pb->amp = amp;
  pb->phase = phase;
  pb->probe = reinterpret_cast<const float2*>(probe);
  pb->pos = pos;
  pb->tilt = tilt;
  pb->dz = dz;
  pb->stream = (cudaStream_t)stream;
  layout_workspace(*g, B, mode, (char*)ws, &pb->ws);
  return PTY_OK;
}

// Clears the status word, then runs the pipeline.  First CUDA call of every entry point.
static int dispatch(const Problem& pb) {
  if (cudaMemsetAsync(pb.ws.status, 0, sizeof(int), pb.stream) != cudaSuccess) {
    set_error("cudaMemsetAsync failed: %s", cudaGetErrorString(cudaGetLastError()));
    return PTY_ECUDA;
  }
  if (pb.fft_impl == PTY_FFT_SPLIT_BF16) return pb.N == 64 ? run_pipeline_gemm<64, 1>(pb) : run_pipeline_gemm<128, 1>(pb);
  if (pb.fft_impl == PTY_FFT_SPLIT_FP16) return pb.N == 64 ? run_pipeline_gemm<64, 2>(pb) : run_pipeline_gemm<128, 2>(pb);
  if (pb.fft_impl == PTY_FFT_SPLIT3_BF16) return pb.N == 64 ? run_pipeline_gemm<64, 3>(pb) : run_pipeline_gemm<128, 3>(pb);
  switch (pb.N) {
    case 64: return run_pipeline<64>(pb);
    case 128: return run_pipeline<128>(pb);
    case 256: return run_pipeline<256>(pb);
    default: set_error("N = %d not supported", pb.N); return PTY_EINVAL;
  }
}

// ---------------------------------------------------------------------------------------------
// Adam (PyTorch semantics), one launch over every enabled parameter.
// ---------------------------------------------------------------------------------------------
struct AdamSeg {
  float* p;
  const float* g;
  float* m;
  float* v;
  size_t n;
  float lr;
};
struct AdamArgs {
  AdamSeg seg[6];
  int nseg;
  float beta1, beta2, eps, bc1, bc2;
};

__global__ void k_adam(AdamArgs a) {
  for (int k = 0; k < a.nseg; ++k) {
    const AdamSeg s = a.seg[k];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < s.n; i += (size_t)gridDim.x * blockDim.x) {
      const float g = s.g[i];
      const float m = a.beta1 * s.m[i] + (1.f - a.beta1) * g;
      const float v = a.beta2 * s.v[i] + (1.f - a.beta2) * g * g;
      s.m[i] = m;
      s.v[i] = v;
      const float mh = m / a.bc1;
      const float vh = v / a.bc2;
      s.p[i] -= s.lr * mh / (sqrtf(vh) + a.eps);
    }
  }
}

// Output checks and dispatch of a loss-and-gradient pass prepared in pb.
static int grad_call(Problem& pb, const pty_geom* geom, int B, const float* I_meas, double* loss, float* I_model,
                     float* g_amp, float* g_phase, float* g_probe, float* g_pos, float* g_tilt, float* g_dz,
                     int accumulate) {
  const int gm = geom->grad_mask;
  REQUIRE(B == 0 || I_meas, "I_meas is NULL");
  REQUIRE(!(gm & PTY_GRAD_AMP) || g_amp, "g_amp is NULL but PTY_GRAD_AMP is requested");
  REQUIRE(!(gm & PTY_GRAD_PHASE) || g_phase, "g_phase is NULL but PTY_GRAD_PHASE is requested");
  REQUIRE(!(gm & PTY_GRAD_PROBE) || (g_probe && aligned(g_probe, 8)), "g_probe is NULL or misaligned");
  REQUIRE(!(gm & PTY_GRAD_POS) || g_pos, "g_pos is NULL but PTY_GRAD_POS is requested");
  REQUIRE(!(gm & PTY_GRAD_TILT) || g_tilt, "g_tilt is NULL but PTY_GRAD_TILT is requested");
  REQUIRE(!(gm & PTY_GRAD_DZ) || g_dz, "g_dz is NULL but PTY_GRAD_DZ is requested");
  pb.I_meas = I_meas;
  pb.loss_out = loss;
  pb.I_model = I_model;
  pb.g_amp = g_amp;
  pb.g_phase = g_phase;
  pb.g_probe = reinterpret_cast<float2*>(g_probe);
  pb.g_pos = g_pos;
  pb.g_tilt = g_tilt;
  pb.g_dz = g_dz;
  pb.accumulate = accumulate ? 1 : 0;
  return dispatch(pb);
}

// FP32 FMA throughput probe: eight independent chains per thread, 16 fused multiply-adds of each
// per iteration.  The result is stored only if it equals a value it never takes, so the work is
// not optimised away and nothing is written.
__global__ void __launch_bounds__(512) k_fma_probe(float* sink, int iters) {
  float a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = (float)(threadIdx.x + c);
  const float b = 0.999f, d = 0.001f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
#pragma unroll
      for (int c = 0; c < 8; ++c) a[c] = fmaf(a[c], b, d);
    }
  }
  float r = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) r += a[c];
  if (r == -1.0f) sink[0] = r;
}

}  // namespace pty

using namespace pty;

extern "C" {

size_t pty_workspace_size(const pty_geom* geom, int B) {
  if (validate_geom(geom) != PTY_OK || B < 0) return 0;
  return layout_workspace(*geom, B, MODE_GRAD, nullptr, nullptr);
}

int pty_plan_ckpt(const pty_geom* geom, int B, size_t budget_bytes, int* stride, size_t* ws_bytes) {
  int rc = validate_geom(geom);
  if (rc) return rc;
  REQUIRE(B >= 0, "batch size %d < 0", B);
  REQUIRE(stride, "stride is NULL");
  pty_geom g = *geom;
  g.ckpt_stride = 1;
  const size_t full = layout_workspace(g, B, MODE_GRAD, nullptr, nullptr);
  int best = full <= budget_bytes ? 1 : 0;
  size_t best_bytes = full, least = full;
  if (!best && g.fft_impl == PTY_FFT_FP32) {
    // every K > 1 replays each slice once; fewer, longer segments (larger K) ran faster, so take the
    // largest K whose workspace fits (the record shrinks, then grows again past K ~ sqrt(Nz / 2))
    for (int K = 2; K < g.Nz; ++K) {
      g.ckpt_stride = K;
      const size_t n = layout_workspace(g, B, MODE_GRAD, nullptr, nullptr);
      if (n < least) least = n;
      if (n <= budget_bytes && n < full) {
        best = K;
        best_bytes = n;
      }
    }
  }
  if (!best) {
    set_error("no checkpoint plan fits %zu bytes: the smallest workspace for this batch is %zu bytes%s", budget_bytes,
              least, geom->fft_impl != PTY_FFT_FP32 ? " (the split-precision modes keep every checkpoint)" : "");
    return PTY_EWORKSPACE;
  }
  *stride = best;
  if (ws_bytes) *ws_bytes = best_bytes;
  return PTY_OK;
}

int pty_forward(const pty_geom* geom, int B, const int32_t* idx, const float* amp, const float* phase,
                const float* probe, const float* pos, const float* tilt, const float* dz, float* I_model, void* ws,
                size_t ws_bytes, void* stream) {
  Problem pb;
  int rc = prepare(geom, B, MODE_FORWARD, idx, amp, phase, probe, pos, tilt, dz, ws, ws_bytes, stream, &pb);
  if (rc) return rc;
  REQUIRE(B == 0 || I_model, "I_model is NULL");
  pb.I_model = I_model;
  return dispatch(pb);
}

int pty_loss_grad(const pty_geom* geom, int B, const int32_t* idx, const float* amp, const float* phase,
                  const float* probe, const float* pos, const float* tilt, const float* dz, const float* I_meas,
                  double* loss, float* I_model, float* g_amp, float* g_phase, float* g_probe, float* g_pos,
                  float* g_tilt, float* g_dz, int accumulate, void* ws, size_t ws_bytes, void* stream) {
  Problem pb;
  int rc = prepare(geom, B, MODE_GRAD, idx, amp, phase, probe, pos, tilt, dz, ws, ws_bytes, stream, &pb);
  if (rc) return rc;
  return grad_call(pb, geom, B, I_meas, loss, I_model, g_amp, g_phase, g_probe, g_pos, g_tilt, g_dz, accumulate);
}

int pty_loss_stats(const pty_geom* geom, int B, const int32_t* idx, const float* amp, const float* phase,
                   const float* probe, const float* pos, const float* tilt, const float* dz, const float* I_meas,
                   double* stats, void* ws, size_t ws_bytes, void* stream) {
  Problem pb;
  int rc = prepare(geom, B, MODE_STATS, idx, amp, phase, probe, pos, tilt, dz, ws, ws_bytes, stream, &pb);
  if (rc) return rc;
  REQUIRE(B == 0 || I_meas, "I_meas is NULL");
  REQUIRE(stats && aligned(stats, 8), "stats is NULL or not 8-byte aligned");
  pb.I_meas = I_meas;
  pb.stats_out = stats;
  return dispatch(pb);
}

int pty_loss_grad_part(const pty_geom* geom, int B, const int32_t* idx, const float* amp, const float* phase,
                       const float* probe, const float* pos, const float* tilt, const float* dz, const float* I_meas,
                       const double* whole_stats, double* loss, float* I_model, float* g_amp, float* g_phase,
                       float* g_probe, float* g_pos, float* g_tilt, float* g_dz, int accumulate, void* ws,
                       size_t ws_bytes, void* stream) {
  int rc = validate_geom(geom);
  if (rc) return rc;
  REQUIRE(whole_stats && aligned(whole_stats, 8), "whole_stats is NULL or not 8-byte aligned");
  REQUIRE(geom->w_pacbed == 0.f && geom->w_sparse == 0.f,
          "the PACBED and sparsity terms compare or average over the whole batch at once; a batch split into "
          "parts supports the likelihood terms (Eq. 5 / 6) only");
  Problem pb;
  rc = prepare(geom, B, MODE_GRAD, idx, amp, phase, probe, pos, tilt, dz, ws, ws_bytes, stream, &pb);
  if (rc) return rc;
  pb.whole = whole_stats;
  return grad_call(pb, geom, B, I_meas, loss, I_model, g_amp, g_phase, g_probe, g_pos, g_tilt, g_dz, accumulate);
}

int pty_forward_save(const pty_geom* geom, int B, const int32_t* idx, const float* amp, const float* phase,
                     const float* probe, const float* pos, const float* tilt, const float* dz, float* I_model,
                     void* ws, size_t ws_bytes, void* stream) {
  Problem pb;
  int rc = prepare(geom, B, MODE_FORWARD_SAVE, idx, amp, phase, probe, pos, tilt, dz, ws, ws_bytes, stream, &pb);
  if (rc) return rc;
  REQUIRE(B == 0 || I_model, "I_model is NULL");
  pb.I_model = I_model;
  return dispatch(pb);
}

int pty_backward(const pty_geom* geom, int B, const int32_t* idx, const float* amp, const float* phase,
                 const float* probe, const float* pos, const float* tilt, const float* dz, const float* dL_dI,
                 float* g_amp, float* g_phase, float* g_probe, float* g_pos, float* g_tilt, float* g_dz,
                 int accumulate, void* ws, size_t ws_bytes, void* stream) {
  Problem pb;
  int rc = prepare(geom, B, MODE_BACKWARD, idx, amp, phase, probe, pos, tilt, dz, ws, ws_bytes, stream, &pb);
  if (rc) return rc;
  const int gm = geom->grad_mask;
  REQUIRE(B == 0 || dL_dI, "dL_dI is NULL");
  REQUIRE(!(gm & PTY_GRAD_AMP) || g_amp, "g_amp is NULL but PTY_GRAD_AMP is requested");
  REQUIRE(!(gm & PTY_GRAD_PHASE) || g_phase, "g_phase is NULL but PTY_GRAD_PHASE is requested");
  REQUIRE(!(gm & PTY_GRAD_PROBE) || (g_probe && aligned(g_probe, 8)), "g_probe is NULL or misaligned");
  REQUIRE(!(gm & PTY_GRAD_POS) || g_pos, "g_pos is NULL but PTY_GRAD_POS is requested");
  REQUIRE(!(gm & PTY_GRAD_TILT) || g_tilt, "g_tilt is NULL but PTY_GRAD_TILT is requested");
  REQUIRE(!(gm & PTY_GRAD_DZ) || g_dz, "g_dz is NULL but PTY_GRAD_DZ is requested");
  pb.dldi = dL_dI;
  pb.g_amp = g_amp;
  pb.g_phase = g_phase;
  pb.g_probe = reinterpret_cast<float2*>(g_probe);
  pb.g_pos = g_pos;
  pb.g_tilt = g_tilt;
  pb.g_dz = g_dz;
  pb.accumulate = accumulate ? 1 : 0;
  return dispatch(pb);
}

int pty_adam_update(const pty_geom* geom, float* amp, float* phase, float* probe, float* pos, float* tilt,
                    float* dz, const float* g_amp, const float* g_phase, const float* g_probe, const float* g_pos,
                    const float* g_tilt, const float* g_dz, const pty_adam* adam, int step, void* stream) {
  int rc = validate_geom(geom);
  if (rc) return rc;
  REQUIRE(adam, "adam state is NULL");
  REQUIRE(step >= 1, "Adam step count must be >= 1");
  const size_t nobj = (size_t)(geom->obj_modes > 1 ? geom->obj_modes : 1) * geom->Nz * geom->H * geom->W;
  const size_t nprobe = 2 * (size_t)geom->M * geom->N * geom->N;
  const size_t ntilt = geom->global_tilt ? 2 : 2 * (size_t)geom->Ntot;
  AdamArgs a;
  memset(&a, 0, sizeof(a));
  const int gm = geom->grad_mask;
  struct {
    int bit;
    float* p;
    const float* g;
    float *m, *v;
    size_t n;
    float lr;
    const char* name;
  } c[6] = {
      {PTY_GRAD_AMP, amp, g_amp, adam->m_amp, adam->v_amp, nobj, adam->lr_amp, "amp"},
      {PTY_GRAD_PHASE, phase, g_phase, adam->m_phase, adam->v_phase, nobj, adam->lr_phase, "phase"},
      {PTY_GRAD_PROBE, probe, g_probe, adam->m_probe, adam->v_probe, nprobe, adam->lr_probe, "probe"},
      {PTY_GRAD_POS, pos, g_pos, adam->m_pos, adam->v_pos, 2 * (size_t)geom->Ntot, adam->lr_pos, "pos"},
      {PTY_GRAD_TILT, tilt, g_tilt, adam->m_tilt, adam->v_tilt, ntilt, adam->lr_tilt, "tilt"},
      {PTY_GRAD_DZ, dz, g_dz, adam->m_dz, adam->v_dz, 1, adam->lr_dz, "dz"},
  };
  for (int k = 0; k < 6; ++k) {
    if (!(gm & c[k].bit) || !(c[k].lr > 0.f)) continue;
    REQUIRE(c[k].p && c[k].g && c[k].m && c[k].v, "Adam for %s needs parameter, gradient and both moments", c[k].name);
    a.seg[a.nseg++] = AdamSeg{c[k].p, c[k].g, c[k].m, c[k].v, c[k].n, c[k].lr};
  }
  if (a.nseg == 0) return PTY_OK;
  a.beta1 = adam->beta1;
  a.beta2 = adam->beta2;
  a.eps = adam->eps;
  a.bc1 = (float)(1.0 - pow((double)adam->beta1, step));
  a.bc2 = (float)(1.0 - pow((double)adam->beta2, step));
  k_adam<<<152 * 8, 256, 0, (cudaStream_t)stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("k_adam launch failed: %s", cudaGetErrorString(e));
    return PTY_ECUDA;
  }
  note_launch();
  return PTY_OK;
}

int pty_step(const pty_geom* geom, int B, const int32_t* idx, float* amp, float* phase, float* probe, float* pos,
             float* tilt, float* dz, const float* I_meas, double* loss, float* g_amp, float* g_phase, float* g_probe,
             float* g_pos, float* g_tilt, float* g_dz, const pty_adam* adam, int step, void* ws, size_t ws_bytes,
             void* stream) {
  int rc = pty_loss_grad(geom, B, idx, amp, phase, probe, pos, tilt, dz, I_meas, loss, nullptr, g_amp, g_phase,
                         g_probe, g_pos, g_tilt, g_dz, 0, ws, ws_bytes, stream);
  if (rc) return rc;
  return pty_adam_update(geom, amp, phase, probe, pos, tilt, dz, g_amp, g_phase, g_probe, g_pos, g_tilt, g_dz, adam,
                         step, stream);
}

int pty_status(const void* ws, void* stream) {
  if (!ws) return -1;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    set_error("stream synchronisation failed: %s", cudaGetErrorString(cudaGetLastError()));
    return -1;
  }
  int v = 0;
  if (cudaMemcpy(&v, ws, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    set_error("status read failed: %s", cudaGetErrorString(cudaGetLastError()));
    return -1;
  }
  return v;
}

const char* pty_last_error(void) { return g_err; }

int pty_supported_sizes(void) { return (1 << 6) | (1 << 7) | (1 << 8); }

// ---------------------------------------------------------------------------------------------
// pty_loss_grad_noalloc: the same pass, with its scratch in a fixed device array of this library.
// ---------------------------------------------------------------------------------------------
}  // extern "C"

namespace {
constexpr size_t kNoallocBytes = (size_t)PTY_NOALLOC_SCRATCH_BYTES;
// Loaded with the library's device code on every GPU that uses it and held until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];
// Device address of g_noalloc_scratch per device ordinal (host code may not use the symbol itself).
// Filled without a lock: two host threads making their first call on a device at once both look
// the address up and store the same value, which is harmless.  cudaDeviceReset would make a cached
// address stale; the library does not support a reset between calls.
void* g_noalloc_addr[256] = {nullptr};
}  // namespace

extern "C" {

int pty_loss_grad_noalloc(const pty_geom* geom, int B, const int32_t* idx, const float* amp, const float* phase,
                          const float* probe, const float* pos, const float* tilt, const float* dz,
                          const float* I_meas, double* loss, float* I_model, float* g_amp, float* g_phase,
                          float* g_probe, float* g_pos, float* g_tilt, float* g_dz, int accumulate, int* status,
                          void* stream) {
  int rc = validate_geom(geom);
  if (rc) return rc;
  REQUIRE(B >= 0, "batch size %d < 0", B);
  const size_t need = layout_workspace(*geom, B, MODE_GRAD, nullptr, nullptr);
  if (need > kNoallocBytes) {
    const size_t empty = layout_workspace(*geom, 0, MODE_GRAD, nullptr, nullptr);
    if (empty > kNoallocBytes)
      set_error("pty_loss_grad_noalloc: the object alone needs %zu bytes of scratch (transmission and its "
                "gradient) but the fixed area holds %zu; no batch fits; use pty_loss_grad with a caller-owned "
                "workspace", empty, kNoallocBytes);
    else
      set_error("pty_loss_grad_noalloc: this batch needs %zu bytes of scratch but the fixed area holds %zu; "
                "use a smaller batch or pty_loss_grad with a caller-owned workspace", need, kNoallocBytes);
    return PTY_EWORKSPACE;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    set_error("pty_loss_grad_noalloc: no current CUDA device");
    return PTY_ECUDA;
  }
  if (!g_noalloc_addr[dev]) {  // first call on this device: look up the array's device address
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("pty_loss_grad_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return PTY_ECUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  void* ws = g_noalloc_addr[dev];
  rc = pty_loss_grad(geom, B, idx, amp, phase, probe, pos, tilt, dz, I_meas, loss, I_model, g_amp, g_phase, g_probe,
                     g_pos, g_tilt, g_dz, accumulate, ws, kNoallocBytes, stream);
  if (rc == PTY_OK && status) {
    if (cudaMemcpyAsync(status, ws, sizeof(int), cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess) {
      set_error("pty_loss_grad_noalloc: status copy failed: %s", cudaGetErrorString(cudaGetLastError()));
      return PTY_ECUDA;
    }
  }
  return rc;
}

long long pty_launch_count(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int pty_fma_probe(float* sink, int blocks, int iters, void* stream) {
  REQUIRE(sink && blocks > 0 && iters > 0, "pty_fma_probe: sink NULL or blocks / iters <= 0");
  k_fma_probe<<<blocks, 512, 0, (cudaStream_t)stream>>>(sink, iters);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("k_fma_probe launch failed: %s", cudaGetErrorString(e));
    return PTY_ECUDA;
  }
  note_launch();
  return PTY_OK;
}

int pty_set_wait_limit(long long polls) {
  g_stage_spin = polls < 0 ? -1 : (long)(polls < PTY_WAIT_POLLS_DEFAULT ? polls : PTY_WAIT_POLLS_DEFAULT);
  return PTY_OK;
}

int pty_profile_enable(int on) {
  if (on && !g_prof_created) {
    for (int c = 0; c < kProfCalls; ++c)
      for (int k = 0; k <= PTY_PROF_STAGES; ++k)
        if (cudaEventCreate(&g_prof_ev[c][k]) != cudaSuccess) {
          set_error("cudaEventCreate failed");
          return PTY_ECUDA;
        }
    g_prof_created = true;
  }
  g_prof_on = on != 0;
  g_prof_calls = 0;
  return PTY_OK;
}

int pty_profile_read(double* ms, int n) {
  const int m = n < PTY_PROF_STAGES ? n : PTY_PROF_STAGES;
  for (int k = 0; k < m; ++k) ms[k] = 0.0;
  for (int c = 0; c < g_prof_calls; ++c) {
    int prev = 0;  // time from the previous recorded mark to this stage's mark
    for (int k = 1; k <= PTY_PROF_STAGES; ++k) {
      if (!g_prof_have[c][k]) continue;
      if (cudaEventSynchronize(g_prof_ev[c][k]) != cudaSuccess) return -1;
      float t = 0.f;
      if (cudaEventElapsedTime(&t, g_prof_ev[c][prev], g_prof_ev[c][k]) != cudaSuccess) return -1;
      if (k - 1 < m) ms[k - 1] += t;
      prev = k;
    }
  }
  return g_prof_calls;
}

}  // extern "C"
