// pipeline.cuh -- kernels of the batched multislice forward model, loss and adjoint, templated on
// the window size N.  One CTA owns one (scan position, probe mode) wavefield for the whole slice
// loop; the wave never leaves shared memory except as checkpoints for the adjoint.
//
// Kernel sequence of one pty_loss_grad call (one stream, no host synchronisation):
//   k_prepare_object   T = amp exp(i phase) for the whole object; zero dL/dT accumulator
//   k_probe_spectrum   P^_m = F[P_m]                                              (M CTAs)
//   k_forward          shift, Nz transmissions, Nz-1 propagations, far field      (B*M CTAs)
//   k_loss             mode sum, Eq. 5/6 per pixel, dL/dI, per-pattern sums      (B CTAs)
//   k_loss_finalize    batch loss and dL/dI normaliser (FP64)                      (1 CTA)
//   k_adjoint          reverse of k_forward, scatter-adds dL/dT, probe-spectrum
//                      gradient, FP64-reduced position / tilt / dz partials       (B*M CTAs)
//   k_object_grad      dL/damp, dL/dphase from dL/dT (chain rule of amp exp(i phase))
//   k_probe_grad       dL/dP_m = F^-1[accumulated spectrum gradient]              (M CTAs)
//   k_scalar_grad      positions, tilts, dz from the per-wave partials
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "fft_cluster.cuh"
#include "fft_smem.cuh"
#include "pty_internal.h"

#ifndef PTY_TF128
#define PTY_TF128 256
#endif
#ifndef PTY_TA128
#define PTY_TA128 512
#endif
#ifndef PTY_ADJ_SPLIT_COL
#define PTY_ADJ_SPLIT_COL 1
#endif
#ifndef PTY_ADJ_BATCH
#define PTY_ADJ_BATCH 8
#endif
// the same for the N = 256 adjoint's pointwise passes (large-window adjoint: 43.95 ms at 8, 42.98 at 16,
// 43.74 at 32)
#ifndef PTY_ADJ256_BATCH
#define PTY_ADJ256_BATCH 16
#endif
// Order in which the adjoint's CTAs take the waves: 0 position-major (the modes of one position run
// side by side and scatter-add into the same dL/dT addresses), G > 0 groups of G positions with the
// modes outermost inside a group (waves running side by side then belong to different positions).
// Large-window adjoint: 42.70 ms at 0, 42.42 at 4, 42.38 at 32, 42.40 with every mode outermost.
#ifndef PTY_ADJ_GROUP
#define PTY_ADJ_GROUP 32
#endif
// The propagation step inside the row transform (0) reads each task's 32 spectrum values in one
// batch (PTY_KQ = 32): multislice adjoint 3.274 ms against 3.455 as its own pass (1)
#ifndef PTY_ADJ_SPLIT_ROW
#define PTY_ADJ_SPLIT_ROW 0
#endif
// The same two choices for the N = 256 cluster adjoint.  Its column step is the cross-CTA step, so
// a separate transmission pass costs a second pass through distributed shared memory per slice
// (large-window workload: adjoint 63.5 ms split, 46.8 ms fused).  The propagation step fused into
// the row transform with each task's 16 spectrum loads in one batch: 39.98 ms against 42.41 as its
// own pass (with batches of 4 the fused form was the slower one, 44.17 ms).
#ifndef PTY_ADJ256_SPLIT_COL
#define PTY_ADJ256_SPLIT_COL 0
#endif
#ifndef PTY_ADJ256_SPLIT_ROW
#define PTY_ADJ256_SPLIT_ROW 0
#endif
#ifndef PTY_FWD_SPLIT_COL
#define PTY_FWD_SPLIT_COL 0
#endif
// 1: the N = 128 forward and adjoint ask for the smallest shared-memory carve-out that holds their
// CTA (cudaFuncAttributePreferredSharedMemoryCarveout), leaving the rest of the SM's memory as L1
#ifndef PTY_CARVEOUT
#define PTY_CARVEOUT 1
#endif
// Adjoint L2 prefetch plan (cp.async.bulk.prefetch.L2 of whole 128 KB blocks).  0: at the start of
// slice s, the checkpoint of slice s - 1 and the spectrum of the next slice's propagation.  1: at
// the start of slice s the spectrum its own propagation reads, after its transmission step the
// checkpoint the next slice reads.  2: only before the slice loop.  3: none.  Measured on the
// multislice workload (N = 128, M = 6, Nz = 8, 512 positions): adjoint 4.13 / 4.07 / 3.74 / 3.69
// ms; the bulk prefetches cost more than the load latency they hide, so none is the default.
#ifndef PTY_ADJ_PF
#define PTY_ADJ_PF 3
#endif
// 1: the forward prefetches the next slice's transmission patch to L2 (measured: 2.496 ms with,
// 2.490 ms without on the same workload)
#ifndef PTY_FWD_PF
#define PTY_FWD_PF 0
#endif
// 1: the N = 256 adjoint prefetches to L2, at the start of each slice, its CTA's part of the next
// slice's transmission patch, checkpoint and spectrum (the large-window object does not fit L2)
#ifndef PTY_ADJ256_PF
#define PTY_ADJ256_PF 0
#endif
// Adjoint L1 prefetch: > 0 prefetches the first PTY_ADJ_L1PF KB of each checkpoint and spectrum
// block into L1 (prefetch.global.L1, one 128-byte line per thread) two transform steps before the
// pass that reads it, so that those loads hit the SM's own cache; 0: off.
#ifndef PTY_ADJ_L1PF
#define PTY_ADJ_L1PF 0
#endif
// 1: the adjoint reads checkpoints and spectra with evict-first (streaming) loads, so they do not
// displace the transmission and its gradient accumulator from L2 (adjoint 3.685 -> 3.655 ms)
#ifndef PTY_ADJ_LDCS
#define PTY_ADJ_LDCS 1
#endif
#ifndef PTY_KS
#define PTY_KS 4
#endif
#ifndef PTY_KT
#define PTY_KT 4
#endif
#ifndef PTY_KP
#define PTY_KP 4
#endif
#ifndef PTY_KF
#define PTY_KF 4
#endif
#ifndef PTY_KG
#define PTY_KG 4
#endif
// (the adjoint's checkpoint and transmission reads in the fused column step; large-window adjoint
// 39.8 ms at 4, 41.5 at 8 and 45.0 at 16 even with the transmission read 4 at a time)
#ifndef PTY_KA
#define PTY_KA 4
#endif
// (the adjoint's spectrum reads in the fused propagation step; capped at a task's elements)
#ifndef PTY_KQ
#define PTY_KQ 32
#endif
#ifndef PTY_KR
#define PTY_KR 4
#endif

namespace pty {

template <int N>
struct Launch;
// Threads per CTA of the forward (TF) and adjoint (TA) kernels and of the small kernels (T), with the
// CTAs per SM the register budget is sized for.  At N = 128 one wave (132 KB) fills the SM's shared
// memory: the forward runs 256 threads with up to 255 registers each, the adjoint 512 threads so
// that more of its checkpoint / transmission loads are in flight.
template <>
struct Launch<64> {
  static constexpr int T = 256, TF = 128, TA = 128, MINB_F = 4, MINB_A = 4;
};
template <>
struct Launch<128> {
  static constexpr int T = 512, TF = PTY_TF128, TA = PTY_TA128, MINB_F = 1, MINB_A = 1;
};
// N = 256: every wave kernel runs as clusters of PTY_N256_CTAS CTAs (fft_cluster.cuh): four CTAs
// of 512 threads (one per SM), or eight of 128 threads (three per SM, from different clusters).
// PTY_TF256 / PTY_TA256 (0: the CTA size) give the forward / adjoint other thread counts with four
// CTAs per wave.  Large-window workload at 256 threads (up to 255 registers): forward 33.86 ms
// against 31.28, adjoint 49.79 against 39.97 (42.79 with checkpoint loads in batches of 16).
#ifndef PTY_TF256
#define PTY_TF256 0
#endif
#ifndef PTY_TA256
#define PTY_TA256 0
#endif
template <>
struct Launch<256> {
  static constexpr int T = PTY_N256_CTAS == 8 ? 128 : 512;
  static constexpr int TF = PTY_TF256 ? PTY_TF256 : T, TA = PTY_TA256 ? PTY_TA256 : T;
  static constexpr int MINB_F = PTY_N256_CTAS == 8 ? 3 : 1, MINB_A = MINB_F;
};

// Rows of a wave one CTA holds in shared memory (1 / PTY_N256_CTAS of the wave at N = 256).
template <int N>
__host__ __device__ constexpr int wave_rows() {
  return N == 256 ? 256 / PTY_N256_CTAS : N;
}

// exp(i pi x); x is reduced modulo 2 in double precision before the float sincospi.
__device__ __forceinline__ float2 expipi(double x) {
  x = x - 2.0 * rint(0.5 * x);
  float s, c;
  sincospif((float)x, &s, &c);
  return make_float2(c, s);
}

// Signed DFT frequency index of bin k.
template <int N>
__device__ __forceinline__ int signed_bin(int k) {
  return k < N / 2 ? k : k - N;
}

// Patch corner round(pos) (half to even) and sub-pixel remainder; clamps and flags if outside.
template <int N>
__device__ __forceinline__ void patch_corner(const float* pos, int j, int H, int W, int* i0, int* i1,
                                             float* d0, float* d1, int* status) {
  const float p0 = pos[2 * j], p1 = pos[2 * j + 1];
  float r0 = rintf(p0), r1 = rintf(p1);
  *d0 = p0 - r0;
  *d1 = p1 - r1;
  const bool fin = isfinite(p0) && isfinite(p1);
  const bool ok = fin && r0 >= 0.f && r1 >= 0.f && r0 + N <= (float)H && r1 + N <= (float)W;
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(status, PTY_EBOUNDS);
    if (!fin) {
      r0 = 0.f;
      r1 = 0.f;
      *d0 = 0.f;
      *d1 = 0.f;
    }
    r0 = fminf(fmaxf(r0, 0.f), (float)(H - N));
    r1 = fminf(fmaxf(r1, 0.f), (float)(W - N));
  }
  *i0 = (int)r0;
  *i1 = (int)r1;
}

// Batch entry b's scan index; an index outside [0, Ntot) is flagged and replaced by 0.
__device__ __forceinline__ int checked_index(const int32_t* idx, int b, int Ntot, int* status) {
  int j = idx[b];
  if (j < 0 || j >= Ntot) {
    if (threadIdx.x == 0) atomicOr(status, PTY_EBOUNDS);
    j = 0;
  }
  return j;
}

__device__ __forceinline__ void tilt_of(const float* tilt, int global_tilt, int j, float* t0, float* t1) {
  const float* t = global_tilt ? tilt : tilt + 2 * j;
  *t0 = t[0];
  *t1 = t[1];
}

// ---------------------------------------------------------------------------------------------
// Object transmission and accumulator reset
// ---------------------------------------------------------------------------------------------
static __global__ void k_prepare_object(const float* __restrict__ amp, const float* __restrict__ phase,
                                 float2* __restrict__ T, float2* __restrict__ gT, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float s, c;
    sincosf(phase[i], &s, &c);
    const float a = amp[i];
    T[i] = make_float2(a * c, a * s);
    if (gT) gT[i] = make_float2(0.f, 0.f);
  }
}

// ---------------------------------------------------------------------------------------------
// Probe spectra P^_m = F[P_m] (k-space layout); zero the probe-gradient accumulator.
// ---------------------------------------------------------------------------------------------
template <int N, int T>
__global__ void __launch_bounds__(T) k_probe_spectrum(const float2* __restrict__ probe, float2* __restrict__ Phat,
                                                      float2* __restrict__ gPhat) {
  using F = Fft2<N, T>;
  constexpr int RS = F::RS, R = F::ROWS;
  extern __shared__ __align__(16) float2 sm[];
  float2* s = sm;
  float2* tw = s + R * RS;
  const int m = blockIdx.x / F::C, q = F::rank(), tid = threadIdx.x;
  build_twiddles<N>(tw);
  const float2* P = probe + (size_t)m * N * N + (size_t)q * R * N;  // this CTA's rows of mode m
  for (int e = tid; e < R * N; e += T) s[(e / N) * RS + e % N] = P[e];
  __syncthreads();
  F::forward(s, tw);
  float2* out = Phat + (size_t)m * N * N;
  float2* g = gPhat ? gPhat + (size_t)m * N * N : nullptr;
  for (int e = tid; e < R * N; e += T) {  // local k-space row e % R, column e / R
    const int k = kidx<N>(q * R + e % R, e / R);
    out[k] = s[(e % R) * RS + e / R];
    if (g) g[k] = make_float2(0.f, 0.f);
  }
}

// ---------------------------------------------------------------------------------------------
// Forward: one CTA per (batch entry b, mode m)
// ---------------------------------------------------------------------------------------------
struct FwdArgs {
  int M, Ko, Nz, H, W, Ntot, global_tilt;  // Ko: object modes
  float dx, lam;
  const int32_t* idx;
  const float *pos, *tilt, *dz;
  const float2* T;
  const float2* Phat;
  float2* ckpt;     // every slice's entering wave [wave][Nz][N*N], or nullptr
  float2* vhat;     // every propagated spectrum [wave][Nz-1][N*N], or nullptr
  float2* anchors;  // recompute mode: spectrum entering slice q*K, [wave][nseg-1][N*N], or nullptr
  int kstride;      // recompute mode: slices per segment K (anchors at slices K, 2K, ...)
  float2* Psi;
  float* Imode;
  int* status;
  // segment replay (k_recompute): slices [s0, s1) from the anchor of s0, into per-segment buffers
  int s0, s1;
};

template <int N>
__host__ __device__ constexpr size_t fwd_smem_bytes() {
  return sizeof(float2) * ((size_t)wave_rows<N>() * (N + 1) + 5 * N);
}

// Bulk-copy staging of the forward's transmission patch (N = 128, fused column step, even object
// width): rows 0..N/2-1 of the next slice's patch are copied into shared memory after the wave and
// its tables while the current slice's last three transform steps run, one copy per row by the
// lanes of warp 0.  A row copy starts at the 16-byte boundary at or left of the patch corner: N
// elements, or N + 2 from the column before an odd corner (with W and N even, an odd corner lies
// at most at W - N - 1, so the copy stays inside the row).  Stage rows have a pitch of N + 2.
#ifndef PTY_FWD_STAGE
#define PTY_FWD_STAGE 0
#endif
template <int N>
__host__ __device__ constexpr bool fwd_staged() {
  return PTY_FWD_STAGE && N == 128 && !PTY_FWD_SPLIT_COL;
}
template <int N>
__host__ __device__ constexpr size_t fwd_stage_offset() {
  return (fwd_smem_bytes<N>() + 127) / 128 * 128;
}
template <int N>
__host__ __device__ constexpr size_t fwd_stage_bytes() {
  return (size_t)(N / 2) * (N + 2) * sizeof(float2);
}
// Dynamic shared memory of k_forward (k_recompute takes fwd_smem_bytes).
template <int N>
__host__ __device__ constexpr size_t fwd_kernel_smem_bytes() {
  return fwd_staged<N>() ? fwd_stage_offset<N>() + fwd_stage_bytes<N>() + 16 : fwd_smem_bytes<N>();
}
template <int N>
__device__ __forceinline__ float2* fwd_stage() {
  extern __shared__ __align__(16) float2 sm[];
  return reinterpret_cast<float2*>(reinterpret_cast<char*>(sm) + fwd_stage_offset<N>());
}

// Loads of data written by earlier kernels and read-only here (checkpoints, spectra, transmission):
// non-coherent and not volatile, so the compiler may batch them ahead of this thread's atomics.
__device__ __forceinline__ float2 ld_ro(const float2* p) {
  float2 v;
  asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_ro(const float4* p) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_ro(const float* p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

// Checkpoints and spectra the adjoint reads exactly once
__device__ __forceinline__ float2 ld_once(const float2* p) {
#if PTY_ADJ_LDCS
  return __ldcs(p);
#else
  return ld_ro(p);
#endif
}

// L2 prefetch of a byte range (rounded out to 16-byte boundaries).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  const uintptr_t a = (uintptr_t)p & ~(uintptr_t)15;
  const uintptr_t e = ((uintptr_t)p + bytes + 15) & ~(uintptr_t)15;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a)) : "memory");
}
// L1 prefetch of the first `bytes` of a block, one 128-byte line per thread and pass.
__device__ __forceinline__ void prefetch_l1(const void* base, int bytes) {
  for (int l = threadIdx.x * 128; l < bytes; l += blockDim.x * 128)
    asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<const char*>(base) + l));
}
// Rows [0, N) of an N-wide patch with row stride W (elements), one row per thread and pass.  With
// C > 1 CTAs per wave, CTA `rank` takes its own N / C columns of every row (the columns its
// cross-CTA step reads).
template <int N, int C = 1>
__device__ __forceinline__ void prefetch_patch(const float2* base, int W, int rank = 0) {
  for (int r = threadIdx.x; r < N; r += blockDim.x)
    prefetch_l2(base + (size_t)r * W + rank * (N / C), sizeof(float2) * (N / C));
}
// A contiguous N*N block, split over the first 8 threads.
template <int N>
__device__ __forceinline__ void prefetch_block(const float2* base) {
  constexpr size_t chunk = sizeof(float2) * N * N / 8;
  if (threadIdx.x < 8) prefetch_l2(reinterpret_cast<const char*>(base) + threadIdx.x * chunk, chunk);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// L2 policy for data read once: evict first.
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// Arrive on the mbarrier `bar` and add `bytes` to the transaction count its phase waits for.
__device__ __forceinline__ void stage_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Copy `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to shared memory,
// completing on `bar`.  Earlier generic-proxy accesses of dst by this thread (and, through a
// barrier, by the CTA) are ordered before the copy by the proxy fence.
__device__ __forceinline__ void stage_copy(uint32_t bar, void* dst, const void* src, uint32_t bytes, uint64_t pol) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(bar), "l"(pol)
      : "memory");
}
// One thread: one copy of `bytes` that alone completes the barrier's current phase.
__device__ __forceinline__ void stage_issue(uint32_t bar, void* dst, const void* src, uint32_t bytes) {
  const uint64_t pol = evict_first_policy();
  stage_expect(bar, bytes);
  stage_copy(bar, dst, src, bytes, pol);
}
constexpr long kStageSpin = 1L << 24;  // non-blocking polls before a stage wait gives up (well under a second)
// Bounded wait for phase `parity` of `bar`; false on timeout.
__device__ __forceinline__ bool stage_wait(uint32_t bar, uint32_t parity) {
  for (long i = 0; i < kStageSpin; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Per-wave tables, written by the first N threads (axis-0 tables indexed by k-space row p0, axis-1
// tables by k-space column p1).  Forward: shift ramps R (axis 0 carries the 1/N^2 of the inverse
// DFT) and the two factors of Eq. 4's propagator (axis 0 carries 1/N^2).
template <int N>
__device__ void fwd_tables(float2* ra0, float2* ra1, float2* pm0, float2* pm1, float d0, float d1, float th0, float th1,
                           float dz, float dx, float lam) {
  for (int tid = threadIdx.x; tid < N; tid += blockDim.x) {
    const int q0 = signed_bin<N>(kbin0<N>(tid)), q1 = signed_bin<N>(kbin1<N>(tid));
    const float inv_nn = 1.0f / (float)(N * N);
    ra0[tid] = cscale(expipi(-2.0 * q0 * (double)d0 / N), inv_nn);
    ra1[tid] = expipi(-2.0 * q1 * (double)d1 / N);
    // Eq. 4 split into its two axes: exp(i pi (-lam dz k_a^2 + 2 dz k_a tan th_a))
    const double k0 = q0 / (N * (double)dx), k1 = q1 / (N * (double)dx);
    pm0[tid] = cscale(expipi(-(double)lam * dz * k0 * k0 + 2.0 * dz * k0 * tan((double)th0)), inv_nn);
    pm1[tid] = expipi(-(double)lam * dz * k1 * k1 + 2.0 * dz * k1 * tan((double)th1));
  }
}
// Adjoint: conjugate propagator factors (axis 0 with 1/N^2), conjugate shift ramps, and the real
// factors of the dz, tilt and position terms (signs and 2 pi / N^2 folded in).
template <int N>
__device__ void adj_tables(float2* cm0, float2* cm1, float2* cr0, float2* cr1, float* e0, float* e1, float* c0,
                           float* c1, float* f0, float* f1, float d0, float d1, float th0, float th1, float dz,
                           float dx, float lam) {
  constexpr int NN = N * N;
  for (int tid = threadIdx.x; tid < N; tid += blockDim.x) {
    // axis-0 tables are indexed by k-space row p0, axis-1 tables by k-space column p1
    const int q0 = signed_bin<N>(kbin0<N>(tid)), q1 = signed_bin<N>(kbin1<N>(tid));
    const float inv_nn = 1.0f / (float)NN;
    const double k0 = q0 / (N * (double)dx), k1 = q1 / (N * (double)dx);
    const double tn0 = tan((double)th0), tn1 = tan((double)th1);
    cm0[tid] = cscale(cconj(expipi(-(double)lam * dz * k0 * k0 + 2.0 * dz * k0 * tn0)), inv_nn);
    cm1[tid] = cconj(expipi(-(double)lam * dz * k1 * k1 + 2.0 * dz * k1 * tn1));
    cr0[tid] = expipi(2.0 * q0 * (double)d0 / N);
    cr1[tid] = expipi(2.0 * q1 * (double)d1 / N);
    const double PI = 3.14159265358979323846;
    const double cs0 = cos((double)th0), cs1 = cos((double)th1);
    e0[tid] = (float)(PI * lam * k0 * k0 - 2.0 * PI * k0 * tn0);
    e1[tid] = (float)(PI * lam * k1 * k1 - 2.0 * PI * k1 * tn1);
    c0[tid] = (float)(-2.0 * PI * dz * k0 / (cs0 * cs0));
    c1[tid] = (float)(-2.0 * PI * dz * k1 / (cs1 * cs1));
    f0[tid] = (float)(2.0 * PI * q0 / ((double)N * NN));
    f1[tid] = (float)(2.0 * PI * q1 / ((double)N * NN));
  }
}

// ---- forward hooks (see NoHook for the calling convention).  Natural-layout hooks run in the
// col step (lanes own consecutive columns); k-space hooks run in the row step (lanes own
// consecutive k-space rows p0, so global k-space buffers are indexed p1 * N + p0). ----
// shifted-probe spectrum P^_m R_j (k-space), replaces the shared-memory contents
template <int N>
struct ShiftLoad {
  static constexpr bool kReplaces = true;
  static constexpr bool kPreload = false;  // may run in a step that has read two tasks
  static constexpr int kChunk = PTY_KS;
  const float2* Ph;
  const float2 *ra0, *ra1;
  template <int K>
  __device__ __forceinline__ void operator()(int r0, int rs, int c0, int cs, float2* v) {
    float2 p[K];
#pragma unroll
    for (int k = 0; k < K; ++k) p[k] = ld_ro(Ph + kidx<N>(r0 + k * rs, c0 + k * cs));
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = cmul(cmul(p[k], ra0[r0 + k * rs]), ra1[c0 + k * cs]);
  }
};
// transmission of slice s: checkpoint the entering wave, then multiply by T (natural layout)
template <int N>
struct TransLoad {
  static constexpr bool kReplaces = false;
  static constexpr bool kPreload = true;  // may run in a step that has read two tasks
  static constexpr int kChunk = PTY_KT;
  const float2* Ts;  // patch corner in T
  int W;
  float2* ck;    // checkpoint block or nullptr
  int odd = -1;  // >= 0: rows 0..N/2-1 of the patch are staged (fwd_stage), column c at c + odd
  template <int K>
  __device__ __forceinline__ void operator()(int r0, int rs, int c0, int cs, float2* v) {
    float2 t[K];
    const bool staged = odd >= 0 && r0 + (K - 1) * rs < N / 2;
    const float2* st = fwd_stage<N>();
#pragma unroll
    for (int k = 0; k < K; ++k)
      t[k] = staged ? st[(r0 + k * rs) * (N + 2) + c0 + k * cs + odd]
                    : ld_ro(Ts + (size_t)(r0 + k * rs) * W + c0 + k * cs);
    if (ck) {
#pragma unroll
      for (int k = 0; k < K; ++k) __stcs(ck + (r0 + k * rs) * N + c0 + k * cs, v[k]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = cmul(v[k], t[k]);
  }
};
// propagator of Eq. 4 (with 1/N^2 of the following inverse DFT), k-space; optionally stored
template <int N>
struct PropStore {
  static constexpr bool kReplaces = false;
  static constexpr bool kPreload = true;  // may run in a step that has read two tasks
  static constexpr int kChunk = PTY_KP;
  const float2 *m0, *m1;
  float2* vh;
  template <int K>
  __device__ __forceinline__ void operator()(int r0, int rs, int c0, int cs, float2* v) {
    if (rs == 0) {  // a chunk of one k-space row (every caller): its axis-0 factor is read once
      const float2 f0 = m0[r0];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int c = c0 + k * cs;
        v[k] = cmul(cmul(v[k], f0), m1[c]);
        if (vh) __stcs(vh + kidx<N>(r0, c), v[k]);
      }
      return;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int r = r0 + k * rs, c = c0 + k * cs;
      v[k] = cmul(cmul(v[k], m0[r]), m1[c]);
      if (vh) __stcs(vh + kidx<N>(r, c), v[k]);
    }
  }
};
// far field: orthonormal scale, store Psi (for the adjoint) and the mode's intensity
template <int N>
struct FarStore {
  static constexpr bool kReplaces = false;
  static constexpr bool kPreload = true;  // may run in a step that has read two tasks
  static constexpr int kChunk = PTY_KF;
  float2* Psi;
  float* Im;
  template <int K>
  __device__ __forceinline__ void operator()(int r0, int rs, int c0, int cs, float2* v) {
    const float inv_n = 1.0f / (float)N;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int e = kidx<N>(r0 + k * rs, c0 + k * cs);
      const float2 x = cscale(v[k], inv_n);
      if (Psi) __stcs(Psi + e, x);
      Im[e] = fmaf(x.x, x.x, x.y * x.y);
    }
  }
};

// OM: object modes (a.Ko > 1).  The single-mode instantiation folds Ko = 1, so its code is that of a
// plain (position, probe mode) kernel.
template <int N, int T, bool OM = false>
__global__ void __launch_bounds__(T, Launch<N>::MINB_F) k_forward(FwdArgs a) {
  using F = Fft2<N, T>;
  constexpr int RS = F::RS;
  constexpr int NN = N * N;
  extern __shared__ __align__(16) float2 sm[];
  float2* s = sm;
  float2* tw = s + F::ROWS * RS;
  float2* ra0 = tw + N;   // shift ramp along axis 0, carries 1/N^2 of the inverse DFT
  float2* ra1 = ra0 + N;  // shift ramp along axis 1
  float2* pm0 = ra1 + N;  // propagator factor along axis 0, carries 1/N^2
  float2* pm1 = pm0 + N;  // propagator factor along axis 1
  const int tid = threadIdx.x;
  const int bm = blockIdx.x / F::C;  // wave (position, mode); a cluster of F::C CTAs per wave
  const int Ko = OM ? a.Ko : 1;
  const int b = bm / (a.M * Ko), m = (bm / Ko) % a.M;  // waves: (position, probe mode, object mode)
  const int j = checked_index(a.idx, b, a.Ntot, a.status);
  int i0, i1;
  float d0, d1, th0, th1;
  patch_corner<N>(a.pos, j, a.H, a.W, &i0, &i1, &d0, &d1, a.status);
  tilt_of(a.tilt, a.global_tilt, j, &th0, &th1);
  const float dz = a.dz[0];
  const size_t plane = (size_t)a.H * a.W;
  const float2* Tpatch = a.T + (OM ? (size_t)(bm % Ko) * a.Nz * plane : 0) + (size_t)i0 * a.W + i1;
#if PTY_FWD_PF
  prefetch_patch<N, F::C>(Tpatch, a.W, F::rank());
#endif

  // Staging (fwd_staged): copy k holds slice k's rows, so the k-th wait is on phase parity k & 1;
  // copy k + 1 is issued after the column step that read copy k.  A wait that gives up flags
  // PTY_ETIMEOUT; that thread then reads global memory and tests the barrier no more, and warp 0
  // stops issuing once its lane 0 gave up.
  constexpr bool kStage = fwd_staged<N>() && F::C == 1;
  const bool staged = kStage && (a.W % 2) == 0;
  const int odd = i1 & 1;
  float2* stg = fwd_stage<N>();
  const uint32_t sbar = smem_u32(stg + (N / 2) * (N + 2));
  uint32_t sst = 0;  // bit 0: parity of the next wait; bit 31: a wait of this thread gave up
  auto stage_rows = [&](int sl) {  // warp 0: rows 0..N/2-1 of slice sl's patch
    if (tid < 32 && !(__shfl_sync(0xffffffffu, sst, 0) >> 31)) {
      const uint32_t row_bytes = (uint32_t)((N + 2 * odd) * sizeof(float2));
      const uint64_t pol = evict_first_policy();
      if (tid == 0) stage_expect(sbar, (N / 2) * row_bytes);
      __syncwarp();
      for (int r = tid; r < N / 2; r += 32)
        stage_copy(sbar, stg + r * (N + 2), Tpatch + sl * plane + (size_t)r * a.W - odd, row_bytes, pol);
    }
  };
  if constexpr (kStage) {
    if (staged) {
      if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      }
      if (tid < 32) __syncwarp();
      stage_rows(0);
    }
  }

  build_twiddles<N>(tw);
  fwd_tables<N>(ra0, ra1, pm0, pm1, d0, d1, th0, th1, dz, a.dx, a.lam);
  __syncthreads();

  // Shifted probe P_j = F^-1[P^_m R]: the row and block steps of the inverse here; its column step
  // is fused with the first transmission below.  Every propagation F^-1[M F[T psi]] likewise runs
  // as: fused column step (inverse end, T, checkpoint, forward start), block step, fused row step
  // (forward end, M, inverse start), block step.
  ShiftLoad<N> shift{a.Phat + (size_t)m * NN, ra0, ra1};
  F::row_inv(s, tw, shift);
  F::block_inv(s, tw);
  for (int sl = 0; sl < a.Nz; ++sl) {
#if PTY_FWD_PF
    if (sl + 1 < a.Nz) prefetch_patch<N, F::C>(Tpatch + (sl + 1) * plane, a.W, F::rank());
#endif
    TransLoad<N> trans{Tpatch + sl * plane, a.W, a.ckpt ? a.ckpt + ((size_t)bm * a.Nz + sl) * NN : nullptr};
#if PTY_FWD_SPLIT_COL
    NoHook none;
    F::col_inv(s, tw);
    F::template pointwise<(N == 256 ? PTY_ADJ256_BATCH : PTY_ADJ_BATCH)>(s, trans);
    F::col_fwd(s, tw, none);
#else
    if constexpr (kStage) {
      if (staged && !(sst >> 31)) {
        if (stage_wait(sbar, sst & 1)) {
          sst ^= 1;
          trans.odd = odd;
        } else {
          sst |= 0x80000000u;
          atomicOr(a.status, PTY_ETIMEOUT);
        }
      }
    }
    F::template col_inv_fwd<true>(s, tw, trans);
    if constexpr (kStage) {  // every thread is past the stage: fetch the next slice's rows
      if (staged && sl + 1 < a.Nz) stage_rows(sl + 1);
    }
#endif
    F::block_fwd(s, tw);
    if (sl + 1 < a.Nz) {
      float2* vh = nullptr;
      if (a.vhat) {
        vh = a.vhat + ((size_t)bm * (a.Nz - 1) + sl) * NN;
      } else if (a.anchors && (sl + 1) % a.kstride == 0) {
        const int nanch = (a.Nz + a.kstride - 1) / a.kstride - 1;
        vh = a.anchors + ((size_t)bm * nanch + (sl + 1) / a.kstride - 1) * NN;
      }
      PropStore<N> prop{pm0, pm1, vh};
      F::row_fwd_inv(s, tw, prop);
      F::block_inv(s, tw);
    } else {
      FarStore<N> far{a.Psi ? a.Psi + (size_t)bm * NN : nullptr, a.Imode + (size_t)bm * NN};
      F::template row_fwd<false>(s, far);
    }
  }
  if constexpr (kStage) {  // a copy whose wait gave up may still be in flight: give it time to land
    if (staged && tid == 0 && (sst >> 31)) stage_wait(sbar, sst & 1);
  }
}

// ---------------------------------------------------------------------------------------------
// Segment replay for the recompute mode: one CTA per wave re-runs slices [s0, s1) from the stored
// spectrum entering slice s0 (or from the shifted probe when s0 = 0) and writes the entering waves
// (slot sl - s0) and propagated spectra (slot j holds the spectrum entering slice s0 + j) that the
// adjoint of that segment reads.  The spectrum entering slice s is F[psi_in,s] / N^2, exactly what
// the forward kernel stores as an anchor, so the replay reproduces the forward's values.
// ---------------------------------------------------------------------------------------------
// entering spectrum of the segment (k-space), replaces; also copied into segment slot 0
template <int N>
struct AnchorLoad {
  static constexpr bool kReplaces = true;
  static constexpr bool kPreload = false;  // may run in a step that has read two tasks
  static constexpr int kChunk = PTY_KS;
  const float2* an;
  float2* slot0;  // or nullptr
  template <int K>
  __device__ __forceinline__ void operator()(int r0, int rs, int c0, int cs, float2* v) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = ld_ro(an + kidx<N>(r0 + k * rs, c0 + k * cs));
    if (slot0) {
#pragma unroll
      for (int k = 0; k < K; ++k) __stcs(slot0 + kidx<N>(r0 + k * rs, c0 + k * cs), v[k]);
    }
  }
};
// entering wave of the last slice of a segment (natural layout), stored only
template <int N>
struct CkptStore {
  static constexpr bool kReplaces = false;
  static constexpr bool kPreload = true;  // may run in a step that has read two tasks
  static constexpr int kChunk = 4;
  float2* ck;
  template <int K>
  __device__ __forceinline__ void operator()(int r0, int rs, int c0, int cs, float2* v) {
#pragma unroll
    for (int k = 0; k < K; ++k) __stcs(ck + (r0 + k * rs) * N + c0 + k * cs, v[k]);
  }
};

template <int N, int T, bool OM = false>
__global__ void __launch_bounds__(T, Launch<N>::MINB_F) k_recompute(FwdArgs a) {
  using F = Fft2<N, T>;
  constexpr int RS = F::RS;
  constexpr int NN = N * N;
  extern __shared__ __align__(16) float2 sm[];
  float2* s = sm;
  float2* tw = s + F::ROWS * RS;
  float2* ra0 = tw + N;
  float2* ra1 = ra0 + N;
  float2* pm0 = ra1 + N;
  float2* pm1 = pm0 + N;
  const int bm = blockIdx.x / F::C;  // wave (position, mode); a cluster of F::C CTAs per wave
  const int Ko = OM ? a.Ko : 1;
  const int b = bm / (a.M * Ko), m = (bm / Ko) % a.M;  // waves: (position, probe mode, object mode)
  const int j = checked_index(a.idx, b, a.Ntot, a.status);
  int i0, i1;
  float d0, d1, th0, th1;
  patch_corner<N>(a.pos, j, a.H, a.W, &i0, &i1, &d0, &d1, a.status);
  tilt_of(a.tilt, a.global_tilt, j, &th0, &th1);
  const float dz = a.dz[0];
  const size_t plane = (size_t)a.H * a.W;
  const float2* Tpatch = a.T + (OM ? (size_t)(bm % Ko) * a.Nz * plane : 0) + (size_t)i0 * a.W + i1;
  const int K = a.kstride;
  build_twiddles<N>(tw);
  fwd_tables<N>(ra0, ra1, pm0, pm1, d0, d1, th0, th1, dz, a.dx, a.lam);
  __syncthreads();
  float2* ck_seg = a.ckpt ? a.ckpt + (size_t)bm * K * NN : nullptr;
  float2* vh_seg = a.vhat ? a.vhat + (size_t)bm * K * NN : nullptr;
  if (a.s0 == 0) {
    ShiftLoad<N> shift{a.Phat + (size_t)m * NN, ra0, ra1};
    F::row_inv(s, tw, shift);
  } else {
    const int nanch = (a.Nz + K - 1) / K - 1;
    AnchorLoad<N> anc{a.anchors + ((size_t)bm * nanch + a.s0 / K - 1) * NN, vh_seg};
    F::row_inv(s, tw, anc);
  }
  F::block_inv(s, tw);
  for (int sl = a.s0; sl < a.s1; ++sl) {
    float2* ck = ck_seg ? ck_seg + (size_t)(sl - a.s0) * NN : nullptr;
    if (sl + 1 < a.s1) {
      TransLoad<N> trans{Tpatch + sl * plane, a.W, ck};
      F::template col_inv_fwd<true>(s, tw, trans);
      F::block_fwd(s, tw);
      PropStore<N> prop{pm0, pm1, vh_seg ? vh_seg + (size_t)(sl + 1 - a.s0) * NN : nullptr};
      F::row_fwd_inv(s, tw, prop);
      F::block_inv(s, tw);
    } else if (ck) {
      CkptStore<N> store{ck};
      F::template col_inv_fwd<false>(s, tw, store);
    }
  }
}

// External dL/dI (DC-centred [B][N][N]) into the adjoint's k-space layout; the normaliser becomes 1.
template <int N>
__global__ void k_dldi_to_kspace(const float* __restrict__ dldi, float* __restrict__ u, double* scal, int B) {
  const size_t n = (size_t)B * N * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / (N * N)), q = (int)(i % (N * N));
    const int k0 = (q / N + N / 2) & (N - 1), k1 = (q % N + N / 2) & (N - 1);
    u[(size_t)b * N * N + kpos1<N>(k1) * N + kpos0<N>(k0)] = dldi[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[0] = 1.0;
}

// ---------------------------------------------------------------------------------------------
// Loss: one CTA per pattern.  Sums modes, evaluates Eq. 5 or 6 per pixel and dL/dI up to the
// batch-wide normaliser, and writes FP64 per-pattern sums.
// ---------------------------------------------------------------------------------------------
struct LossArgs {
  int M, Ntot, loss;
  int* status;
  float p, eps;
  const int32_t* idx;
  const float* Imode;
  const float* I_meas;
  float* I_model;
  float* u;
  double* lpart;
  // PACBED term (nullptr when off): batch sums of I_model and I_meas in k-space order, and the
  // per-pattern sums of I_meas^pac_p
  float* pac;
  double* pacpart;
  float pac_p;
};

// x^p for x >= 0 (0 for x <= 0 when p != 1), with the common exponents exact.
__device__ __forceinline__ float pow_nn(float x, float p) {
  if (p == 1.0f) return x;
  if (x <= 0.f) return 0.f;
  return p == 0.5f ? sqrtf(x) : powf(x, p);
}

template <int N>
__host__ __device__ constexpr size_t loss_smem_bytes() {
  return sizeof(float) * (size_t)N * (N + 1) + 64 * sizeof(double);
}

template <int T>
__device__ __forceinline__ void block_sum2(double& x, double& y, double* red) {
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, o);
    y += __shfl_down_sync(0xffffffffu, y, o);
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) {
    red[2 * w] = x;
    red[2 * w + 1] = y;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sx = 0.0, sy = 0.0;
    for (int i = 0; i < T / 32; ++i) {
      sx += red[2 * i];
      sy += red[2 * i + 1];
    }
    x = sx;
    y = sy;
  }
}

// Eq. 5 / 6 at one detector pixel: the summand of the loss (term), the pattern term of its
// normaliser (Dp = I_meas^p) and dL/dI up to the batch-wide normaliser (u).
__device__ __forceinline__ void loss_pixel(float I, float d, float p, float eps, int loss, float* term, float* Dp,
                                           float* u) {
  float Ip, dpow;
  if (p == 1.0f) {
    Ip = I;
    *Dp = d;
    dpow = 1.0f;
  } else if (p == 0.5f) {
    Ip = sqrtf(fmaxf(I, 0.f));
    *Dp = sqrtf(fmaxf(d, 0.f));
    dpow = I > 0.f ? 0.5f / Ip : 0.f;
  } else {
    Ip = powf(fmaxf(I, 0.f), p);
    *Dp = powf(fmaxf(d, 0.f), p);
    dpow = I > 0.f ? p * powf(I, p - 1.0f) : 0.f;
  }
  if (loss == PTY_LOSS_POISSON) {
    *term = *Dp * logf(Ip + eps) - Ip;
    *u = -(*Dp / (Ip + eps) - 1.0f) * dpow;
  } else {
    const float df = Ip - *Dp;
    *term = df * df;
    *u = df * dpow;
  }
}

// PAC: the PACBED sums are on (a.pac != nullptr); the plain instantiation carries none of that work.
template <int N, int T, bool PAC = false>
__global__ void __launch_bounds__(T) k_loss(LossArgs a) {
  constexpr int RS = N + 1;
  constexpr int NN = N * N;
  extern __shared__ __align__(16) float lsm[];
  float* L = lsm;
  double* red = reinterpret_cast<double*>(lsm + N * RS + ((N * RS) & 1));
  const int b = blockIdx.x, tid = threadIdx.x;
  // mode sum, four pixels of one k-space row per thread and load (N is a multiple of 4)
  const float4* Im4 = reinterpret_cast<const float4*>(a.Imode + (size_t)b * a.M * NN);
  for (int e4 = tid; e4 < NN / 4; e4 += T) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int m = 0; m < a.M; ++m) {
      const float4 v = ld_ro(Im4 + (size_t)m * (NN / 4) + e4);
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    float* row = L + (4 * e4 / N) * RS + (4 * e4) % N;
    row[0] = acc.x;
    row[1] = acc.y;
    row[2] = acc.z;
    row[3] = acc.w;
  }
  __syncthreads();
  const float* Id = a.I_meas ? a.I_meas + (size_t)checked_index(a.idx, b, a.Ntot, a.status) * NN : nullptr;
  const float p = a.p;
  float sd = 0.f, st = 0.f, sp = 0.f;
  for (int q = tid; q < NN; q += T) {
    const int k0 = (q / N + N / 2) & (N - 1), k1 = (q % N + N / 2) & (N - 1);
    const int l = kpos1<N>(k1) * RS + kpos0<N>(k0);  // staging row p1, column p0 (global p1 * N + p0)
    const float I = L[l];
    if (a.I_model) a.I_model[(size_t)b * NN + q] = I;
    if (Id) {
      const float d = Id[q];
      float term, u, Dp;
      loss_pixel(I, d, p, a.eps, a.loss, &term, &Dp, &u);
      sd += Dp;
      st += term;
      L[l] = u;
      if (PAC) {  // sums in detector order: a warp's atomics land on consecutive addresses
        atomicAdd(a.pac + q, I);
        atomicAdd(a.pac + NN + q, d);
        sp += pow_nn(d, a.pac_p);
      }
    }
  }
  __syncthreads();
  if (a.u) {
    for (int e = tid; e < NN; e += T) a.u[(size_t)b * NN + e] = L[(e / N) * RS + e % N];
  }
  if (a.lpart) {
    double x = sd, y = st;
    block_sum2<T>(x, y, red);
    if (tid == 0) {
      a.lpart[2 * b] = x;
      a.lpart[2 * b + 1] = y;
    }
  }
  if (PAC) {
    __syncthreads();
    double x = sp, y = 0.0;
    block_sum2<T>(x, y, red);
    if (tid == 0) a.pacpart[b] = x;
  }
}

// The same without shared-memory staging (the N = 256 staging area would not fit): walks the
// pattern in k-space order (coalesced mode sum and dL/dI), gathering the measured pattern and
// scattering the modelled one in detector order.
template <int N, int T, bool PAC = false>
__global__ void __launch_bounds__(T) k_loss_gather(LossArgs a) {
  constexpr int NN = N * N;
  __shared__ double red[2 * (T / 32)];
  const int b = blockIdx.x, tid = threadIdx.x;
  const float* Im = a.Imode + (size_t)b * a.M * NN;
  const float* Id = a.I_meas ? a.I_meas + (size_t)checked_index(a.idx, b, a.Ntot, a.status) * NN : nullptr;
  float sd = 0.f, st = 0.f, sp = 0.f;
  for (int e = tid; e < NN; e += T) {  // e = p1 * N + p0
    float I = 0.f;
    for (int m = 0; m < a.M; ++m) I += Im[(size_t)m * NN + e];
    const int k0 = kbin0<N>(e % N), k1 = kbin1<N>(e / N);
    const int q = ((k0 + N / 2) & (N - 1)) * N + ((k1 + N / 2) & (N - 1));
    if (a.I_model) a.I_model[(size_t)b * NN + q] = I;
    if (Id) {
      float term, u, Dp;
      const float d = Id[q];
      loss_pixel(I, d, a.p, a.eps, a.loss, &term, &Dp, &u);
      sd += Dp;
      st += term;
      a.u[(size_t)b * NN + e] = u;
      if (PAC) {
        atomicAdd(a.pac + e, I);
        atomicAdd(a.pac + NN + e, d);
        sp += pow_nn(d, a.pac_p);
      }
    }
  }
  if (a.lpart) {
    double x = sd, y = st;
    block_sum2<T>(x, y, red);
    if (tid == 0) {
      a.lpart[2 * b] = x;
      a.lpart[2 * b + 1] = y;
    }
  }
  if (PAC) {
    __syncthreads();
    double x = sp, y = 0.0;
    block_sum2<T>(x, y, red);
    if (tid == 0) a.pacpart[b] = x;
  }
}

// PACBED term (Eq. 7) of one batch, one CTA of 1024 threads: the batch-mean patterns A and C from
// the sums, d = A^p - C^p, the loss w sqrt(<d^2>) / <I_meas^p> added to *loss_out, and the
// derivative w d p A^(p-1) / (<I_meas^p> N^2 B sqrt(<d^2>)), the same for every pattern, written to
// pac[2 N^2 ..] (k-space order) for the adjoint.  The sums are in the order of the loss kernel's
// loop: detector order (k_loss, N <= 128) or k-space order (k_loss_gather, N = 256).
template <int N>
__global__ void __launch_bounds__(1024) k_pacbed(float* __restrict__ pac, const double* __restrict__ pacpart, int B,
                                                 float p, float w, double* loss_out, double* scal, int* status) {
  constexpr int NN = N * N;
  __shared__ double red[64];
  __shared__ double sh[2];
  const int tid = threadIdx.x;
  const float inv_b = 1.0f / (float)B;
  double m2 = 0.0, z = 0.0;
  for (int e = tid; e < NN; e += 1024) {
    const float d = pow_nn(pac[e] * inv_b, p) - pow_nn(pac[NN + e] * inv_b, p);
    m2 += (double)d * d;
  }
  for (int b = tid; b < B; b += 1024) z += pacpart[b];
  block_sum2<1024>(m2, z, red);
  if (tid == 0) {
    const double ms = m2 / NN, Z = z / ((double)NN * B);
    const double L = sqrt(ms) / Z;
    if (!isfinite(L)) atomicOr(status, PTY_ENONFINITE);
    sh[0] = ms > 0.0 && Z > 0.0 ? (double)w / (Z * NN * B * sqrt(ms)) : 0.0;
    scal[2] = L;
    if (loss_out) *loss_out += (double)w * L;
  }
  __syncthreads();
  const float c = (float)sh[0];
  for (int e = tid; e < NN; e += 1024) {
    const float A = pac[e] * inv_b;
    const float d = pow_nn(A, p) - pow_nn(pac[NN + e] * inv_b, p);
    const float dpow = p == 1.0f ? 1.0f : (A > 0.f ? p * powf(A, p - 1.0f) : 0.f);
    int ek = e;  // k-space position of sum element e
    if constexpr (N != 256) {
      const int k0 = (e / N + N / 2) & (N - 1), k1 = (e % N + N / 2) & (N - 1);
      ek = kpos1<N>(k1) * N + kpos0<N>(k0);
    }
    pac[2 * NN + ek] = c * d * dpow;
  }
}

// The far-field weight of the adjoint with the PACBED term folded in, for every pattern of the
// batch: u <- 2 (s u + g_pacbed) / N, s the dL/dI normaliser (scal[0]); the adjoint then reads u
// with gs = 1, so its first transform carries no extra operand.
template <int N>
__global__ void k_pacbed_fold(float* __restrict__ u, const float* __restrict__ pacg, const double* __restrict__ scal,
                              size_t n) {
  constexpr int NN = N * N;
  const float gs = (float)(2.0 * scal[0] / N), gp = 2.0f / N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    u[i] = fmaf(gp, pacg[i % NN], gs * u[i]);
}

// Batch loss (Eq. 5 / 6) and the normaliser of dL/dI, in FP64, fixed summation order.  With the
// means of Eq. 5 / 6 written out over D detector pixels and B patterns, Poisson is -Y / S and
// Gaussian sqrt(D B Q) / S, where S = sum of I_meas^p, Y = sum of the Poisson summands and
// Q = sum of the squared residuals.  `whole` (or nullptr) holds {S, Q, D B} of the whole batch when
// this call holds one part of it: the normaliser then comes from the whole batch, and the loss
// written is this part's share of the whole batch's loss (the shares of the parts add up to it).
static __global__ void k_loss_finalize(const double* __restrict__ lpart, int B, int loss, double DB, double* scal,
                                       double* loss_out, int* status, const double* __restrict__ whole) {
  __shared__ double red[64];
  double x = 0.0, y = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    x += lpart[2 * b];
    y += lpart[2 * b + 1];
  }
  block_sum2<256>(x, y, red);
  if (threadIdx.x == 0) {
    const double S = whole ? whole[0] : x;
    double Lv, scale;
    if (loss == PTY_LOSS_POISSON) {
      Lv = -y / S;
      scale = 1.0 / S;
    } else {
      const double Q = whole ? whole[1] : y, DBw = whole ? whole[2] : DB;
      // this part's share y / Q of sqrt(D B Q) / S is sqrt(D B / Q) y / S
      Lv = Q > 0.0 ? sqrt(DBw / Q) * y / S : 0.0;
      scale = Q > 0.0 ? sqrt(DBw) / (sqrt(Q) * S) : 0.0;
    }
    if (!isfinite(Lv) || !isfinite(scale)) {
      atomicOr(status, PTY_ENONFINITE);
      scale = 0.0;
    }
    scal[0] = scale;
    scal[1] = Lv;
    if (loss_out) *loss_out = Lv;
  }
}

// Per-pattern sum of I_meas^p (one CTA per batch entry) into lpart[2 b]; lpart[2 b + 1] = 0.  The
// Poisson normaliser needs only the measured patterns, so its statistics need no forward pass.
template <int N, int T>
__global__ void __launch_bounds__(T) k_meas_sum(const float* __restrict__ I_meas, const int32_t* __restrict__ idx,
                                                int Ntot, float p, double* __restrict__ lpart, int* status) {
  constexpr int NN = N * N;
  __shared__ double red[2 * (T / 32)];
  const int b = blockIdx.x;
  const float* Id = I_meas + (size_t)checked_index(idx, b, Ntot, status) * NN;
  float sd = 0.f;
  for (int q = threadIdx.x; q < NN; q += T) sd += pow_nn(Id[q], p);
  double x = sd, y = 0.0;
  block_sum2<T>(x, y, red);
  if (threadIdx.x == 0) {
    lpart[2 * b] = x;
    lpart[2 * b + 1] = 0.0;
  }
}

// {sum over the batch of lpart[2 b], of lpart[2 b + 1], D B} into out[3] (fixed summation order).
static __global__ void k_batch_stats(const double* __restrict__ lpart, int B, double DB, double* __restrict__ out,
                                     int* status) {
  __shared__ double red[64];
  double x = 0.0, y = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    x += lpart[2 * b];
    y += lpart[2 * b + 1];
  }
  block_sum2<256>(x, y, red);
  if (threadIdx.x == 0) {
    if (!isfinite(x) || !isfinite(y)) atomicOr(status, PTY_ENONFINITE);
    out[0] = x;
    out[1] = y;
    out[2] = DB;
  }
}

// ---------------------------------------------------------------------------------------------
// Adjoint: one CTA per (b, m), slices in reverse.
// ---------------------------------------------------------------------------------------------
// Wave (b M' + m', M' = modes per position) of the adjoint's w-th CTA (or cluster) out of `waves`.
// G = 0: w itself.  G > 0: w runs over groups of G positions (the last group may be smaller), and
// within a group over modes, then positions.  A bijection of [0, waves).
template <int G>
__device__ __forceinline__ int adj_wave(int w, int waves, int MK) {
  if constexpr (G == 0) {
    return w;
  } else {
    const int B = waves / MK, full = B / G * G;
    int b, mk;
    if (w < full * MK) {
      const int g = w / (G * MK), r = w % (G * MK);
      mk = r / G;
      b = g * G + r % G;
    } else {
      const int r = w - full * MK, R = B - full;
      mk = r / R;
      b = full + r % R;
    }
    return b * MK + mk;
  }
}

struct AdjArgs {
  int M, Ko, Nz, H, W, Ntot, global_tilt, grad_mask;  // Ko: object modes
  float dx, lam;
  const int32_t* idx;
  const float *pos, *tilt, *dz;
  const float2* T;
  const float2* Phat;
  // entering wave of slice s at ckpt[wave][s - ck_first], spectrum entering slice s at
  // vhat[wave][s - 1 - vh_first]; ck_per_wave / vh_per_wave slots per wave
  const float2* ckpt;
  const float2* vhat;
  int ck_first, ck_per_wave, vh_first, vh_per_wave;
  const float2* Psi;
  const float* u;
  const double* scal;
  float2* gT;
  float2* gPhat;
  double* spart;  // [wave][5], accumulated over the segments of one pass
  int u_scaled;  // 1: u holds 2 dL/dI / N with the PACBED term folded in (k_pacbed_fold)
  int* status;
  // slices [s0, s1) of this launch; the adjoint wave is carried between launches in gstate
  int s0, s1;
  float2* gstate;
};

// Bulk-copy staging of the adjoint's once-read blocks (N = 128, split transmission and propagation
// passes, so it also needs PTY_ADJ_SPLIT_ROW = 1).  The checkpoint a slice's transmission pass reads and the spectrum its propagation pass
// reads are contiguous 128 KB blocks; the first half of each (natural rows 0..63, k-space columns
// 0..63: the first two load batches of those passes) is copied by one thread with cp.async.bulk into
// the 64 KB of shared memory the wave leaves free, three transform steps before it is read.  The
// other half is read from global memory as before.
#ifndef PTY_ADJ_STAGE
#define PTY_ADJ_STAGE 0
#endif
template <int N, int T>
__host__ __device__ constexpr bool adj_staged() {
  return PTY_ADJ_STAGE && N == 128 && PTY_ADJ_SPLIT_COL && PTY_ADJ_SPLIT_ROW;
}
// Large-window adjoint: the cross-CTA column step of CTA q reads the entering wave at every row and
// at q's column slab [N/C q, N/C (q + 1)).  With PTY_ADJ256_STAGE = 1 warp 0 copies rows 0..N/2-1 of
// that slab of the next slice's checkpoint (N/2 row pieces of N/C float2, 64 KB) into the free
// shared memory right after the current column step, five passes before the next one reads it.
#ifndef PTY_ADJ256_STAGE
#define PTY_ADJ256_STAGE 0
#endif
template <int N>
__host__ __device__ constexpr bool adj256_staged() {
  return PTY_ADJ256_STAGE && N == 256 && !PTY_ADJ256_SPLIT_COL;
}
// Whether the adjoint's transmission (COL) and propagation (ROW) steps run as their own pointwise
// passes (true) or inside the neighbouring transform steps (false), per window size.
template <int N>
__host__ __device__ constexpr bool adj_split_col() {
  return N == 256 ? PTY_ADJ256_SPLIT_COL != 0 : PTY_ADJ_SPLIT_COL != 0;
}
template <int N>
__host__ __device__ constexpr bool adj_split_row() {
  return N == 256 ? PTY_ADJ256_SPLIT_ROW != 0 : PTY_ADJ_SPLIT_ROW != 0;
}
constexpr int kStageBytes = 64 * 1024;
// Byte offset of the stage in the adjoint's shared memory: after the wave, the tables and the
// reduction slots of up to 1024 threads, so that it does not depend on the CTA size.
template <int N>
__host__ __device__ constexpr size_t adj_stage_offset() {
  return (sizeof(float2) * ((size_t)wave_rows<N>() * (N + 1) + 5 * N) + sizeof(float) * 6 * N +
          sizeof(double) * 5 * 32 + 127) / 128 * 128;
}
template <int N, int T>
__host__ __device__ constexpr size_t adj_smem_bytes() {
  static_assert(T <= 1024, "reduction slots");
  return adj_staged<N, T>() || adj256_staged<N>() ? adj_stage_offset<N>() + kStageBytes + 16
                            : sizeof(float2) * ((size_t)wave_rows<N>() * (N + 1) + 5 * N) + sizeof(float) * 6 * N +
                                  sizeof(double) * 5 * (T / 32);
}
// The stage in the calling kernel's dynamic shared memory.
template <int N>
__device__ __forceinline__ float2* adj_stage() {
  extern __shared__ __align__(16) float2 sm[];
  return reinterpret_cast<float2*>(reinterpret_cast<char*>(sm) + adj_stage_offset<N>());
}


// ---- adjoint hooks ----
// g_psi at the far field = F_ortho^-1[2 dL/dI Psi]: forms 2 dL/dI Psi / N (k-space), replaces
template <int N>
struct FarGradLoad {
  static constexpr bool kReplaces = true;
  static constexpr bool kPreload = false;  // may run in a step that has read two tasks
  static constexpr int kChunk = PTY_KG;
  const float* u;
  const float2* Psi;
  float gs;  // 2 x (dL/dI normaliser) / N, or 1 when u already holds the scaled weight
  template <int K>
  __device__ __forceinline__ void operator()(int r0, int rs, int c0, int cs, float2* v) {
    float2 p[K];
    float w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int e = kidx<N>(r0 + k * rs, c0 + k * cs);
      p[k] = ld_ro(Psi + e);
      w[k] = ld_ro(u + e);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = cscale(p[k], gs * w[k]);
  }
};
// transmission of slice s backwards: dL/dT += conj(psi_in) g (scatter-add), g <- conj(T) g
template <int N>
struct AdjTransLoad {
  static constexpr bool kReplaces = false;
  static constexpr bool kPreload = false;  // may run in a step that has read two tasks
  static constexpr int kChunk = PTY_KA;
  const float2* Ts;  // patch corner in T
  float2* gTs;       // patch corner in the dL/dT accumulator
  const float2* ck;  // checkpoint of the wave entering slice s, or nullptr (no object gradient)
  int W;
  bool stg = false;  // rows 0..N/2-1 of ck are in the stage (adj_stage): (r, c) at r * st_ld + c - st_c0
  int st_ld = N, st_c0 = 0;
  template <int K>
  __device__ __forceinline__ void operator()(int r0, int rs, int c0, int cs, float2* v) {
    float2 t[K], ps[K];
    const bool staged = stg && r0 + (K - 1) * rs < N / 2;
    const float2* st = adj_stage<N>();
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int r = r0 + k * rs, c = c0 + k * cs;
      t[k] = ld_ro(Ts + (size_t)r * W + c);
      if (ck) ps[k] = staged ? st[r * st_ld + c - st_c0] : ld_once(ck + r * N + c);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (ck) atomicAdd(gTs + (size_t)(r0 + k * rs) * W + c0 + k * cs, cmulc(ps[k], v[k]));
      v[k] = cmulc(t[k], v[k]);
    }
  }
};
// propagation backwards in k-space: dz / tilt terms against the stored forward spectrum, then
// g^ <- conj(M) g^ / N^2.  Accumulates -sum w (e0 + e1), -sum w c0, -sum w c1 with w = Im(conj(g^) v^).
template <int N>
struct AdjPropStore {
  static constexpr bool kReplaces = false;
  static constexpr bool kPreload = false;  // may run in a step that has read two tasks
  static constexpr int kChunk = PTY_KQ;
  const float2 *cm0, *cm1;
  const float2* vh;  // stored v^/N^2 of this propagation, or nullptr
  const float *e0, *e1, *c0t, *c1t;
  float &dz, &t0, &t1;
  bool stg = false;  // k-space columns 0..N/2-1 of vh (its first half) are in the stage (adj_stage)
  template <int K>
  __device__ __forceinline__ void operator()(int r0, int rs, int c0, int cs, float2* v) {
    if (vh) {
      float2 x[K];
      const bool staged = stg && c0 + (K - 1) * cs < N / 2;
      const float2* st = adj_stage<N>();
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int e = kidx<N>(r0 + k * rs, c0 + k * cs);
        x[k] = staged ? st[e] : ld_once(vh + e);
      }
      if (rs == 0) {
        // a chunk of one k-space row (every caller): the row's dz and tilt factors multiply the
        // chunk's sum of w once, sum_k w (e0 + e1_k) = e0 sum_k w + sum_k w e1_k
        float sw = 0.f, sd = 0.f, s1 = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int c = c0 + k * cs;
          const float w = v[k].x * x[k].y - v[k].y * x[k].x;
          sw += w;
          sd = fmaf(w, e1[c], sd);
          s1 = fmaf(w, c1t[c], s1);
        }
        dz = fmaf(sw, e0[r0], dz + sd);
        t0 = fmaf(sw, c0t[r0], t0);
        t1 += s1;
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int r = r0 + k * rs, c = c0 + k * cs;
          const float w = v[k].x * x[k].y - v[k].y * x[k].x;
          dz = fmaf(w, e0[r] + e1[c], dz);
          t0 = fmaf(w, c0t[r], t0);
          t1 = fmaf(w, c1t[c], t1);
        }
      }
    }
    if (rs == 0) {
      const float2 f0 = cm0[r0];
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] = cmul(cmul(v[k], f0), cm1[c0 + k * cs]);
      return;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = cmul(cmul(v[k], cm0[r0 + k * rs]), cm1[c0 + k * cs]);
  }
};
// dL/dP_j in k-space: probe-spectrum gradient conj(R) g^ (scatter-add) and the position terms
// sum f_a Im(conj(g^) R P^) (f_a carries 2 pi / N^2).
template <int N>
struct ProbeStore {
  static constexpr bool kReplaces = false;
  static constexpr bool kPreload = false;  // may run in a step that has read two tasks
  static constexpr int kChunk = PTY_KR;
  float2* gP;  // or nullptr
  const float2* Ph;
  const float2 *cr0, *cr1;
  const float *f0, *f1;
  bool pos;
  float &p0, &p1;
  template <int K>
  __device__ __forceinline__ void operator()(int r0, int rs, int c0, int cs, float2* v) {
    float2 ph[K];
    if (pos) {
#pragma unroll
      for (int k = 0; k < K; ++k) ph[k] = ld_ro(Ph + kidx<N>(r0 + k * rs, c0 + k * cs));
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int r = r0 + k * rs, c = c0 + k * cs;
      const float2 cr = cmul(cr0[r], cr1[c]);  // conj(R)
      if (gP) atomicAdd(gP + kidx<N>(r, c), cmul(cr, v[k]));
      if (pos) {
        const float2 PR = cmulc(cr, ph[k]);  // R P^
        const float w = v[k].x * PR.y - v[k].y * PR.x;
        p0 = fmaf(w, f0[r], p0);
        p1 = fmaf(w, f1[c], p1);
      }
    }
  }
};

template <int N, int T, bool OM = false>
__global__ void __launch_bounds__(T, Launch<N>::MINB_A) k_adjoint(AdjArgs a) {
  using F = Fft2<N, T>;
  constexpr int RS = F::RS;
  constexpr int NN = N * N;
  extern __shared__ __align__(16) float2 sm[];
  float2* s = sm;
  float2* tw = s + F::ROWS * RS;
  float2* cm0 = tw + N;   // conj propagator, axis 0, carries 1/N^2
  float2* cm1 = cm0 + N;  // conj propagator, axis 1
  float2* cr0 = cm1 + N;  // conj shift ramp, axis 0
  float2* cr1 = cr0 + N;  // conj shift ramp, axis 1
  float* e0 = reinterpret_cast<float*>(cr1 + N);  // -(dM/d dz)/(i M) per axis
  float* e1 = e0 + N;
  float* c0 = e1 + N;  // -(dM/d theta_a)/(i M)
  float* c1 = c0 + N;
  float* f0 = c1 + N;  // 2 pi f_a / N^2 (position term)
  float* f1 = f0 + N;
  double* red = reinterpret_cast<double*>(f1 + N);
  const int tid = threadIdx.x, lane = tid & 31;
  // wave (position, mode); a cluster of F::C CTAs per wave
  const int bm = adj_wave<PTY_ADJ_GROUP>(blockIdx.x / F::C, gridDim.x / F::C, a.M * (OM ? a.Ko : 1));
  const int Ko = OM ? a.Ko : 1;
  const int b = bm / (a.M * Ko), m = (bm / Ko) % a.M;  // waves: (position, probe mode, object mode)
  const int j = checked_index(a.idx, b, a.Ntot, a.status);
  int i0, i1;
  float d0, d1, th0, th1;
  patch_corner<N>(a.pos, j, a.H, a.W, &i0, &i1, &d0, &d1, a.status);
  tilt_of(a.tilt, a.global_tilt, j, &th0, &th1);
  const float dz = a.dz[0];
  const bool want_obj = (a.grad_mask & (PTY_GRAD_AMP | PTY_GRAD_PHASE)) != 0;
  const bool want_probe = (a.grad_mask & PTY_GRAD_PROBE) != 0;
  const bool want_pos = (a.grad_mask & PTY_GRAD_POS) != 0;
  const bool want_prop = (a.grad_mask & (PTY_GRAD_DZ | PTY_GRAD_TILT)) != 0 && a.vhat != nullptr;
  const size_t plane = (size_t)a.H * a.W;
  const size_t patch = (OM ? (size_t)(bm % Ko) * a.Nz * plane : 0) + (size_t)i0 * a.W + i1;
  // slot pointers relative to slice numbers (ck_base + s * NN is slice s's entering wave, vh_base +
  // (s - 1) * NN the spectrum entering slice s)
  const float2* ck_base = want_obj ? a.ckpt + ((ptrdiff_t)bm * a.ck_per_wave - a.ck_first) * NN : nullptr;
  const float2* vh_base = want_prop ? a.vhat + ((ptrdiff_t)bm * a.vh_per_wave - a.vh_first) * NN : nullptr;
#if PTY_ADJ_PF < 3
  if (want_obj) prefetch_block<N>(ck_base + (size_t)(a.s1 - 1) * NN);
  if (want_prop && a.s1 - 1 > a.s0 - 1 && a.s1 >= 2) prefetch_block<N>(vh_base + (size_t)(a.s1 - 2) * NN);
#endif

  // Staging (adj_staged): copies alternate checkpoint (slice sl, issued after the previous slice's
  // propagation pass) and spectrum (issued after the transmission pass); every thread waits on each
  // copy once, in issue order, so the k-th wait is on phase parity k & 1, and copy k + 1 is issued
  // only after every thread has passed wait k.  A wait that gives up flags PTY_ETIMEOUT; from then
  // on that thread reads global memory and never tests the barrier again (a later parity test
  // could match an earlier phase), and thread 0 stops issuing.
  constexpr bool kStage = adj_staged<N, T>();
  float2* stg = adj_stage<N>();
  const uint32_t sbar = smem_u32(stg + kStageBytes / sizeof(float2));
  // bit 0: parity of the next wait; bit 31: one of this thread's waits gave up (bit 0 then holds
  // the parity of that wait)
  uint32_t sst = 0;
  auto stage_get = [&]() -> bool {  // wait for the next copy; false if it is not there
    if (sst >> 31) return false;
    if (stage_wait(sbar, sst & 1)) {
      sst ^= 1;
      return true;
    }
    sst |= 0x80000000u;
    atomicOr(a.status, PTY_ETIMEOUT);
    return false;
  };
  if constexpr (kStage) {
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbar) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      if (want_obj) stage_issue(sbar, stg, ck_base + (size_t)(a.s1 - 1) * NN, kStageBytes);
    }
  }
  // Large-window stage (adj256_staged): one copy batch per slice, issued by warp 0 after the column
  // step that read the previous batch and waited for by every thread before the next column step,
  // so the k-th wait is again on parity k & 1.  Warp 0 stops issuing once its lane 0 gave up.
  constexpr bool kSlab = adj256_staged<N>();
  constexpr int SW = N / F::C;  // columns of the slab
  auto stage_slab = [&](int sl) {
    if (tid < 32 && !(__shfl_sync(0xffffffffu, sst, 0) >> 31)) {
      constexpr uint32_t piece = SW * sizeof(float2);
      static_assert(!kSlab || (N / 2) * piece == kStageBytes, "the slab half fills the stage");
      const uint64_t pol = evict_first_policy();
      if (tid == 0) stage_expect(sbar, (N / 2) * piece);
      __syncwarp();
      const float2* src = ck_base + (size_t)sl * NN + SW * F::rank();
      for (int r = tid; r < N / 2; r += 32) stage_copy(sbar, stg + r * SW, src + (size_t)r * N, piece, pol);
    }
  };
  if constexpr (kSlab) {
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbar) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) __syncwarp();
    if (want_obj) stage_slab(a.s1 - 1);
  }

  build_twiddles<N>(tw);
  adj_tables<N>(cm0, cm1, cr0, cr1, e0, e1, c0, c1, f0, f1, d0, d1, th0, th1, dz, a.dx, a.lam);
#if PTY_ADJ_L1PF
  if (want_obj) prefetch_l1(ck_base + (size_t)(a.s1 - 1) * NN, PTY_ADJ_L1PF * 1024);
#endif
  __syncthreads();

  if (a.s1 == a.Nz) {
    // g_psi = F_ortho^-1[2 dL/dI Psi] = (1/N) unnormalised inverse of 2 dL/dI Psi; its column step
    // is fused with the last slice's transmission below (same step structure as the forward kernel).
    FarGradLoad<N> farg{a.u + (size_t)b * NN, a.Psi + (size_t)bm * NN,
                        a.u_scaled ? 1.0f : (float)(2.0 * a.scal[0] / N)};
    F::row_inv(s, tw, farg);
    F::block_inv(s, tw);
  } else {
    const float2* g = a.gstate + (size_t)bm * NN + (size_t)F::rank() * F::ROWS * N;
    for (int e = tid; e < F::ROWS * N; e += T) s[(e / N) * RS + e % N] = ld_ro(g + e);
    __syncthreads();
  }

  float gdz = 0.f, gt0 = 0.f, gt1 = 0.f, gp0 = 0.f, gp1 = 0.f;
  NoHook none;
  for (int sl = a.s1 - 1; sl >= a.s0; --sl) {
#if PTY_ADJ256_PF
    if constexpr (F::C > 1) {
      if (sl - 1 >= a.s0) {
        prefetch_patch<N, F::C>(a.T + (sl - 1) * plane + patch, a.W, F::rank());
        if (want_obj) prefetch_patch<N, F::C>(ck_base + (size_t)(sl - 1) * NN, N, F::rank());
      }
      if (want_prop && sl - 2 >= a.s0 - 1 && sl >= 2)
        prefetch_patch<N, F::C>(vh_base + (size_t)(sl - 2) * NN, N, F::rank());
    }
#endif
#if PTY_ADJ_PF == 0
    if (sl - 1 >= a.s0 && want_obj) prefetch_block<N>(ck_base + (size_t)(sl - 1) * NN);
    if (sl - 2 >= a.s0 - 1 && sl >= 2 && want_prop) prefetch_block<N>(vh_base + (size_t)(sl - 2) * NN);
#elif PTY_ADJ_PF == 1
    if (sl >= 1 && sl < a.s1 - 1 && want_prop) prefetch_block<N>(vh_base + (size_t)(sl - 1) * NN);
#endif
    AdjTransLoad<N> trans{a.T + sl * plane + patch, a.gT + sl * plane + patch,
                          want_obj ? ck_base + (size_t)sl * NN : nullptr, a.W};
    if (sl > 0 || want_probe || want_pos) {  // (sl > 0: propagate back into slice sl - 1)
      if constexpr (adj_split_col<N>()) {
      // column inverse, then the transmission step as its own pass with deep load batches, then
      // the column forward: one more shared-memory round trip, but no DFT registers are live
      // while the checkpoint and transmission loads are in flight
      F::col_inv(s, tw);
      if constexpr (kStage) {
        if (want_obj) trans.stg = stage_get();
      }
      F::template pointwise<(N == 256 ? PTY_ADJ256_BATCH : PTY_ADJ_BATCH)>(s, trans);
      if constexpr (kStage) {  // the stage is free again: fetch this slice's spectrum
        if (tid == 0 && !(sst >> 31) && want_prop && sl > 0)
          stage_issue(sbar, stg, vh_base + (size_t)(sl - 1) * NN, kStageBytes);
      }
#if PTY_ADJ_L1PF
      if (want_prop && sl > 0) prefetch_l1(vh_base + (size_t)(sl - 1) * NN, PTY_ADJ_L1PF * 1024);
#endif
      F::col_fwd(s, tw, none);
      } else {
        if constexpr (kSlab) {
          if (want_obj) {
            trans.stg = stage_get();
            trans.st_ld = SW;
            trans.st_c0 = SW * F::rank();
          }
        }
        F::template col_inv_fwd<true>(s, tw, trans);
        if constexpr (kSlab) {  // every thread is past the column step: fetch the next slice's slab
          if (want_obj && sl - 1 >= a.s0) stage_slab(sl - 1);
        }
      }
#if PTY_ADJ_PF == 1
      if (sl - 1 >= a.s0 && want_obj) prefetch_block<N>(ck_base + (size_t)(sl - 1) * NN);
#endif
      F::block_fwd(s, tw);
      if (sl > 0) {
        AdjPropStore<N> prop{cm0, cm1, want_prop ? vh_base + (size_t)(sl - 1) * NN : nullptr, e0, e1, c0, c1,
                             gdz, gt0, gt1};
        if constexpr (adj_split_row<N>()) {
        F::template row_fwd<true>(s, none);
        if constexpr (kStage) {
          if (want_prop) prop.stg = stage_get();
        }
        F::template pointwise_k<(N == 256 ? PTY_ADJ256_BATCH : PTY_ADJ_BATCH)>(s, prop);
        if constexpr (kStage) {  // the stage is free again: fetch the next slice's checkpoint
          if (tid == 0 && !(sst >> 31) && want_obj && sl - 1 >= a.s0)
            stage_issue(sbar, stg, ck_base + (size_t)(sl - 1) * NN, kStageBytes);
        }
#if PTY_ADJ_L1PF
        if (want_obj && sl - 1 >= a.s0) prefetch_l1(ck_base + (size_t)(sl - 1) * NN, PTY_ADJ_L1PF * 1024);
#endif
        F::row_inv(s, tw, none);
        } else {
          F::row_fwd_inv(s, tw, prop);
        }
        F::block_inv(s, tw);
      } else {
        ProbeStore<N> probe{want_probe ? a.gPhat + (size_t)m * NN : nullptr, a.Phat + (size_t)m * NN, cr0, cr1, f0,
                            f1, want_pos, gp0, gp1};
        F::template row_fwd<false>(s, probe);
      }
    } else if (want_obj) {
      if constexpr (kStage) trans.stg = stage_get();
      if constexpr (kSlab) {
        trans.stg = stage_get();
        trans.st_ld = SW;
        trans.st_c0 = SW * F::rank();
      }
      F::template col_inv_fwd<false>(s, tw, trans);
    }
  }
  if constexpr (kStage || kSlab) {  // a copy whose wait gave up may still be in flight: give it time to land
    if (tid == 0 && (sst >> 31)) stage_wait(sbar, sst & 1);
  }

  // FP64 reduction of the five scalar partials over the CTA
  double v5[5] = {gp0, gp1, gt0, gt1, gdz};
#pragma unroll
  for (int q = 0; q < 5; ++q)
    for (int o = 16; o > 0; o >>= 1) v5[q] += __shfl_down_sync(0xffffffffu, v5[q], o);
  const int w = tid / 32;
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) red[5 * w + q] = v5[q];
  }
  __syncthreads();
  if (tid < 5) {
    double acc = 0.0;
    for (int i = 0; i < T / 32; ++i) acc += red[5 * i + tid];
    if constexpr (F::C == 1) {
      a.spart[(size_t)bm * 5 + tid] += acc;
    } else {  // the CTAs of a cluster each hold part of the wave
      atomicAdd(a.spart + (size_t)bm * 5 + tid, acc);
    }
  }
  if (a.s0 > 0) {  // hand the adjoint wave to the launch of the previous segment
    float2* g = a.gstate + (size_t)bm * NN + (size_t)F::rank() * F::ROWS * N;
    for (int e = tid; e < F::ROWS * N; e += T) g[e] = s[(e / N) * RS + e % N];
  }
}

// ---------------------------------------------------------------------------------------------
// Phase-sparsity term (Eq. 8): <|phase|^p>^(1/p) over every slice of every batch position's patch.
// With c(y, x) the number of batch patches that contain pixel (y, x), the sum over patches is the
// sum over pixels of c |phase|^p and the gradient of a pixel is c times a patch's, so the term is
// one pass over the object with no atomics on it: patch rows mark +1 / -1 at their column ends in
// a row-difference array (2 int atomics per patch row), a warp-per-row scan turns the marks into c.
// ---------------------------------------------------------------------------------------------
constexpr int kSparseBlocks = 152 * 8;  // CTAs of the sum pass (its FP64 partials)

// one CTA per batch position, one thread per patch row
template <int N>
__global__ void __launch_bounds__(N) k_cover_marks(const float* __restrict__ pos, const int32_t* __restrict__ idx,
                                                   int Ntot, int H, int W, int* __restrict__ D, int* status) {
  const int j = checked_index(idx, blockIdx.x, Ntot, status);
  int i0, i1;
  float d0, d1;
  patch_corner<N>(pos, j, H, W, &i0, &i1, &d0, &d1, status);  // clamped inside the object
  int* row = D + (size_t)(i0 + threadIdx.x) * (W + 1);
  atomicAdd(row + i1, 1);
  atomicAdd(row + i1 + N, -1);
}

// c(y, x) = inclusive prefix sum of the marks along row y; one warp per row, in place
static __global__ void k_cover_scan(int* __restrict__ D, int H, int W) {
  const int lane = threadIdx.x & 31;
  const int y = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (y >= H) return;
  int* row = D + (size_t)y * (W + 1);
  int carry = 0;
  for (int x0 = 0; x0 < W; x0 += 32) {
    const int x = x0 + lane;
    int v = x < W ? row[x] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    v += carry;
    if (x < W) row[x] = v;
    carry = __shfl_sync(0xffffffffu, v, 31);
  }
}

// FP64 partials of sum over every slice of c |phase|^p
template <int T>
__global__ void __launch_bounds__(T) k_sparse_sum(const float* __restrict__ phase, const int* __restrict__ C,
                                                  int H, int W, size_t n, float p, double* __restrict__ part) {
  __shared__ double red[2 * (T / 32)];
  const size_t plane = (size_t)H * W;
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)T + threadIdx.x; i < n; i += (size_t)gridDim.x * T) {
    const size_t q = i % plane;
    const int c = C[(q / W) * (W + 1) + q % W];
    if (c) acc += (double)c * pow_nn(fabsf(phase[i]), p);
  }
  double y = 0.0;
  block_sum2<T>(acc, y, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// the term (added to *loss_out) and the gradient factor (S/n)^(1/p - 1) / n into scal[3]
static __global__ void k_sparse_finalize(const double* __restrict__ part, int nparts, double n, float p, float w,
                                         double* loss_out, double* scal, int* status) {
  __shared__ double red[16];
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) x += part[i];
  block_sum2<256>(x, y, red);
  if (threadIdx.x == 0) {
    const double mean = x / n;
    const double L = mean > 0.0 ? pow(mean, 1.0 / p) : 0.0;
    if (!isfinite(L)) atomicOr(status, PTY_ENONFINITE);
    scal[3] = mean > 0.0 ? pow(mean, 1.0 / p - 1.0) / n : 0.0;
    if (loss_out) *loss_out += (double)w * L;
  }
}

// dL/dphase += w scal[3] c |phase|^(p - 1) sign(phase) at every pixel (c = patches containing it)
static __global__ void k_sparse_grad(const float* __restrict__ phase, const int* __restrict__ C, int H, int W,
                                     size_t n, float p, float w, const double* __restrict__ scal,
                                     float* __restrict__ g_phase) {
  const size_t plane = (size_t)H * W;
  const float f = w * (float)scal[3];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t q = i % plane;
    const int c = C[(q / W) * (W + 1) + q % W];
    const float x = phase[i], a = fabsf(x);
    if (c && a > 0.f) {
      const float wp = p == 1.0f ? 1.0f : powf(a, p - 1.0f);
      g_phase[i] += copysignf(f * (float)c * wp, x);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Finalisers
// ---------------------------------------------------------------------------------------------
// dL/damp = Re(conj(e^{i phase}) dL/dT), dL/dphase = Re(conj(i T) dL/dT) = Im(conj(T) dL/dT)
static __global__ void k_object_grad(const float* __restrict__ amp, const float* __restrict__ phase,
                              const float2* __restrict__ gT, float* __restrict__ g_amp, float* __restrict__ g_phase,
                              int accumulate, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float s, c;
    sincosf(phase[i], &s, &c);
    const float2 g = gT[i];
    const float a = amp[i];
    const float ga = fmaf(c, g.x, s * g.y);
    const float gp = a * fmaf(c, g.y, -s * g.x);
    if (g_amp) g_amp[i] = accumulate ? g_amp[i] + ga : ga;
    if (g_phase) g_phase[i] = accumulate ? g_phase[i] + gp : gp;
  }
}

// The accumulator holds A = sum_j conj(R_j) F[dL/dP_j] (R_j the shift ramp of position j).  The
// probe-spectrum gradient is A / N^2 and dL/dP_m = F^H[A / N^2] = (plain inverse sum of A) / N^2.
template <int N, int T>
__global__ void __launch_bounds__(T) k_probe_grad(const float2* __restrict__ gPhat, float2* __restrict__ g_probe,
                                                  int accumulate) {
  using F = Fft2<N, T>;
  constexpr int RS = F::RS;
  extern __shared__ __align__(16) float2 sm[];
  float2* s = sm;
  float2* tw = s + F::ROWS * RS;
  const int m = blockIdx.x / F::C, q = F::rank(), tid = threadIdx.x;
  constexpr int R = F::ROWS;
  build_twiddles<N>(tw);
  const float2* G = gPhat + (size_t)m * N * N;
  for (int e = tid; e < R * N; e += T) s[(e % R) * RS + e / R] = G[kidx<N>(q * R + e % R, e / R)];
  __syncthreads();
  F::inverse(s, tw);
  const float sc = 1.0f / (float)(N * N);
  float2* out = g_probe + (size_t)m * N * N + (size_t)q * R * N;  // this CTA's rows
  for (int e = tid; e < R * N; e += T) {
    const float2 v = cscale(s[(e / N) * RS + e % N], sc);
    out[e] = accumulate ? cadd(out[e], v) : v;
  }
}

// Positions, tilts (summed over modes; over positions too for a global tilt) and dz.
static __global__ void k_scalar_grad(const double* __restrict__ spart, const int32_t* __restrict__ idx, int B, int M,
                              int Ntot, int global_tilt, int grad_mask, float* g_pos, float* g_tilt, float* g_dz,
                              int accumulate) {
  __shared__ double red[64];
  double dzs = 0.0, t0s = 0.0;
  double t1s = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    double p0 = 0.0, p1 = 0.0, a0 = 0.0, a1 = 0.0;
    for (int m = 0; m < M; ++m) {
      const double* sp = spart + ((size_t)b * M + m) * 5;
      p0 += sp[0];
      p1 += sp[1];
      a0 += sp[2];
      a1 += sp[3];
      dzs += sp[4];
    }
    const int j = idx[b];
    if (j < 0 || j >= Ntot) continue;  // flagged by the forward kernel
    if ((grad_mask & PTY_GRAD_POS) && g_pos) {
      atomicAdd(g_pos + 2 * j, (float)p0);
      atomicAdd(g_pos + 2 * j + 1, (float)p1);
    }
    if ((grad_mask & PTY_GRAD_TILT) && g_tilt) {
      if (global_tilt) {
        t0s += a0;
        t1s += a1;
      } else {
        atomicAdd(g_tilt + 2 * j, (float)a0);
        atomicAdd(g_tilt + 2 * j + 1, (float)a1);
      }
    }
  }
  double x = dzs, y = t0s;
  block_sum2<256>(x, y, red);
  __syncthreads();
  double z = t1s, dummy = 0.0;
  block_sum2<256>(z, dummy, red);
  if (threadIdx.x == 0) {
    if ((grad_mask & PTY_GRAD_DZ) && g_dz) g_dz[0] = accumulate ? g_dz[0] + (float)x : (float)x;
    if ((grad_mask & PTY_GRAD_TILT) && g_tilt && global_tilt) {
      g_tilt[0] = accumulate ? g_tilt[0] + (float)y : (float)y;
      g_tilt[1] = accumulate ? g_tilt[1] + (float)z : (float)z;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Host side: one pass of the pipeline for size N
// ---------------------------------------------------------------------------------------------
#define PTY_LAUNCH_CHECK(what, stage)                                     \
  do {                                                                    \
    cudaError_t e_ = cudaGetLastError();                                  \
    if (e_ != cudaSuccess) {                                              \
      set_error("%s launch failed: %s", what, cudaGetErrorString(e_));    \
      return PTY_ECUDA;                                                   \
    }                                                                     \
    note_launch();                                                        \
    if (stage >= 0) prof_mark(stage, st);                                 \
  } while (0)

// Launch of a per-wave kernel: plain for one CTA per wave, as clusters of C CTAs otherwise.
template <int C, class... KArgs, class... Args>
cudaError_t launch_waves(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                         Args... args) {
  if constexpr (C == 1) {
    kern<<<grid, block, smem, st>>>(args...);
    return cudaGetLastError();
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid * C);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
  }
}

#define PTY_LAUNCH_RC(expr, what, stage)                                  \
  do {                                                                    \
    cudaError_t e_ = (expr);                                              \
    if (e_ == cudaSuccess) e_ = cudaGetLastError();                       \
    if (e_ != cudaSuccess) {                                              \
      set_error("%s launch failed: %s", what, cudaGetErrorString(e_));    \
      return PTY_ECUDA;                                                   \
    }                                                                     \
    note_launch();                                                        \
    if (stage >= 0) prof_mark(stage, st);                                 \
  } while (0)

// Phases of one pass.  Forward (with or without what the adjoint needs), loss, adjoint + gradients.
template <int N>
struct Pass {
  static constexpr int T = Launch<N>::T, TF = Launch<N>::TF, TA = Launch<N>::TA;
  static constexpr int NN = N * N;
  static constexpr int C = Fft2<N, TF>::C;  // CTAs per wave
  const Problem& pb;
  const Workspace& ws;
  cudaStream_t st;
  bool save, want_obj, want_probe, want_prop;
  int K, nseg;

  explicit Pass(const Problem& p) : pb(p), ws(p.ws), st(p.stream) {
    save = pb.mode != MODE_FORWARD && pb.mode != MODE_STATS;
    const int gm = pb.grad_mask;
    want_obj = save && (gm & (PTY_GRAD_AMP | PTY_GRAD_PHASE));
    want_probe = save && (gm & PTY_GRAD_PROBE);
    want_prop = save && (gm & (PTY_GRAD_DZ | PTY_GRAD_TILT)) && pb.Nz > 1;
    K = pb.kstride;
    nseg = (pb.Nz + K - 1) / K;
  }

  // the fused kernels for this problem's object-mode count
  auto fwd_kernel() const { return pb.Ko > 1 ? k_forward<N, TF, true> : k_forward<N, TF, false>; }
  auto recompute_kernel() const { return pb.Ko > 1 ? k_recompute<N, TF, true> : k_recompute<N, TF, false>; }
  auto adj_kernel() const { return pb.Ko > 1 ? k_adjoint<N, TA, true> : k_adjoint<N, TA, false>; }

  int set_attributes() {
    bool ok = cudaFuncSetAttribute(fwd_kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)fwd_kernel_smem_bytes<N>()) == cudaSuccess &&
              cudaFuncSetAttribute(recompute_kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)fwd_smem_bytes<N>()) == cudaSuccess &&
              cudaFuncSetAttribute(adj_kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)adj_smem_bytes<N, TA>()) == cudaSuccess &&
              cudaFuncSetAttribute(k_probe_spectrum<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)probe_smem()) == cudaSuccess &&
              cudaFuncSetAttribute(k_probe_grad<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)probe_smem()) == cudaSuccess;
    if constexpr (N != 256) {
      ok = ok && cudaFuncSetAttribute(k_loss<N, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)loss_smem_bytes<N>()) == cudaSuccess;
      ok = ok && cudaFuncSetAttribute(k_loss<N, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)loss_smem_bytes<N>()) == cudaSuccess;
    }
#if PTY_CARVEOUT
    // One N = 128 wave kernel CTA per SM: ask for the smallest shared-memory carve-out that holds it,
    // so the rest of the SM's on-chip memory serves as L1 for the loads in flight.
    if constexpr (N == 128) {
      int dev = 0, smem_sm = 0;
      ok = ok && cudaGetDevice(&dev) == cudaSuccess &&
           cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
           smem_sm > 0;
      auto pct = [&](size_t bytes) { return (int)((100 * (bytes + 1024) + smem_sm - 1) / (size_t)smem_sm); };
      ok = ok &&
           cudaFuncSetAttribute(fwd_kernel(), cudaFuncAttributePreferredSharedMemoryCarveout,
                                pct(fwd_kernel_smem_bytes<N>())) == cudaSuccess &&
           cudaFuncSetAttribute(adj_kernel(), cudaFuncAttributePreferredSharedMemoryCarveout,
                                pct(adj_smem_bytes<N, TA>())) == cudaSuccess;
    }
#endif
    if (!ok) {
      set_error("cudaFuncSetAttribute failed: %s", cudaGetErrorString(cudaGetLastError()));
      return PTY_ECUDA;
    }
    return PTY_OK;
  }
  static size_t probe_smem() { return sizeof(float2) * ((size_t)wave_rows<N>() * (N + 1) + N); }
  unsigned object_blocks() const {
    const size_t nobj = (size_t)pb.Ko * pb.Nz * pb.H * pb.W;
    return (unsigned)((nobj + 255) / 256 < 152 * 16 ? (nobj + 255) / 256 : 152 * 16);
  }

  FwdArgs fwd_args() const {
    FwdArgs fa;
    fa.M = pb.M;
    fa.Ko = pb.Ko;
    fa.Nz = pb.Nz;
    fa.H = pb.H;
    fa.W = pb.W;
    fa.Ntot = pb.Ntot;
    fa.global_tilt = pb.global_tilt;
    fa.dx = pb.dx;
    fa.lam = pb.lam;
    fa.idx = pb.idx;
    fa.pos = pb.pos;
    fa.tilt = pb.tilt;
    fa.dz = pb.dz;
    fa.T = ws.T;
    fa.Phat = ws.Phat;
    fa.ckpt = nullptr;
    fa.vhat = nullptr;
    fa.anchors = nullptr;
    fa.kstride = K;
    fa.Psi = save ? ws.Psi : nullptr;
    fa.Imode = ws.Imode;
    fa.status = ws.status;
    fa.s0 = 0;
    fa.s1 = pb.Nz;
    return fa;
  }

  // T and probe spectra (start of every forward).
  int forward_begin() {
    const size_t nobj = (size_t)pb.Ko * pb.Nz * pb.H * pb.W;
    prof_begin(st);
    k_prepare_object<<<object_blocks(), 256, 0, st>>>(pb.amp, pb.phase, ws.T, nullptr, nobj);
    PTY_LAUNCH_CHECK("k_prepare_object", 0);
    PTY_LAUNCH_RC(launch_waves<C>(k_probe_spectrum<N, T>, pb.M, T, probe_smem(), st, pb.probe, ws.Phat,
                                   (float2*)nullptr),
                  "k_probe_spectrum", 1);
    return PTY_OK;
  }
  // Forward arguments with the checkpoint outputs of this pass's memory plan.
  FwdArgs fwd_args_saved() const {
    FwdArgs fa = fwd_args();
    if (save) {
      if (K == 1) {
        fa.ckpt = want_obj ? ws.ckpt : nullptr;
        fa.vhat = want_prop ? ws.vhat : nullptr;
      } else if (nseg > 1) {
        fa.anchors = ws.anchors;
      }
    }
    return fa;
  }
  // Mode sum, and the loss when I_meas is given.
  int loss_phase(const float* I_meas) {
    LossArgs la;
    la.M = pb.M * pb.Ko;  // waves summed into each pattern
    la.Ntot = pb.Ntot;
    la.status = ws.status;
    la.loss = pb.loss;
    la.p = pb.p;
    la.eps = pb.eps;
    la.idx = pb.idx;
    la.Imode = ws.Imode;
    la.I_meas = I_meas;
    la.I_model = pb.I_model;
    la.u = I_meas ? ws.u : nullptr;
    la.lpart = I_meas ? ws.lpart : nullptr;
    const bool pac = I_meas && pb.w_pac > 0.f && ws.pac;
    la.pac = pac ? ws.pac : nullptr;
    la.pacpart = pac ? ws.pacpart : nullptr;
    la.pac_p = pb.p_pac;
    if (pac && cudaMemsetAsync(ws.pac, 0, sizeof(float) * 2 * NN, st) != cudaSuccess) return memset_failed();
    if constexpr (N == 256) {
      (pac ? k_loss_gather<N, T, true> : k_loss_gather<N, T, false>)<<<pb.B, T, 0, st>>>(la);
    } else {
      (pac ? k_loss<N, T, true> : k_loss<N, T, false>)<<<pb.B, T, loss_smem_bytes<N>(), st>>>(la);
    }
    PTY_LAUNCH_CHECK("k_loss", 3);
    if (I_meas) {
      k_loss_finalize<<<1, 256, 0, st>>>(ws.lpart, pb.B, pb.loss, (double)pb.B * NN, ws.scal, pb.loss_out, ws.status,
                                         pb.whole);
      PTY_LAUNCH_CHECK("k_loss_finalize", 4);
      if (pac) {
        k_pacbed<N><<<1, 1024, 0, st>>>(ws.pac, ws.pacpart, pb.B, pb.p_pac, pb.w_pac, pb.loss_out, ws.scal,
                                        ws.status);
        PTY_LAUNCH_CHECK("k_pacbed", -1);
        if (pb.mode == MODE_GRAD) {
          const size_t n = (size_t)pb.B * NN;
          k_pacbed_fold<N><<<(unsigned)((n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8), 256, 0, st>>>(
              ws.u, ws.pac + 2 * NN, ws.scal, n);
          PTY_LAUNCH_CHECK("k_pacbed_fold", -1);
        }
      }
    }
    return PTY_OK;
  }
  // T, probe spectra, the forward kernel (storing checkpoints when `save`) and the mode sum (and
  // the loss when I_meas is given).
  int forward(const float* I_meas) {
    int rc = forward_begin();
    if (rc || pb.B == 0) return rc;
    PTY_LAUNCH_RC(launch_waves<C>(fwd_kernel(), pb.B * pb.M * pb.Ko, TF, fwd_kernel_smem_bytes<N>(), st, fwd_args_saved()),
                  "k_forward", 2);
    return loss_phase(I_meas);
  }

  // This batch's loss statistics {sum I_meas^p, sum of squared residuals (Gaussian), D B}: Poisson
  // needs the measured patterns only, the Gaussian residuals need the forward model.
  int stats() {
    if (pb.loss == PTY_LOSS_POISSON) {
      if (pb.B > 0) {
        k_meas_sum<N, T><<<pb.B, T, 0, st>>>(pb.I_meas, pb.idx, pb.Ntot, pb.p, ws.lpart, ws.status);
        PTY_LAUNCH_CHECK("k_meas_sum", -1);
      }
    } else {
      int rc = forward(pb.I_meas);
      if (rc) return rc;
    }
    return stats_write();
  }
  // the per-pattern sums of the loss kernel (or k_meas_sum) into the caller's three statistics
  int stats_write() {
    k_batch_stats<<<1, 256, 0, st>>>(ws.lpart, pb.B, (double)pb.B * NN, pb.stats_out, ws.status);
    PTY_LAUNCH_CHECK("k_batch_stats", -1);
    return PTY_OK;
  }

  // dL/dI from the caller instead of the loss (the adjoint of the forward model alone).
  int external_dldi(const float* dldi) {
    if (pb.B == 0) return PTY_OK;
    const size_t n = (size_t)pb.B * NN;
    const unsigned blocks = (unsigned)((n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8);
    k_dldi_to_kspace<N><<<blocks, 256, 0, st>>>(dldi, ws.u, ws.scal, pb.B);
    PTY_LAUNCH_CHECK("k_dldi_to_kspace", -1);
    return PTY_OK;
  }

  AdjArgs adj_args() const {
    AdjArgs aa;
    aa.M = pb.M;
    aa.Ko = pb.Ko;
    aa.Nz = pb.Nz;
    aa.H = pb.H;
    aa.W = pb.W;
    aa.Ntot = pb.Ntot;
    aa.global_tilt = pb.global_tilt;
    aa.grad_mask = pb.grad_mask;
    aa.dx = pb.dx;
    aa.lam = pb.lam;
    aa.idx = pb.idx;
    aa.pos = pb.pos;
    aa.tilt = pb.tilt;
    aa.dz = pb.dz;
    aa.T = ws.T;
    aa.Phat = ws.Phat;
    aa.Psi = ws.Psi;
    aa.u = ws.u;
    aa.scal = ws.scal;
    aa.gT = ws.gT;
    aa.gPhat = ws.gPhat;
    aa.spart = ws.spart;
    aa.u_scaled = (pb.mode == MODE_GRAD && pb.w_pac > 0.f && ws.pac) ? 1 : 0;
    aa.status = ws.status;
    aa.gstate = ws.gstate;
    return aa;
  }

  // Zero the accumulators of the adjoint.
  int adjoint_begin() {
    const size_t nobj = (size_t)pb.Ko * pb.Nz * pb.H * pb.W;
    if (want_obj && cudaMemsetAsync(ws.gT, 0, sizeof(float2) * nobj, st) != cudaSuccess) return memset_failed();
    if (want_probe && cudaMemsetAsync(ws.gPhat, 0, sizeof(float2) * pb.M * NN, st) != cudaSuccess) return memset_failed();
    if (pb.B > 0 && cudaMemsetAsync(ws.spart, 0, sizeof(double) * 5 * pb.B * pb.M * pb.Ko, st) != cudaSuccess)
      return memset_failed();
    return PTY_OK;
  }

  // The adjoint kernels over all slices (segment by segment in the recompute mode).
  int adjoint_waves() {
    if (pb.B > 0) {
      AdjArgs aa = adj_args();
      if (K == 1) {
        aa.ckpt = ws.ckpt;
        aa.vhat = want_prop ? ws.vhat : nullptr;
        aa.ck_first = 0;
        aa.ck_per_wave = pb.Nz;
        aa.vh_first = 0;
        aa.vh_per_wave = pb.Nz - 1;
        aa.s0 = 0;
        aa.s1 = pb.Nz;
        PTY_LAUNCH_RC(launch_waves<C>(adj_kernel(), pb.B * pb.M * pb.Ko, TA, adj_smem_bytes<N, TA>(), st, aa),
                      "k_adjoint", 5);
      } else {
        for (int q = nseg - 1; q >= 0; --q) {
          const int s0 = q * K, s1 = (s0 + K < pb.Nz) ? s0 + K : pb.Nz;
          if (want_obj || want_prop) {
            FwdArgs fa = fwd_args();
            fa.Psi = nullptr;
            fa.anchors = ws.anchors;
            fa.ckpt = want_obj ? ws.ckpt : nullptr;
            fa.vhat = want_prop ? ws.vhat : nullptr;
            fa.s0 = s0;
            fa.s1 = s1;
            PTY_LAUNCH_RC(launch_waves<C>(recompute_kernel(), pb.B * pb.M * pb.Ko, TF, fwd_smem_bytes<N>(), st, fa),
                          "k_recompute", -1);
          }
          aa.ckpt = ws.ckpt;
          aa.vhat = want_prop ? ws.vhat : nullptr;
          aa.ck_first = s0;
          aa.ck_per_wave = K;
          aa.vh_first = s0 - 1;
          aa.vh_per_wave = K;
          aa.s0 = s0;
          aa.s1 = s1;
          PTY_LAUNCH_RC(launch_waves<C>(adj_kernel(), pb.B * pb.M * pb.Ko, TA, adj_smem_bytes<N, TA>(), st, aa),
                        "k_adjoint", q == 0 ? 5 : -1);
        }
      }
    }
    return PTY_OK;
  }

  // dL/damp, dL/dphase, dL/dprobe and the scalar gradients from the accumulators; then the
  // phase-sparsity term of the loss and its gradient.
  int finalize() {
    const int gm = pb.grad_mask;
    const size_t nobj = (size_t)pb.Ko * pb.Nz * pb.H * pb.W;
    if (want_obj) {
      k_object_grad<<<object_blocks(), 256, 0, st>>>(pb.amp, pb.phase, ws.gT, (gm & PTY_GRAD_AMP) ? pb.g_amp : nullptr,
                                                     (gm & PTY_GRAD_PHASE) ? pb.g_phase : nullptr, pb.accumulate, nobj);
      PTY_LAUNCH_CHECK("k_object_grad", 6);
    }
    if (pb.mode == MODE_GRAD && pb.w_sp > 0.f && ws.sppart && pb.B > 0) {
      // coverage count of the batch's patches, then one pass over every slice of every object mode
      if (cudaMemsetAsync(ws.cover, 0, sizeof(int) * (size_t)pb.H * (pb.W + 1), st) != cudaSuccess)
        return memset_failed();
      k_cover_marks<N><<<pb.B, N, 0, st>>>(pb.pos, pb.idx, pb.Ntot, pb.H, pb.W, ws.cover, ws.status);
      PTY_LAUNCH_CHECK("k_cover_marks", -1);
      k_cover_scan<<<(unsigned)((pb.H + 7) / 8), 256, 0, st>>>(ws.cover, pb.H, pb.W);
      PTY_LAUNCH_CHECK("k_cover_scan", -1);
      const double patch_pixels = (double)pb.B * pb.Ko * pb.Nz * NN;  // the mean's denominator
      k_sparse_sum<256><<<kSparseBlocks, 256, 0, st>>>(pb.phase, ws.cover, pb.H, pb.W, nobj, pb.p_sp, ws.sppart);
      PTY_LAUNCH_CHECK("k_sparse_sum", -1);
      k_sparse_finalize<<<1, 256, 0, st>>>(ws.sppart, kSparseBlocks, patch_pixels, pb.p_sp, pb.w_sp, pb.loss_out,
                                           ws.scal, ws.status);
      PTY_LAUNCH_CHECK("k_sparse_finalize", -1);
      if ((gm & PTY_GRAD_PHASE) && pb.g_phase) {
        if (!want_obj && !pb.accumulate &&
            cudaMemsetAsync(pb.g_phase, 0, sizeof(float) * nobj, st) != cudaSuccess)
          return memset_failed();
        k_sparse_grad<<<object_blocks(), 256, 0, st>>>(pb.phase, ws.cover, pb.H, pb.W, nobj, pb.p_sp, pb.w_sp,
                                                       ws.scal, pb.g_phase);
        PTY_LAUNCH_CHECK("k_sparse_grad", -1);
      }
    }
    if (want_probe) {
      PTY_LAUNCH_RC(launch_waves<C>(k_probe_grad<N, T>, pb.M, T, probe_smem(), st, (const float2*)ws.gPhat,
                                     pb.g_probe, pb.accumulate),
                    "k_probe_grad", 7);
    }
    if (gm & (PTY_GRAD_POS | PTY_GRAD_TILT | PTY_GRAD_DZ)) {
      if (!pb.accumulate) {
        if ((gm & PTY_GRAD_POS) && pb.g_pos &&
            cudaMemsetAsync(pb.g_pos, 0, sizeof(float) * 2 * pb.Ntot, st) != cudaSuccess)
          return memset_failed();
        if ((gm & PTY_GRAD_TILT) && pb.g_tilt && !pb.global_tilt &&
            cudaMemsetAsync(pb.g_tilt, 0, sizeof(float) * 2 * pb.Ntot, st) != cudaSuccess)
          return memset_failed();
      }
      if (pb.B > 0) {
        k_scalar_grad<<<1, 256, 0, st>>>(ws.spart, pb.idx, pb.B, pb.M * pb.Ko, pb.Ntot, pb.global_tilt, gm, pb.g_pos,
                                         pb.g_tilt, pb.g_dz, pb.accumulate);
        PTY_LAUNCH_CHECK("k_scalar_grad", 8);
      } else if (!pb.accumulate) {
        if ((gm & PTY_GRAD_DZ) && pb.g_dz && cudaMemsetAsync(pb.g_dz, 0, sizeof(float), st) != cudaSuccess)
          return memset_failed();
        if ((gm & PTY_GRAD_TILT) && pb.g_tilt && pb.global_tilt &&
            cudaMemsetAsync(pb.g_tilt, 0, 2 * sizeof(float), st) != cudaSuccess)
          return memset_failed();
      }
    }
    return PTY_OK;
  }
  int adjoint() {
    int rc = adjoint_begin();
    if (!rc) rc = adjoint_waves();
    if (!rc) rc = finalize();
    return rc;
  }
  int memset_failed() {
    set_error("cudaMemsetAsync failed: %s", cudaGetErrorString(cudaGetLastError()));
    return PTY_ECUDA;
  }
};

template <int N>
int run_pipeline(const Problem& pb) {
  Pass<N> ps(pb);
  int rc = ps.set_attributes();
  if (rc) return rc;
  switch (pb.mode) {
    case MODE_FORWARD:
    case MODE_FORWARD_SAVE:
      return ps.forward(nullptr);
    case MODE_GRAD:
      rc = ps.forward(pb.I_meas);
      if (rc) return rc;
      if (pb.B == 0 && pb.loss_out) {
        if (cudaMemsetAsync(pb.loss_out, 0, sizeof(double), pb.stream) != cudaSuccess) return ps.memset_failed();
      }
      return ps.adjoint();
    case MODE_STATS:
      return ps.stats();
    case MODE_BACKWARD:
      rc = ps.external_dldi(pb.dldi);
      if (rc) return rc;
      return ps.adjoint();
    default:
      set_error("unknown pass mode %d", pb.mode);
      return PTY_EINVAL;
  }
}

}  // namespace pty
