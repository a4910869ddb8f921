// fft_cluster.cuh -- 2D FFT of one 256 x 256 wavefield spread over a four-CTA thread-block cluster.
//
// The wave (512 KB) does not fit one SM's shared memory, so CTA q of the cluster holds rows
// [64 q, 64 q + 64) as float2 s[64][257] and the four CTAs exchange data through distributed shared
// memory.  Along axis 0 the split is n = 64 n1 + n2 (n1 = the CTA, n2 = its local row):
//   C1   for every (local row n2, column c): 4-point DFT over the four CTAs, times W_256^{n2 k1},
//        result k1 written to CTA k1 (the only step touching other CTAs' shared memory);
//   C2a  16-point DFT over the local rows n2 = 4 m1 + m2 (over m1), times W_64^{m2 j1};
//   C2b  4-point DFT over m2: local position 4 j1 + j2 of CTA q holds bin q + 4 j1 + 64 j2.
// Along axis 1 (local to each CTA) n = 16 a + b:
//   RA   16-point DFT over a, times W_256^{b k1};   RB   16-point DFT over b.
// The forward transform runs C1, C2a, C2b, RA, RB (natural -> k-space), the inverse the mirror
// images in reverse order.  The step API is that of the single-CTA Fft2 in fft_smem.cuh, so the
// same kernels drive both: "col" is the cross-CTA step next to the natural layout (its hook sees 4
// elements, rows 64 n1 + n2 of one column, lanes on consecutive columns), "block" the three local
// steps in between, "row" the step next to k-space (hook on 16 consecutive positions of one local
// row, lanes on consecutive rows).  Every cross-CTA step starts and ends with a cluster barrier;
// all CTAs of a cluster run the same sequence of steps.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fft_smem.cuh"

// Tasks of the cross-CTA step unrolled together (each thread runs eight; unrolling lets the loads of
// several tasks, remote and in a hook, be in flight at once).
#ifndef PTY_C1_UNROLL
#define PTY_C1_UNROLL 1
#endif

namespace pty {

constexpr int kC1Unroll = PTY_C1_UNROLL;

template <int T>
struct Fft2<256, T> {
  static constexpr int N = 256, L = 64, RS = N + 1;
  static constexpr int C = 4, ROWS = L;
  static_assert(T == 512, "task counts below assume 512 threads");
  template <class H>
  static constexpr bool kPlain = std::is_same_v<std::decay_t<H>, NoHook>;

  __device__ static int rank() { return (int)cooperative_groups::this_cluster().block_rank(); }
  __device__ static void cluster_sync() { cooperative_groups::this_cluster().sync(); }
  __device__ static float2* remote(float2* s, int q) { return cooperative_groups::this_cluster().map_shared_rank(s, q); }

  template <int K, class H>
  __device__ static __forceinline__ void hook(H& h, int row0, int rs, int col0, int cs, float2* v) {
    if constexpr (!kPlain<H>) {
      constexpr int KC = std::decay_t<H>::kChunk < K ? std::decay_t<H>::kChunk : K;
#pragma unroll
      for (int q = 0; q < K; q += KC) h.template operator()<KC>(row0 + q * rs, rs, col0 + q * cs, cs, v + q);
    }
  }

  // ---- C1 and its inverse, optionally fused around a natural-layout hook ----
  // INV_IN: the input is k-space side (after C2a^-1) and gets the inverse 4-point DFT first;
  // FWD_OUT: the forward 4-point DFT is applied before writing back.  Natural-layout elements are
  // rows 64 n1 + n2 (n1 = 0..3) of column c.
  template <bool INV_IN, bool FWD_OUT, bool WRITE, class H>
  __device__ static void c1_step(float2* s, const float2* tw, H& h) {
    const int q = rank();
    float2* rem[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) rem[r] = remote(s, r);
    cluster_sync();
#pragma unroll kC1Unroll
    for (int i = 0; i < 8; ++i) {
      const int t = threadIdx.x + i * T;
      const int c = 64 * q + t % 64, n2 = t / 64;
      const int e = n2 * RS + c;
      float2 v[4];
      if (!(std::remove_reference_t<H>::kReplaces && !INV_IN)) {
#pragma unroll
        for (int r = 0; r < 4; ++r) v[r] = rem[r][e];
      }
      if (INV_IN) {
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) v[k1] = cmulc(tw[n2 * k1], v[k1]);
        dft<4, true>(v);
      }
      hook<4>(h, n2, L, c, 0, v);
      if (FWD_OUT) {
        dft<4, false>(v);
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) v[k1] = cmul(v[k1], tw[n2 * k1]);
      }
      if (WRITE) {
#pragma unroll
        for (int r = 0; r < 4; ++r) rem[r][e] = v[r];
      }
    }
    cluster_sync();
  }

  // ---- local steps ----
  __device__ static void c2a_fwd(float2* s, const float2* tw) {
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
      const int t = threadIdx.x + i * T;
      const int c = t % N, m2 = t / N;
      float2 v[16];
#pragma unroll
      for (int m1 = 0; m1 < 16; ++m1) v[m1] = s[(4 * m1 + m2) * RS + c];
      dft<16, false>(v);
#pragma unroll
      for (int j1 = 1; j1 < 16; ++j1) v[j1] = cmul(v[j1], tw[4 * m2 * j1]);
#pragma unroll
      for (int j1 = 0; j1 < 16; ++j1) s[(4 * j1 + m2) * RS + c] = v[j1];
    }
    __syncthreads();
  }
  __device__ static void c2a_inv(float2* s, const float2* tw) {
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
      const int t = threadIdx.x + i * T;
      const int c = t % N, m2 = t / N;
      float2 v[16];
#pragma unroll
      for (int j1 = 0; j1 < 16; ++j1) v[j1] = s[(4 * j1 + m2) * RS + c];
#pragma unroll
      for (int j1 = 1; j1 < 16; ++j1) v[j1] = cmulc(tw[4 * m2 * j1], v[j1]);
      dft<16, true>(v);
#pragma unroll
      for (int m1 = 0; m1 < 16; ++m1) s[(4 * m1 + m2) * RS + c] = v[m1];
    }
    __syncthreads();
  }
  template <bool INV>
  __device__ static void c2b(float2* s) {
#pragma unroll 2
    for (int i = 0; i < 8; ++i) {
      const int t = threadIdx.x + i * T;
      const int c = t % N, j1 = t / N;
      float2 v[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) v[m] = s[(4 * j1 + m) * RS + c];
      dft<4, INV>(v);
#pragma unroll
      for (int m = 0; m < 4; ++m) s[(4 * j1 + m) * RS + c] = v[m];
    }
    __syncthreads();
  }
  __device__ static void ra_fwd(float2* s, const float2* tw) {
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
      const int t = threadIdx.x + i * T;
      const int r = t % L, b = t / L;
      float2 v[16];
#pragma unroll
      for (int a = 0; a < 16; ++a) v[a] = s[r * RS + 16 * a + b];
      dft<16, false>(v);
#pragma unroll
      for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw[b * k1]);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) s[r * RS + 16 * k1 + b] = v[k1];
    }
    __syncthreads();
  }
  __device__ static void ra_inv(float2* s, const float2* tw) {
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
      const int t = threadIdx.x + i * T;
      const int r = t % L, b = t / L;
      float2 v[16];
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) v[k1] = s[r * RS + 16 * k1 + b];
      dft<16, true>(v);
#pragma unroll
      for (int a = 0; a < 16; ++a) s[r * RS + 16 * a + b] = v[a];
    }
    __syncthreads();
  }
  // RB, RB^-1 and the fused RB -> hook -> RB^-1.  k-space elements of task (r, k1): positions
  // 16 k1 + k2 of local row r, global k-space row 64 q + r.
  template <bool FWD_IN, bool INV_OUT, bool WRITE, class H>
  __device__ static void rb_step(float2* s, const float2* tw, H& h) {
    const int q = rank();
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
      const int t = threadIdx.x + i * T;
      const int r = t % L, k1 = t / L;
      float2 v[16];
      if (!(std::remove_reference_t<H>::kReplaces && !FWD_IN)) {
#pragma unroll
        for (int b = 0; b < 16; ++b) v[b] = s[r * RS + 16 * k1 + b];
      }
      if (FWD_IN) dft<16, false>(v);
      hook<16>(h, 64 * q + r, 0, 16 * k1, 1, v);
      if (INV_OUT) {
        dft<16, true>(v);
#pragma unroll
        for (int b = 1; b < 16; ++b) v[b] = cmulc(tw[b * k1], v[b]);
      }
      if (WRITE) {
#pragma unroll
        for (int b = 0; b < 16; ++b) s[r * RS + 16 * k1 + b] = v[b];
      }
    }
    __syncthreads();
  }

  // ---- the step API shared with the single-CTA FFT ----
  template <class LH>
  __device__ static void col_fwd(float2* s, const float2* tw, LH& lh) {
    c1_step<false, true, true>(s, tw, lh);
  }
  __device__ static void block_fwd(float2* s, const float2* tw) {
    c2a_fwd(s, tw);
    c2b<false>(s);
    ra_fwd(s, tw);
  }
  template <bool WRITE, class SH>
  __device__ static void row_fwd(float2* s, SH& sh) {
    rb_step<true, false, WRITE>(s, nullptr, sh);
  }
  template <class LH>
  __device__ static void row_inv(float2* s, const float2* tw, LH& lh) {
    rb_step<false, true, true>(s, tw, lh);
  }
  __device__ static void block_inv(float2* s, const float2* tw) {
    ra_inv(s, tw);
    c2b<true>(s);
    c2a_inv(s, tw);
  }
  __device__ static void col_inv(float2* s, const float2* tw) {
    NoHook none;
    c1_step<true, false, true>(s, tw, none);
  }
  template <bool FWD, class H>
  __device__ static void col_inv_fwd(float2* s, const float2* tw, H& h) {
    c1_step<true, FWD, FWD>(s, tw, h);
  }
  template <class H>
  __device__ static void row_fwd_inv(float2* s, const float2* tw, H& h) {
    rb_step<true, true, true>(s, tw, h);
  }
  template <bool WRITE = true, class LH = NoHook, class SH = NoHook>
  __device__ static void forward(float2* s, const float2* tw, LH&& load = LH(), SH&& store = SH()) {
    col_fwd(s, tw, load);
    block_fwd(s, tw);
    row_fwd<WRITE>(s, store);
  }
  template <class LH = NoHook>
  __device__ static void inverse(float2* s, const float2* tw, LH&& load = LH()) {
    row_inv(s, tw, load);
    block_inv(s, tw);
    col_inv(s, tw);
  }

  // Natural-layout pointwise pass: thread t owns column t % 256 and local rows t / 256 + 2 i.
  template <int U, class H>
  __device__ static void pointwise(float2* s, H& h) {
    constexpr int NE = L * N / T, RPI = T / N;
    static_assert(NE % U == 0, "batch must divide the elements per thread");
    const int c = threadIdx.x % N, r0 = threadIdx.x / N, g0 = L * rank();
#pragma unroll 1
    for (int i0 = 0; i0 < NE; i0 += U) {
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = s[(r0 + (i0 + u) * RPI) * RS + c];
      h.template operator()<U>(g0 + r0 + i0 * RPI, RPI, c, 0, v);
#pragma unroll
      for (int u = 0; u < U; ++u) s[(r0 + (i0 + u) * RPI) * RS + c] = v[u];
    }
    __syncthreads();
  }
  // k-space pointwise pass: thread t owns local row t % 64 and columns t / 64 + 8 i.
  template <int U, class H>
  __device__ static void pointwise_k(float2* s, H& h) {
    constexpr int NE = L * N / T, CPI = T / L;
    static_assert(NE % U == 0, "batch must divide the elements per thread");
    const int r = threadIdx.x % L, c0 = threadIdx.x / L, g = L * rank() + r;
#pragma unroll 1
    for (int i0 = 0; i0 < NE; i0 += U) {
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = s[r * RS + c0 + (i0 + u) * CPI];
      h.template operator()<U>(g, 0, c0 + i0 * CPI, CPI, v);
#pragma unroll
      for (int u = 0; u < U; ++u) s[r * RS + c0 + (i0 + u) * CPI] = v[u];
    }
    __syncthreads();
  }
};

}  // namespace pty
