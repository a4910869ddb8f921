// fft_cluster.cuh -- 2D FFT of one 256 x 256 wavefield spread over a four-CTA thread-block cluster.
//
// The wave (512 KB) does not fit one SM's shared memory, so CTA q of the cluster holds rows
// [64 q, 64 q + 64) as float2 s[64][257] and the four CTAs exchange data through distributed shared
// memory.  Each CTA runs 256 threads.  Axis 0 (across the CTAs) splits as n = 8 a + b (a < 32,
// b < 8), so row n lives in CTA a / 8 at local row 8 (a % 8) + b, and bin k = k1 + 32 k2; axis 1
// (local) splits as n = 32 a' + b' (a' < 8, b' < 32), bin k = k1' + 8 k2'.  A forward transform is
// three steps, like the single-CTA FFT:
//   X1     for every (column c, b): 32-point DFT over a (eight rows from each CTA), times
//          W_256^{b k1}; result k1 goes back to the place of a = k1 (CTA k1 / 8, local row
//          8 (k1 % 8) + b).  The only step touching other CTAs' shared memory;
//   block  for every 8 x 8 block {local rows 8 g + b} x {columns 32 a' + b'}: the 8-point column
//          DFTs over b (-> k2; local row 8 g + k2 of CTA q then holds bin 8 q + g + 32 k2), then
//          the 8-point row DFTs over a' (-> k1') times W_256^{b' k1'};
//   row    for every (local row, k1'): 32-point DFT over b' (-> k2', column 32 k1' + k2').
// k-space positions: axis 0 bin k1 + 32 k2 at row 8 k1 + k2, axis 1 bin k1' + 8 k2' at column
// 32 k1' + k2'.  The inverse runs the mirror images in reverse order.  The step API is that of the
// single-CTA Fft2 in fft_smem.cuh, so the same kernels drive both: "col" is the cross-CTA step next
// to the natural layout (its hook sees 32 elements, rows 8 a + b of one column, lanes on
// consecutive columns), "row" the step next to k-space (hook on 32 consecutive positions of one
// local row, lanes on consecutive rows).  Every cross-CTA step starts and ends with a cluster
// barrier; all CTAs of a cluster run the same sequence of steps.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fft_smem.cuh"

namespace pty {

template <int T>
struct Fft2<256, T> {
  static constexpr int N = 256, L = 64, RS = N + 1;
  static constexpr int C = 4, ROWS = L;
  static_assert(T == 256, "task counts below assume 256 threads");
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

  // ---- X1 and its inverse, optionally fused around a natural-layout hook ----
  // Task (c, b): element a is row 8 a + b (CTA a / 8, local row 8 (a % 8) + b); the k-space side
  // keeps bin k1 in the same place.  INV_IN: the input is the k-space side and gets the conjugate
  // twiddle and the inverse 32-point DFT first; FWD_OUT: the forward DFT and the twiddle are
  // applied before writing back.
  template <bool INV_IN, bool FWD_OUT, bool WRITE, class H>
  __device__ static void x1_step(float2* s, const float2* tw, H& h) {
    const int q = rank();
    float2* rem[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) rem[r] = remote(s, r);
    cluster_sync();
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
      const int t = threadIdx.x + i * T;
      const int c = 64 * q + t % 64, b = t / 64;
      float2 v[32];
      if (!(std::remove_reference_t<H>::kReplaces && !INV_IN)) {
#pragma unroll
        for (int a = 0; a < 32; ++a) v[a] = rem[a / 8][(8 * (a % 8) + b) * RS + c];
      }
      if (INV_IN) {
        if (!PTY_TW_SKIP || b != 0) {
#pragma unroll
          for (int k1 = 1; k1 < 32; ++k1) v[k1] = cmulc(tw[b * k1], v[k1]);
        }
        dft<32, true>(v);
      }
      hook<32>(h, b, 8, c, 0, v);
      if (FWD_OUT) {
        dft<32, false>(v);
        if (!PTY_TW_SKIP || b != 0) {
#pragma unroll
          for (int k1 = 1; k1 < 32; ++k1) v[k1] = cmul(v[k1], tw[b * k1]);
        }
      }
      if (WRITE) {
#pragma unroll
        for (int a = 0; a < 32; ++a) rem[a / 8][(8 * (a % 8) + b) * RS + c] = v[a];
      }
    }
    cluster_sync();
  }

  // ---- the local 8 x 8 block step ----
  // Task (g, b'): local rows 8 g + (0..7) x columns 32 (0..7) + b'; one task per thread, lanes on
  // consecutive b'.
  template <bool INV>
  __device__ static void block_step(float2* s, const float2* tw) {
    const int bp = threadIdx.x % 32, g = threadIdx.x / 32;
    float2 d[8][8];  // [row digit][column digit]
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) d[r][c] = s[(8 * g + r) * RS + 32 * c + bp];
    if (!INV) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {  // 8-point column DFTs (b -> k2)
        float2 col[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) col[r] = d[r][c];
        dft<8, false>(col);
#pragma unroll
        for (int r = 0; r < 8; ++r) d[r][c] = col[r];
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) {  // 8-point row DFTs (a' -> k1'), then W_256^{b' k1'}
        dft<8, false>(d[r]);
        if (!PTY_TW_SKIP || bp != 0) {
#pragma unroll
          for (int c = 1; c < 8; ++c) d[r][c] = cmul(d[r][c], tw[bp * c]);
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        if (!PTY_TW_SKIP || bp != 0) {
#pragma unroll
          for (int c = 1; c < 8; ++c) d[r][c] = cmulc(tw[bp * c], d[r][c]);
        }
        dft<8, true>(d[r]);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float2 col[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) col[r] = d[r][c];
        dft<8, true>(col);
#pragma unroll
        for (int r = 0; r < 8; ++r) d[r][c] = col[r];
      }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) s[(8 * g + r) * RS + 32 * c + bp] = d[r][c];
    __syncthreads();
  }

  // RB, RB^-1 and the fused RB -> hook -> RB^-1.  k-space elements of task (r, k1'): positions
  // 32 k1' + k2' of local row r, global k-space row 64 q + r.
  template <bool FWD_IN, bool INV_OUT, bool WRITE, class H>
  __device__ static void rb_step(float2* s, const float2* tw, H& h) {
    const int q = rank();
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
      const int t = threadIdx.x + i * T;
      const int r = t % L, k1 = t / L;
      float2 v[32];
      if (!(std::remove_reference_t<H>::kReplaces && !FWD_IN)) {
#pragma unroll
        for (int b = 0; b < 32; ++b) v[b] = s[r * RS + 32 * k1 + b];
      }
      if (FWD_IN) dft<32, false>(v);
      hook<32>(h, 64 * q + r, 0, 32 * k1, 1, v);
      if (INV_OUT) dft<32, true>(v);
      if (WRITE) {
#pragma unroll
        for (int b = 0; b < 32; ++b) s[r * RS + 32 * k1 + b] = v[b];
      }
    }
    __syncthreads();
  }

  // ---- the step API shared with the single-CTA FFT ----
  template <class LH>
  __device__ static void col_fwd(float2* s, const float2* tw, LH& lh) {
    x1_step<false, true, true>(s, tw, lh);
  }
  __device__ static void block_fwd(float2* s, const float2* tw) { block_step<false>(s, tw); }
  template <bool WRITE, class SH>
  __device__ static void row_fwd(float2* s, SH& sh) {
    rb_step<true, false, WRITE>(s, nullptr, sh);
  }
  template <class LH>
  __device__ static void row_inv(float2* s, const float2* tw, LH& lh) {
    rb_step<false, true, true>(s, tw, lh);
  }
  __device__ static void block_inv(float2* s, const float2* tw) { block_step<true>(s, tw); }
  __device__ static void col_inv(float2* s, const float2* tw) {
    NoHook none;
    x1_step<true, false, true>(s, tw, none);
  }
  template <bool FWD, class H>
  __device__ static void col_inv_fwd(float2* s, const float2* tw, H& h) {
    x1_step<true, FWD, FWD>(s, tw, h);
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

  // Natural-layout pointwise pass: thread t owns column t % 256 and every local row.
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
  // k-space pointwise pass: thread t owns local row t % 64 and columns t / 64 + 4 i.
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
