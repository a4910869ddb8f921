// fft_cluster.cuh -- 2D FFT of one 256 x 256 wavefield spread over a thread-block cluster of C CTAs
// (C = PTY_N256_CTAS: 4 CTAs of 512 threads, or 8 of 128).
//
// The wave (512 KB) does not fit one SM's shared memory, so CTA q of the cluster holds the L = 256 / C
// rows [L q, L q + L) as float2 s[L][257] and the CTAs exchange data through distributed shared
// memory.  Axis 0 (across the CTAs) splits as n = 16 a + b (a, b = 0..15), so row n lives in CTA
// a / AP at local row 16 (a % AP) + b (AP = 16 / C values of a per CTA), and bin k = k1 + 16 k2:
//   X1   for every (column c, b): 16-point DFT over a (AP rows from each CTA), times W_256^{b k1};
//        result k1 goes back to the place of a = k1 (CTA k1 / AP, local row 16 (k1 % AP) + b).
//        The only step touching other CTAs' shared memory;
//   X2   for every (column c, k1): 16-point DFT over b (16 consecutive local rows); local row
//        16 (k1 % AP) + k2 of CTA k1 / AP then holds bin k1 + 16 k2, i.e. global position 16 k1 + k2.
// Axis 1 (local to each CTA) splits as n = 16 a + b:
//   RA   16-point DFT over a, times W_256^{b k1};   RB   16-point DFT over b.
// The forward transform runs X1, X2, RA, RB (natural -> k-space), the inverse the mirror images in
// reverse order.  The step API is that of the single-CTA Fft2 in fft_smem.cuh, so the same kernels
// drive both: "col" is the cross-CTA step next to the natural layout (its hook sees 16 elements,
// rows 16 a + b of one column, lanes on consecutive columns), "block" the two local steps in
// between, "row" the step next to k-space (hook on 16 consecutive positions of one local row, lanes
// on consecutive rows).  Every cross-CTA step starts and ends with a cluster barrier; all CTAs of a
// cluster run the same sequence of steps.  Every step has L N / 16 tasks per CTA.  The local steps
// (X2, RA, RB, the k-space pass) touch 16-row blocks of one CTA only, so with PTY_GROUPS256 = G > 1
// each of G thread groups works on its own L / G rows and waits only for its own threads.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fft_smem.cuh"

// 1: every step reads both of a thread's tasks before it transforms either, so the second task's
// shared-memory (or remote) loads are in flight while the first is transformed; the tasks of a
// step touch disjoint elements.  0: one task at a time.
#ifndef PTY_PRELOAD
#define PTY_PRELOAD 1
#endif
// 1: steps with a hook that declares kPreload read both tasks first too (large-window forward: 36.5
// against 32.8 ms, from register spills; off)
#ifndef PTY_PRELOAD_HOOKS
#define PTY_PRELOAD_HOOKS 0
#endif

// CTAs per 256 x 256 wave: 4 (one 132 KB CTA of 512 threads per SM) or 8 (66 KB CTAs of 128
// threads, up to three per SM from different clusters)
#ifndef PTY_N256_CTAS
#define PTY_N256_CTAS 4
#endif

// Thread groups of the local steps (1, 2 or 4): group g of the CTA's threads owns local rows
// [g L / G, (g + 1) L / G), and every step between two cross-CTA steps touches one group's rows
// only, so such a step ends on the group's own named barrier instead of the CTA's.  Large-window
// workload: forward 32.39 / 32.82 / 31.25 ms and adjoint 42.40 / 42.15 / 42.21 ms at 1 / 2 / 4.
#ifndef PTY_GROUPS256
#define PTY_GROUPS256 4
#endif

namespace pty {

// A step's two tasks per thread: load(i, v) reads task i into v[16], work(i, v) transforms it and
// writes it back.  PRE: both loads first (steps without a hook; a hook's own registers and loads
// would not fit beside two tasks at 128 registers per thread).
template <bool PRE, class Load, class Work>
__device__ __forceinline__ void two_tasks(Load&& load, Work&& work) {
  if constexpr (PRE) {
    float2 v[2][16];
    load(0, v[0]);
    load(1, v[1]);
    work(0, v[0]);
    work(1, v[1]);
  } else {
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
      float2 v[16];
      load(i, v);
      work(i, v);
    }
  }
}

// NT tasks per thread, two at a time through two_tasks.
template <int NT, bool PRE, class Load, class Work>
__device__ __forceinline__ void run_tasks(Load&& load, Work&& work) {
  static_assert(NT % 2 == 0, "tasks per thread");
#pragma unroll 1
  for (int i0 = 0; i0 < NT; i0 += 2)
    two_tasks<PRE>([&](int i, float2* v) { load(i0 + i, v); }, [&](int i, float2* v) { work(i0 + i, v); });
}

template <int T>
struct Fft2<256, T> {
  static constexpr int N = 256, C = PTY_N256_CTAS, L = N / C, RS = N + 1, ROWS = L;
  static constexpr int AP = 16 / C;                    // values of a (rows 16 a + b) per CTA
  static constexpr int TASKS = L * N / 16, NT = TASKS / T;  // tasks per step per CTA, per thread
  static_assert((C == 4 || C == 8) && TASKS % T == 0 && NT % 2 == 0, "cluster shape");
  static constexpr int G = PTY_GROUPS256, TG = T / G, RG = L / G;  // groups, their threads and rows
  static_assert(T % G == 0 && (L / 16) % G == 0 && TG % 32 == 0, "thread groups");
  template <class H>
  static constexpr bool kPlain = std::is_same_v<std::decay_t<H>, NoHook>;
  // Both tasks of a step may be read first when the step has no hook, or a hook that declares
  // kPreload (one light enough to run beside two tasks' registers).
  template <class H>
  __host__ __device__ static constexpr bool preload_ok() {
    if constexpr (kPlain<H>) return true;
    else return PTY_PRELOAD_HOOKS && std::decay_t<H>::kPreload;
  }

  __device__ static int rank() { return (int)cooperative_groups::this_cluster().block_rank(); }
  __device__ static int grp() { return G == 1 ? 0 : (int)threadIdx.x / TG; }
  __device__ static int gtid() { return G == 1 ? (int)threadIdx.x : (int)threadIdx.x % TG; }
  // end of a local step: the group's barrier (named barrier 1 + g; 0 is the CTA's)
  __device__ static void group_sync() {
#ifdef __CUDA_ARCH__
    if constexpr (G > 1) {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / TG), "r"(TG) : "memory");
      return;
    }
#endif
    __syncthreads();
  }
  // task i of this thread in X2: column c, 16-row block blk (the group's blocks only)
  __device__ static void x2_task(int i, int& c, int& blk) {
    const int t = gtid() + i * TG;
    c = t % N;
    blk = grp() * (L / 16 / G) + t / N;
  }
  // task i of this thread in RA / RB: local row r (the group's rows only) and digit d
  __device__ static void row_task(int i, int& r, int& d) {
    const int t = gtid() + i * TG;
    r = grp() * RG + t % RG;
    d = t / RG;
  }
  __device__ static void cluster_sync() { cooperative_groups::this_cluster().sync(); }
  __device__ static float2* remote(float2* s, int q) { return cooperative_groups::this_cluster().map_shared_rank(s, q); }

  template <int K, class H>
  __device__ static __forceinline__ void hook(H& h, int row0, int rs, int col0, int cs, float2* v) {
    if constexpr (!kPlain<H>) {
      constexpr int KC = std::decay_t<H>::kChunk < K ? std::decay_t<H>::kChunk : K;
      static_assert(K % KC == 0, "a chunk must divide the task");
#pragma unroll
      for (int q = 0; q < K; q += KC) h.template operator()<KC>(row0 + q * rs, rs, col0 + q * cs, cs, v + q);
    }
  }

  // ---- X1 and its inverse, optionally fused around a natural-layout hook ----
  // Task (c, b): element a is row 16 a + b (CTA a / 4, local row 16 (a % 4) + b); the k-space side
  // keeps bin k1 in the same place.  INV_IN: the input is the k-space side and gets the conjugate
  // twiddle and the inverse 16-point DFT first; FWD_OUT: the forward DFT and the twiddle are
  // applied before writing back.
  template <bool INV_IN, bool FWD_OUT, bool WRITE, class H>
  __device__ static void x1_step(float2* s, const float2* tw, H& h) {
    const int q = rank();
    float2* rem[C];
#pragma unroll
    for (int r = 0; r < C; ++r) rem[r] = remote(s, r);
    cluster_sync();
    constexpr int CW = N / C;  // columns of the cross step's tasks in each CTA
    run_tasks<NT, PTY_PRELOAD && preload_ok<H>()>(
        [&](int i, float2* v) {
          const int t = threadIdx.x + i * T, c = CW * q + t % CW, b = t / CW;
          if (!(std::remove_reference_t<H>::kReplaces && !INV_IN)) {
#pragma unroll
            for (int a = 0; a < 16; ++a) v[a] = rem[a / AP][(16 * (a % AP) + b) * RS + c];
          }
        },
        [&](int i, float2* v) {
          const int t = threadIdx.x + i * T, c = CW * q + t % CW, b = t / CW;
          if (INV_IN) {
            if (!PTY_TW_SKIP || b != 0) {
#pragma unroll
              for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmulc(tw[b * k1], v[k1]);
            }
            dft<16, true>(v);
          }
          hook<16>(h, b, 16, c, 0, v);
          if (FWD_OUT) {
            dft<16, false>(v);
            if (!PTY_TW_SKIP || b != 0) {
#pragma unroll
              for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw[b * k1]);
            }
          }
          if (WRITE) {
#pragma unroll
            for (int a = 0; a < 16; ++a) rem[a / AP][(16 * (a % AP) + b) * RS + c] = v[a];
          }
        });
    cluster_sync();
  }

  // ---- local steps ----
  // X2: task (c, g) for column c and local row group g (k1 % AP): 16-point DFT over the rows
  // 16 g + b (b -> k2), no twiddle after it.
  template <bool INV>
  __device__ static void x2_step(float2* s) {
    run_tasks<NT, PTY_PRELOAD != 0>(
        [&](int i, float2* v) {
          int c, g;
          x2_task(i, c, g);
#pragma unroll
          for (int b = 0; b < 16; ++b) v[b] = s[(16 * g + b) * RS + c];
        },
        [&](int i, float2* v) {
          int c, g;
          x2_task(i, c, g);
          dft<16, INV>(v);
#pragma unroll
          for (int b = 0; b < 16; ++b) s[(16 * g + b) * RS + c] = v[b];
        });
    group_sync();
  }
  __device__ static void ra_fwd(float2* s, const float2* tw) {
    run_tasks<NT, PTY_PRELOAD != 0>(
        [&](int i, float2* v) {
          int r, b;
          row_task(i, r, b);
#pragma unroll
          for (int a = 0; a < 16; ++a) v[a] = s[r * RS + 16 * a + b];
        },
        [&](int i, float2* v) {
          int r, b;
          row_task(i, r, b);
          dft<16, false>(v);
          if (!PTY_TW_SKIP || b != 0) {
#pragma unroll
            for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw[b * k1]);
          }
#pragma unroll
          for (int k1 = 0; k1 < 16; ++k1) s[r * RS + 16 * k1 + b] = v[k1];
        });
    group_sync();
  }
  __device__ static void ra_inv(float2* s, const float2* tw) {
    run_tasks<NT, PTY_PRELOAD != 0>(
        [&](int i, float2* v) {
          int r, b;
          row_task(i, r, b);
#pragma unroll
          for (int k1 = 0; k1 < 16; ++k1) v[k1] = s[r * RS + 16 * k1 + b];
        },
        [&](int i, float2* v) {
          int r, b;
          row_task(i, r, b);
          if (!PTY_TW_SKIP || b != 0) {
#pragma unroll
            for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmulc(tw[b * k1], v[k1]);
          }
          dft<16, true>(v);
#pragma unroll
          for (int a = 0; a < 16; ++a) s[r * RS + 16 * a + b] = v[a];
        });
    group_sync();
  }
  // RB, RB^-1 and the fused RB -> hook -> RB^-1.  k-space elements of task (r, k1): positions
  // 16 k1 + k2 of local row r, global k-space row L q + r.
  template <bool FWD_IN, bool INV_OUT, bool WRITE, class H>
  __device__ static void rb_step(float2* s, const float2* tw, H& h) {
    const int q = rank();
    run_tasks<NT, PTY_PRELOAD && preload_ok<H>()>(
        [&](int i, float2* v) {
          int r, k1;
          row_task(i, r, k1);
          if (!(std::remove_reference_t<H>::kReplaces && !FWD_IN)) {
#pragma unroll
            for (int b = 0; b < 16; ++b) v[b] = s[r * RS + 16 * k1 + b];
          }
        },
        [&](int i, float2* v) {
          int r, k1;
          row_task(i, r, k1);
          if (FWD_IN) dft<16, false>(v);
          hook<16>(h, L * q + r, 0, 16 * k1, 1, v);
          if (INV_OUT) dft<16, true>(v);
          if (WRITE) {
#pragma unroll
            for (int b = 0; b < 16; ++b) s[r * RS + 16 * k1 + b] = v[b];
          }
        });
    group_sync();
  }

  // ---- the step API shared with the single-CTA FFT ----
  template <class LH>
  __device__ static void col_fwd(float2* s, const float2* tw, LH& lh) {
    x1_step<false, true, true>(s, tw, lh);
  }
  __device__ static void block_fwd(float2* s, const float2* tw) {
    x2_step<false>(s);
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
    x2_step<true>(s);
  }
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
    if constexpr (G > 1) __syncthreads();  // the caller may read any row
  }
  template <class LH = NoHook>
  __device__ static void inverse(float2* s, const float2* tw, LH&& load = LH()) {
    row_inv(s, tw, load);
    block_inv(s, tw);
    col_inv(s, tw);
  }

  // Natural-layout pointwise pass.  T >= N: thread t owns column t % 256 and local rows
  // t / 256 + (T / N) i; T < N: thread t owns columns t + T h and every local row.
  template <int U, class H>
  __device__ static void pointwise(float2* s, H& h) {
    if constexpr (G > 1) __syncthreads();  // reads every group's rows
    const int g0 = L * rank();
    if constexpr (T >= N) {
      constexpr int NE = L * N / T, RPI = T / N;
      static_assert(NE % U == 0, "batch must divide the elements per thread");
      const int c = threadIdx.x % N, r0 = threadIdx.x / N;
#pragma unroll 1
      for (int i0 = 0; i0 < NE; i0 += U) {
        float2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = s[(r0 + (i0 + u) * RPI) * RS + c];
        h.template operator()<U>(g0 + r0 + i0 * RPI, RPI, c, 0, v);
#pragma unroll
        for (int u = 0; u < U; ++u) s[(r0 + (i0 + u) * RPI) * RS + c] = v[u];
      }
    } else {
      static_assert(L % U == 0, "batch must divide the rows");
#pragma unroll 1
      for (int hc = 0; hc < N / T; ++hc) {
        const int c = threadIdx.x + hc * T;
#pragma unroll 1
        for (int i0 = 0; i0 < L; i0 += U) {
          float2 v[U];
#pragma unroll
          for (int u = 0; u < U; ++u) v[u] = s[(i0 + u) * RS + c];
          h.template operator()<U>(g0 + i0, 1, c, 0, v);
#pragma unroll
          for (int u = 0; u < U; ++u) s[(i0 + u) * RS + c] = v[u];
        }
      }
    }
    __syncthreads();
  }
  // k-space pointwise pass: thread j of group g owns local row g RG + j % RG and columns
  // j / RG + (T / L) i.
  template <int U, class H>
  __device__ static void pointwise_k(float2* s, H& h) {
    constexpr int NE = L * N / T, CPI = T / L;
    static_assert(NE % U == 0 && TG / RG == CPI, "batch must divide the elements per thread");
    const int r = grp() * RG + gtid() % RG, c0 = gtid() / RG, g = L * rank() + r;
#pragma unroll 1
    for (int i0 = 0; i0 < NE; i0 += U) {
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = s[r * RS + c0 + (i0 + u) * CPI];
      h.template operator()<U>(g, 0, c0 + i0 * CPI, CPI, v);
#pragma unroll
      for (int u = 0; u < U; ++u) s[r * RS + c0 + (i0 + u) * CPI] = v[u];
    }
    group_sync();
  }
};

}  // namespace pty
