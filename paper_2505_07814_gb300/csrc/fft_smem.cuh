// fft_smem.cuh -- 2D complex FFT of one N x N wavefield held in shared memory by one CTA.
//
// Layout.  The wave is float2 s[N][N + 1]: one complex pad per row makes the row stride odd, so a
// warp walking along a row (32 consecutive columns) and a warp walking down 32 rows of one column
// both touch 32 distinct bank pairs.
//
// Algorithm.  N = A * 4.  Along axis 0 (columns) the split is n = 4 n1 + n2, k = k1 + A k2; along
// axis 1 (rows) it is n = A n1 + n2, k = k1 + 4 k2.  A forward 2D transform is three steps, each
// one read and one write of shared memory, with one barrier after each:
//   col    for every (column, n2): A-point DFT over n1, times W_N^{n2 k1};
//   block  for every 4 x 4 block {rows 4 k1 + q} x {cols A p + n2}: the 4-point column DFTs
//          (q -> k2), then the 4-point row DFTs (p -> k1) times W_N^{n2 k1};
//   row    for every (row, k1): A-point DFT over n2.
// The small DFTs run in registers.  The output stays in the digit order the split produces
// (k-space layout below): pointwise k-space work is done in that order and the inverse (the same
// steps mirrored) consumes it, so no reordering pass is ever needed.  Lanes of a warp always own
// consecutive columns (col, block) or consecutive rows (row), so shared memory is conflict-free.
// Neither direction normalises (the inverse is the plain conjugate-sign sum).
//
// k-space layout: s[p0][p1]; axis-0 position p0 = 4 k1 + k2 holds bin k1 + A k2, axis-1 position
// p1 = A k1 + k2 holds bin k1 + 4 k2.  Global k-space buffers are stored transposed, element
// (p0, p1) at p1 * N + p0, so that the row step's lanes (consecutive p0) access them coalesced.
//
// Twiddles come from a per-CTA table tw[t] = exp(-2 pi i t / N) built with sincospif().
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace pty {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// cos(2 pi e / 32) for e = 0..8 (the rest follow by symmetry).
__device__ __forceinline__ constexpr float cos32(int e) {
  return e == 0 ? 1.0f
       : e == 1 ? 0.98078528040323043f
       : e == 2 ? 0.92387953251128676f
       : e == 3 ? 0.83146961230254524f
       : e == 4 ? 0.70710678118654752f
       : e == 5 ? 0.55557023301960222f
       : e == 6 ? 0.38268343236508977f
       : e == 7 ? 0.19509032201612826f
                : 0.0f;
}

// z * W_R^k with W_R = exp(-2 pi i / R) (forward) or its conjugate (INV), for R | 32; k is a
// compile-time constant once the calling loops are unrolled, so everything folds to constants.
template <int R, bool INV>
__device__ __forceinline__ float2 twmul(int k, float2 z) {
  const int e = k * (32 / R);  // angle in units of 2 pi / 32, 0 <= e < 16
  if (e == 0) return z;
  if (e == 8) return INV ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
  // W = c - i s with c = cos(2 pi e / 32), s = sin(2 pi e / 32) = cos(2 pi (8 - e) / 32)
  const float c = e < 8 ? cos32(e) : -cos32(16 - e);
  float s = e < 8 ? cos32(8 - e) : cos32(e - 8);
  if (INV) s = -s;
  return make_float2(fmaf(z.x, c, z.y * s), fmaf(z.y, c, -z.x * s));
}

// tan(2 pi e / 32) for e = 0..4.
__device__ __forceinline__ constexpr float tan32(int e) {
  return e == 0 ? 0.0f
       : e == 1 ? 0.19891236737965800607f
       : e == 2 ? 0.41421356237309503445f
       : e == 3 ? 0.66817863791929887896f
                : 1.0f;
}

// Radix-2 butterfly a <- a + z, b <- a - z with z = W_R^k b, in six fused multiply-adds for any
// rotation but 0 and -i (which cost four adds).  W = c - i s (c + i s for INV) is written as
// f (1 - i r) with |r| <= 1: f = c, r = s / c where |s| <= |c|, else f = s, r = c / s applied to
// the swapped components (the tangent-factored butterfly of Linzer and Feig, "Implementation of
// efficient FFT algorithms on fused multiply-add architectures", IEEE Trans. Signal Processing
// 41(1), 1993).  z / f then takes two FMAs, and a +- f (z / f) four; the plain product z = W b
// followed by the sum and difference takes eight instructions.
template <int R, bool INV>
__device__ __forceinline__ void bfly(int k, float2& a, float2& b) {
  const int e = k * (32 / R);  // angle in units of 2 pi / 32, 0 <= e < 16
  const float2 x = a;
  if (e == 0 || e == 8) {
    const float2 z = e == 0 ? b : (INV ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x));
    a = cadd(x, z);
    b = csub(x, z);
    return;
  }
  const int ea = e < 8 ? e : 16 - e;  // |c| = cos(2 pi ea / 32), |s| = sin(2 pi ea / 32)
  const float sc = e < 8 ? 1.0f : -1.0f, ss = INV ? -1.0f : 1.0f;  // signs of c and s
  float f;
  float2 u;  // z / f
  if (ea <= 4) {  // z = c (b.x + r b.y, b.y - r b.x), r = s / c
    const float r = sc * ss * tan32(ea);
    f = sc * cos32(ea);
    u = make_float2(fmaf(r, b.y, b.x), fmaf(-r, b.x, b.y));
  } else {  // z = s (q b.x + b.y, q b.y - b.x), q = c / s
    const float q = sc * ss * tan32(8 - ea);
    f = ss * cos32(8 - ea);
    u = make_float2(fmaf(q, b.x, b.y), fmaf(q, b.y, -b.x));
  }
  a = make_float2(fmaf(f, u.x, x.x), fmaf(f, u.y, x.y));
  b = make_float2(fmaf(-f, u.x, x.x), fmaf(-f, u.y, x.y));
}

// 1: the DFTs combine with bfly (six FMAs per rotated butterfly); 0: product then sum (eight)
#ifndef PTY_DFT_FMA
#define PTY_DFT_FMA 1
#endif

// In-register R-point DFT (R = 2 ... 32), natural order in and out, radix-2 decimation in time.
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* x) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 2) {
    const float2 a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  } else {
    float2 e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = x[2 * i];
      o[i] = x[2 * i + 1];
    }
    dft<R / 2, INV>(e);
    dft<R / 2, INV>(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
#if PTY_DFT_FMA
      bfly<R, INV>(k, e[k], o[k]);
      x[k] = e[k];
      x[k + R / 2] = o[k];
#else
      const float2 t = twmul<R, INV>(k, o[k]);
      x[k] = cadd(e[k], t);
      x[k + R / 2] = csub(e[k], t);
#endif
    }
  }
}

// Position of frequency bin k along axis 0 / axis 1 of the k-space layout, and the inverse maps.
// N <= 128: axis 0 split k = k1 + A k2 at position 4 k1 + k2, axis 1 split k = k1 + 4 k2 at A k1 + k2.
// N = 256 (four-CTA cluster, fft_cluster.cuh): both axes split k = k1 + 16 k2 at position
// 16 k1 + k2.
template <int N>
__host__ __device__ constexpr int kpos0(int k) {
  if constexpr (N == 256) return 16 * (k % 16) + k / 16;
  else return 4 * (k % (N / 4)) + k / (N / 4);
}
template <int N>
__host__ __device__ constexpr int kbin0(int p) {
  if constexpr (N == 256) return p / 16 + 16 * (p % 16);
  else return p / 4 + (N / 4) * (p % 4);
}
template <int N>
__host__ __device__ constexpr int kpos1(int k) {
  if constexpr (N == 256) return 16 * (k % 16) + k / 16;
  else return (N / 4) * (k % 4) + k / 4;
}
template <int N>
__host__ __device__ constexpr int kbin1(int p) {
  if constexpr (N == 256) return p / 16 + 16 * (p % 16);
  else return p / (N / 4) + 4 * (p % (N / 4));
}
// Index of k-space element (p0, p1) in global k-space buffers (stored transposed).
template <int N>
__host__ __device__ constexpr int kidx(int p0, int p1) {
  return p1 * N + p0;
}

// Element hooks fused into the FFT steps.  A hook sees K elements of one task in registers: element
// k sits at (row0 + k * rs, col0 + k * cs) of the array being transformed.  Load hooks run right
// after the elements are read (natural layout in a forward transform, k-space in an inverse), store
// hooks right before they are written (k-space).  A hook with kReplaces = true produces the values
// itself, so the shared-memory read is skipped.  Hooks are called on chunks of kChunk elements so
// that their global loads can be batched without holding a whole task's worth of registers.
struct NoHook {
  static constexpr bool kReplaces = false;
  static constexpr bool kPreload = true;
  static constexpr int kChunk = 1;
  template <int K>
  __device__ __forceinline__ void operator()(int, int, int, int, float2*) {}
};

// Block-step tasks read together before any is transformed, at most (1: one at a time); the
// group is the largest of 4, 2, 1 that divides the thread's tasks.  Multislice workload: forward
// 2.260 -> 2.216 ms with 4 (its four tasks), adjoint 3.463 -> 3.452 ms with 2.
#ifndef PTY_PRELOAD_BLOCK
#define PTY_PRELOAD_BLOCK 4
#endif

// 1: steps whose inter-step twiddles are all W^0 (digit n2 = 0 in the column steps, k1 = 0 in the
// row steps, warp-uniform for N >= 64) skip the multiplication (exact: it multiplies by 1)
#ifndef PTY_TW_SKIP
#define PTY_TW_SKIP 1
#endif

// Thread groups of the row-local steps (1, 2 or 4).  The block and row steps and the k-space pass
// touch groups of four rows only, so with G > 1 group g of the CTA's threads takes rows
// [g N / G, (g + 1) N / G) in those steps and they end on the group's own named barrier; the column
// steps, which mix all rows, start with the CTA's barrier.  Multislice workload: forward 2.204 /
// 2.286 / 2.281 ms and adjoint 3.453 / 3.599 / 3.551 ms at 1 / 2 / 4, so one group stays.
#ifndef PTY_GROUPS
#define PTY_GROUPS 1
#endif

template <int N, int T>
struct Fft2 {
  static constexpr int A = N / 4, RS = N + 1;
  static_assert(A == 16 || A == 32, "N = 64 or 128");
  static constexpr int C = 1, ROWS = N;  // CTAs per wave, rows of the wave held by this CTA
  __device__ static int rank() { return 0; }
  static constexpr int NCOL = 4 * N / T;    // col-step tasks per thread: (c, n2)
  static constexpr int NBLK = A * A / T;    // block-step tasks per thread: (k1, n2)
  static constexpr int NROW = 4 * N / T;    // row-step tasks per thread: (r, k1)
  static_assert(NCOL * T == 4 * N && NBLK * T == A * A, "tasks must divide the CTA");
  static constexpr int G = PTY_GROUPS, TG = T / G, RG = N / G;  // groups, their threads and rows
  static_assert(T % G == 0 && TG % 32 == 0 && A % G == 0 && TG % RG == 0 || G == 1, "thread groups");
  __device__ static int grp() { return G == 1 ? 0 : (int)threadIdx.x / TG; }
  __device__ static int gtid() { return G == 1 ? (int)threadIdx.x : (int)threadIdx.x % TG; }
  // end of a row-local step: the group's barrier (named barrier 1 + g; 0 is the CTA's)
  __device__ static void group_sync() {
#ifdef __CUDA_ARCH__
    if constexpr (G > 1) {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / TG), "r"(TG) : "memory");
      return;
    }
#endif
    __syncthreads();
  }
  // start of a step that reads every group's rows
  __device__ static void all_sync() {
    if constexpr (G > 1) __syncthreads();
  }
  template <class H>
  static constexpr bool kPlain = std::is_same_v<std::decay_t<H>, NoHook>;

  template <class H>
  __device__ static __forceinline__ void hook(H& h, int row0, int rs, int col0, int cs, float2* v) {
    if constexpr (!kPlain<H>) {
      // chunks of kChunk elements, at most the task's A
      constexpr int KC = std::decay_t<H>::kChunk < A ? std::decay_t<H>::kChunk : A;
      static_assert(A % KC == 0, "a chunk must divide the task");
#pragma unroll
      for (int q = 0; q < A; q += KC) h.template operator()<KC>(row0 + q * rs, rs, col0 + q * cs, cs, v + q);
    }
  }

  // ---- forward steps ----
  template <class LH>
  __device__ static void col_fwd(float2* s, const float2* tw, LH& lh) {
    all_sync();
#pragma unroll 1
    for (int i = 0; i < NCOL; ++i) {
      const int t = threadIdx.x + i * T;
      const int c = t % N, n2 = t / N;
      float2 v[A];
      if (!std::remove_reference_t<LH>::kReplaces) {
#pragma unroll
        for (int n1 = 0; n1 < A; ++n1) v[n1] = s[(4 * n1 + n2) * RS + c];
      }
      hook(lh, n2, 4, c, 0, v);
      dft<A, false>(v);
      if (!PTY_TW_SKIP || n2 != 0) {
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], tw[n2 * k1]);
      }
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) s[(4 * k1 + n2) * RS + c] = v[k1];
    }
    __syncthreads();
  }
  // Block tasks are read BG at a time before any is transformed, so the later tasks'
  // shared-memory loads are in flight while the first is transformed (the tasks of a step touch
  // disjoint elements).
  static constexpr int BG = (PTY_PRELOAD_BLOCK >= 4 && NBLK % 4 == 0) ? 4
                            : (PTY_PRELOAD_BLOCK >= 2 && NBLK % 2 == 0) ? 2 : 1;
  __device__ static void block_load(const float2* s, int i, float2 (&b)[4][4]) {
    const int t = gtid() + i * TG;
    const int n2 = t % A, k1 = grp() * (A / G) + t / A;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int p = 0; p < 4; ++p) b[q][p] = s[(4 * k1 + q) * RS + A * p + n2];
  }
  __device__ static void block_store(float2* s, int i, const float2 (&b)[4][4]) {
    const int t = gtid() + i * TG;
    const int n2 = t % A, k1 = grp() * (A / G) + t / A;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int p = 0; p < 4; ++p) s[(4 * k1 + q) * RS + A * p + n2] = b[q][p];
  }
  __device__ static void block_fwd(float2* s, const float2* tw) {
#pragma unroll 1
    for (int i0 = 0; i0 < NBLK; i0 += BG) {
      float2 b[BG][4][4];  // [task][q: row digit][p: column digit]
#pragma unroll
      for (int j = 0; j < BG; ++j) block_load(s, i0 + j, b[j]);
#pragma unroll
      for (int j = 0; j < BG; ++j) {
        const int n2 = (gtid() + (i0 + j) * TG) % A;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          float2 col[4] = {b[j][0][p], b[j][1][p], b[j][2][p], b[j][3][p]};
          dft<4, false>(col);
#pragma unroll
          for (int q = 0; q < 4; ++q) b[j][q][p] = col[q];
        }
        const float2 w1 = tw[n2], w2 = tw[2 * n2], w3 = tw[3 * n2];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          dft<4, false>(b[j][q]);
          b[j][q][1] = cmul(b[j][q][1], w1);
          b[j][q][2] = cmul(b[j][q][2], w2);
          b[j][q][3] = cmul(b[j][q][3], w3);
        }
        block_store(s, i0 + j, b[j]);
      }
    }
    group_sync();
  }
  template <bool WRITE, class SH>
  __device__ static void row_fwd(float2* s, SH& sh) {
#pragma unroll 1
    for (int i = 0; i < NROW; ++i) {
      const int t = gtid() + i * TG;
      const int r = grp() * RG + t % RG, k1 = t / RG;
      float2 v[A];
#pragma unroll
      for (int n2 = 0; n2 < A; ++n2) v[n2] = s[r * RS + A * k1 + n2];
      dft<A, false>(v);
      hook(sh, r, 0, A * k1, 1, v);
      if (WRITE) {
#pragma unroll
        for (int k2 = 0; k2 < A; ++k2) s[r * RS + A * k1 + k2] = v[k2];
      }
    }
    group_sync();
  }

  // ---- inverse steps (mirror images) ----
  template <class LH>
  __device__ static void row_inv(float2* s, const float2* tw, LH& lh) {
#pragma unroll 1
    for (int i = 0; i < NROW; ++i) {
      const int t = gtid() + i * TG;
      const int r = grp() * RG + t % RG, k1 = t / RG;
      float2 v[A];
      if (!std::remove_reference_t<LH>::kReplaces) {
#pragma unroll
        for (int k2 = 0; k2 < A; ++k2) v[k2] = s[r * RS + A * k1 + k2];
      }
      hook(lh, r, 0, A * k1, 1, v);
      dft<A, true>(v);
      if (!PTY_TW_SKIP || k1 != 0) {
#pragma unroll
        for (int n2 = 1; n2 < A; ++n2) v[n2] = cmulc(tw[n2 * k1], v[n2]);
      }
#pragma unroll
      for (int n2 = 0; n2 < A; ++n2) s[r * RS + A * k1 + n2] = v[n2];
    }
    group_sync();
  }
  __device__ static void block_inv(float2* s, const float2*) {
#pragma unroll 1
    for (int i0 = 0; i0 < NBLK; i0 += BG) {
      float2 b[BG][4][4];
#pragma unroll
      for (int j = 0; j < BG; ++j) block_load(s, i0 + j, b[j]);
#pragma unroll
      for (int j = 0; j < BG; ++j) {
#pragma unroll
        for (int q = 0; q < 4; ++q) dft<4, true>(b[j][q]);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          float2 col[4] = {b[j][0][p], b[j][1][p], b[j][2][p], b[j][3][p]};
          dft<4, true>(col);
#pragma unroll
          for (int q = 0; q < 4; ++q) b[j][q][p] = col[q];
        }
        block_store(s, i0 + j, b[j]);
      }
    }
    group_sync();
  }
  __device__ static void col_inv(float2* s, const float2* tw) {
    all_sync();
#pragma unroll 1
    for (int i = 0; i < NCOL; ++i) {
      const int t = threadIdx.x + i * T;
      const int c = t % N, n2 = t / N;
      float2 v[A];
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) v[k1] = s[(4 * k1 + n2) * RS + c];
      if (!PTY_TW_SKIP || n2 != 0) {
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1) v[k1] = cmulc(tw[n2 * k1], v[k1]);
      }
      dft<A, true>(v);
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) s[(4 * n1 + n2) * RS + c] = v[n1];
    }
    __syncthreads();
  }

  // ---- fused steps: the end of one transform and the start of the next share a task ----
  // col_inv (finishing an inverse FFT, natural output) -> hook (natural (r, c)) -> col_fwd
  // (starting the next forward FFT).  FWD = false: stop after the hook (nothing written back).
  template <bool FWD, class H>
  __device__ static void col_inv_fwd(float2* s, const float2* tw, H& h) {
    all_sync();
#pragma unroll 1
    for (int i = 0; i < NCOL; ++i) {
      const int t = threadIdx.x + i * T;
      const int c = t % N, n2 = t / N;
      float2 v[A];
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) v[k1] = s[(4 * k1 + n2) * RS + c];
      if (!PTY_TW_SKIP || n2 != 0) {
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1) v[k1] = cmulc(tw[n2 * k1], v[k1]);
      }
      dft<A, true>(v);
      hook(h, n2, 4, c, 0, v);
      if (FWD) {
        dft<A, false>(v);
        if (!PTY_TW_SKIP || n2 != 0) {
#pragma unroll
          for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], tw[n2 * k1]);
        }
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) s[(4 * k1 + n2) * RS + c] = v[k1];
      }
    }
    __syncthreads();
  }
  // row_fwd (finishing a forward FFT) -> hook (k-space (p0, p1)) -> row_inv (starting an inverse)
  template <class H>
  __device__ static void row_fwd_inv(float2* s, const float2* tw, H& h) {
#pragma unroll 1
    for (int i = 0; i < NROW; ++i) {
      const int t = gtid() + i * TG;
      const int r = grp() * RG + t % RG, k1 = t / RG;
      float2 v[A];
#pragma unroll
      for (int n2 = 0; n2 < A; ++n2) v[n2] = s[r * RS + A * k1 + n2];
      dft<A, false>(v);
      hook(h, r, 0, A * k1, 1, v);
      dft<A, true>(v);
      if (!PTY_TW_SKIP || k1 != 0) {
#pragma unroll
        for (int n2 = 1; n2 < A; ++n2) v[n2] = cmulc(tw[n2 * k1], v[n2]);
      }
#pragma unroll
      for (int n2 = 0; n2 < A; ++n2) s[r * RS + A * k1 + n2] = v[n2];
    }
    group_sync();
  }

  // natural s[r][c] -> k-space s[p0][p1] (unnormalised forward DFT).  `load` sees natural (r, c);
  // `store` sees k-space (p0, p1).  WRITE = false leaves the result only to `store`.
  template <bool WRITE = true, class LH = NoHook, class SH = NoHook>
  __device__ static void forward(float2* s, const float2* tw, LH&& load = LH(), SH&& store = SH()) {
    col_fwd(s, tw, load);
    block_fwd(s, tw);
    row_fwd<WRITE>(s, store);
    all_sync();  // the caller may read any row
  }
  // k-space s[p0][p1] -> natural s[r][c] (unnormalised inverse DFT); `load` sees k-space (p0, p1).
  template <class LH = NoHook>
  __device__ static void inverse(float2* s, const float2* tw, LH&& load = LH()) {
    row_inv(s, tw, load);
    block_inv(s, tw);
    col_inv(s, tw);
  }

  // Apply a hook to every element of the natural-layout array in batches of U elements per thread:
  // thread t owns column t % N and rows t / N + i * (T / N), so a batch is U rows of one column.  The
  // hook sees the whole batch at once and can keep U of its global loads in flight.
  template <int U, class H>
  __device__ static void pointwise(float2* s, H& h) {
    constexpr int NE = N * N / T, RPI = T / N;
    static_assert(NE % U == 0, "batch must divide the elements per thread");
    all_sync();
    const int c = threadIdx.x % N, r0 = threadIdx.x / N;
#pragma unroll 1
    for (int i0 = 0; i0 < NE; i0 += U) {
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = s[(r0 + (i0 + u) * RPI) * RS + c];
      h.template operator()<U>(r0 + i0 * RPI, RPI, c, 0, v);
#pragma unroll
      for (int u = 0; u < U; ++u) s[(r0 + (i0 + u) * RPI) * RS + c] = v[u];
    }
    __syncthreads();
  }

  // The same for the k-space array with lanes owning consecutive rows p0 (thread t: row t % N,
  // columns t / N + i * (T / N)), so that transposed global k-space buffers (p1 * N + p0) are read
  // coalesced and shared memory is walked with the odd row stride.
  template <int U, class H>
  __device__ static void pointwise_rows(float2* s, H& h) {
    constexpr int NE = N * N / T, CPI = T / N;
    static_assert(NE % U == 0, "batch must divide the elements per thread");
    const int r = grp() * RG + gtid() % RG, c0 = gtid() / RG;
#pragma unroll 1
    for (int i0 = 0; i0 < NE; i0 += U) {
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = s[r * RS + c0 + (i0 + u) * CPI];
      h.template operator()<U>(r, 0, c0 + i0 * CPI, CPI, v);
#pragma unroll
      for (int u = 0; u < U; ++u) s[r * RS + c0 + (i0 + u) * CPI] = v[u];
    }
    group_sync();
  }

  // k-space pointwise pass (lanes on consecutive rows, matching the transposed global buffers)
  template <int U, class H>
  __device__ static void pointwise_k(float2* s, H& h) {
    pointwise_rows<U>(s, h);
  }

  // Apply a hook to every element of the natural-layout array (same task shape as the col step).
  template <class H>
  __device__ static void elementwise(float2* s, H&& h) {
    all_sync();
#pragma unroll 1
    for (int i = 0; i < NCOL; ++i) {
      const int t = threadIdx.x + i * T;
      const int c = t % N, n2 = t / N;
      float2 v[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) v[n1] = s[(4 * n1 + n2) * RS + c];
      hook(h, n2, 4, c, 0, v);
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) s[(4 * n1 + n2) * RS + c] = v[n1];
    }
    __syncthreads();
  }
};

// tw[t] = exp(-2 pi i t / N) for t < N, written by the CTA's threads (a CTA smaller than N writes
// several each).
template <int N>
__device__ __forceinline__ void build_twiddles(float2* tw) {
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    float sn, cs;
    sincospif(2.0f * (float)t / (float)N, &sn, &cs);
    tw[t] = make_float2(cs, -sn);
  }
}

}  // namespace pty
