// fft_smem.cuh -- 2D complex FFT of one N x N wavefield held in shared memory by one CTA.
//
// Layout.  The wave is float2 s[N][N + 1]: one complex pad per row makes the row stride odd, so
// both a warp walking along a row (32 consecutive columns) and a warp walking down 32 rows of one
// column touch 32 distinct bank pairs.
//
// Algorithm.  Every 1D pass transforms along the FIRST index with a two-factor Cooley-Tukey split
// N = R1 * R2 (n = R2 n1 + n2, k = k1 + R1 k2):
//   step A   R1-point DFT over n1 for every (column, n2), times W_N^{n2 k1}, written back in place;
//   step B   R2-point DFT over n2 for every (column, k1), written back in place.
// Lanes of a warp always own consecutive columns, so every shared-memory access is conflict-free;
// the small DFTs run in registers.  The forward output is left in the digit order the split
// produces (position p = R2 k1 + k2 holds frequency k1 + R1 k2): pointwise k-space work is done in
// that order and the inverse pass (the same steps mirrored, decimation in time) consumes it, so no
// reordering pass is ever needed.  A 2D transform is two 1D passes; the first one writes its
// result transposed (s[c][p] instead of s[p][c]) so that the second pass again runs along the
// first index.  Forward: natural s[r][c] -> k-space s[p1][p0]; inverse: k-space -> natural.
// Neither direction normalises (the inverse is the plain conjugate-sign sum).
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

// z * W_R^k with W_R = exp(-2 pi i / R) (forward) or its conjugate (INV); k is a compile-time
// constant once the calling loops are unrolled, so the branches fold away.
template <int R, bool INV>
__device__ __forceinline__ float2 twmul(int k, float2 z) {
  constexpr float H = 0.70710678118654752f;  // cos(pi/4)
  constexpr float C8 = 0.92387953251128676f;  // cos(pi/8)
  constexpr float S8 = 0.38268343236508977f;  // sin(pi/8)
  const int e = k * (16 / R);                 // angle in units of 2 pi / 16
  float c, s;                                 // W = c - i s (forward)
  switch (e) {
    case 0: return z;
    case 4: return INV ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
    case 2: c = H; s = H; break;
    case 6: c = -H; s = H; break;
    case 1: c = C8; s = S8; break;
    case 3: c = S8; s = C8; break;
    case 5: c = -S8; s = C8; break;
    case 7: c = -C8; s = S8; break;
    default: c = 1.f; s = 0.f; break;
  }
  if (INV) s = -s;
  return make_float2(fmaf(z.x, c, z.y * s), fmaf(z.y, c, -z.x * s));
}

// In-register R-point DFT (R = 2, 4, 8, 16), natural order in and out, radix-2 decimation in time.
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
      const float2 t = twmul<R, INV>(k, o[k]);
      x[k] = cadd(e[k], t);
      x[k + R / 2] = csub(e[k], t);
    }
  }
}

template <int N>
struct Radix;
template <>
struct Radix<64> {
  static constexpr int R1 = 8, R2 = 8;
};
template <>
struct Radix<128> {
  static constexpr int R1 = 8, R2 = 16;
};

// Position of frequency bin k (0..N-1, DFT order) along one axis of the k-space layout.
template <int N>
__host__ __device__ constexpr int kpos(int k) {
  return Radix<N>::R2 * (k % Radix<N>::R1) + k / Radix<N>::R1;
}
// Frequency bin held at k-space position p.
template <int N>
__host__ __device__ constexpr int kbin(int p) {
  return p / Radix<N>::R2 + Radix<N>::R1 * (p % Radix<N>::R2);
}

// Element hooks fused into the FFT passes.  A hook sees K elements of one task in registers: the
// elements sit at rows row0 + k * rstride (k < K) of column c of the array being transformed (the
// first index is the row).  Load hooks run right after the elements are read, store hooks right
// before they are written.  A hook with kReplaces = true produces the values itself, so the
// shared-memory read is skipped.
struct NoHook {
  static constexpr bool kReplaces = false;
  template <int K>
  __device__ __forceinline__ void operator()(int, int, int, float2*) {}
};

template <int N, int T>
struct Fft2 {
  static constexpr int R1 = Radix<N>::R1, R2 = Radix<N>::R2, RS = N + 1;
  static_assert(R1 * R2 == N, "radix split");
  static_assert((N * R1) % T == 0 && (N * R2) % T == 0, "tasks must divide the CTA");
  static_assert(T % N == 0, "each thread keeps one column");
  static constexpr int NA = N * R2 / T;  // step-A tasks per thread
  static constexpr int NB = N * R1 / T;  // step-B tasks per thread

  template <class H>
  static constexpr bool kPlain = std::is_same_v<std::decay_t<H>, NoHook>;

  // Forward 1D DFT along the first index.  TRANSPOSE: write result to s[c][p] instead of s[p][c].
  // WRITE = false: the result only goes through the store hook (nothing is written back).  Steps
  // with a hook run one task at a time (the hook's loads are batched inside the task); steps
  // without one unroll over the thread's tasks.
  template <bool TRANSPOSE, bool WRITE = true, class LH = NoHook, class SH = NoHook>
  __device__ static void fwd_pass(float2* s, const float2* tw, LH&& lh = LH(), SH&& sh = SH()) {
    static_assert(!(TRANSPOSE && !kPlain<SH>), "store hooks only on non-transposing passes");
    const int tid = threadIdx.x;
    constexpr int UA = kPlain<LH> ? NA : 1;
#pragma unroll(UA)
    for (int i = 0; i < NA; ++i) {
      const int t = tid + i * T;
      const int c = t % N, n2 = t / N;
      float2 v[R1];
      if (!std::remove_reference_t<LH>::kReplaces) {
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) v[n1] = s[(R2 * n1 + n2) * RS + c];
      }
      lh.template operator()<R1>(n2, R2, c, v);
      dft<R1, false>(v);
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], tw[n2 * k1]);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) s[(R2 * k1 + n2) * RS + c] = v[k1];
    }
    __syncthreads();
    if constexpr (TRANSPOSE) {
      float2 v[NB][R2];
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const int t = tid + i * T;
        const int c = t % N, k1 = t / N;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) v[i][n2] = s[(R2 * k1 + n2) * RS + c];
        dft<R2, false>(v[i]);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const int t = tid + i * T;
        const int c = t % N, k1 = t / N;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) s[c * RS + R2 * k1 + k2] = v[i][k2];
      }
    } else {
      constexpr int UB = kPlain<SH> ? NB : 1;
#pragma unroll(UB)
      for (int i = 0; i < NB; ++i) {
        const int t = tid + i * T;
        const int c = t % N, k1 = t / N;
        float2 v[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) v[n2] = s[(R2 * k1 + n2) * RS + c];
        dft<R2, false>(v);
        sh.template operator()<R2>(R2 * k1, 1, c, v);
        if (WRITE) {
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) s[(R2 * k1 + k2) * RS + c] = v[k2];
        }
      }
    }
    __syncthreads();
  }

  // Inverse 1D DFT along the first index (input in k-space digit order, output natural order).
  template <bool TRANSPOSE, class LH = NoHook>
  __device__ static void inv_pass(float2* s, const float2* tw, LH&& lh = LH()) {
    const int tid = threadIdx.x;
    constexpr int UB = kPlain<LH> ? NB : 1;
#pragma unroll(UB)
    for (int i = 0; i < NB; ++i) {
      const int t = tid + i * T;
      const int c = t % N, k1 = t / N;
      float2 v[R2];
      if (!std::remove_reference_t<LH>::kReplaces) {
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[k2] = s[(R2 * k1 + k2) * RS + c];
      }
      lh.template operator()<R2>(R2 * k1, 1, c, v);
      dft<R2, true>(v);
#pragma unroll
      for (int n2 = 1; n2 < R2; ++n2) v[n2] = cmulc(tw[n2 * k1], v[n2]);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) s[(R2 * k1 + n2) * RS + c] = v[n2];
    }
    __syncthreads();
    if constexpr (TRANSPOSE) {
      float2 v[NA][R1];
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const int t = tid + i * T;
        const int c = t % N, n2 = t / N;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) v[i][k1] = s[(R2 * k1 + n2) * RS + c];
        dft<R1, true>(v[i]);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const int t = tid + i * T;
        const int c = t % N, n2 = t / N;
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) s[c * RS + R2 * n1 + n2] = v[i][n1];
      }
    } else {
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const int t = tid + i * T;
        const int c = t % N, n2 = t / N;
        float2 v[R1];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) v[k1] = s[(R2 * k1 + n2) * RS + c];
        dft<R1, true>(v);
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) s[(R2 * n1 + n2) * RS + c] = v[n1];
      }
    }
    __syncthreads();
  }

  // natural s[r][c] -> k-space s[p1][p0] (unnormalised forward DFT).  `load` sees natural (r, c);
  // `store` sees k-space (p1, p0).  WRITE = false leaves the result only to `store`.
  template <bool WRITE = true, class LH = NoHook, class SH = NoHook>
  __device__ static void forward(float2* s, const float2* tw, LH&& load = LH(), SH&& store = SH()) {
    fwd_pass<true>(s, tw, load);
    fwd_pass<false, WRITE>(s, tw, NoHook(), store);
  }
  // k-space s[p1][p0] -> natural s[r][c] (unnormalised inverse DFT); `load` sees k-space (p1, p0).
  template <class LH = NoHook>
  __device__ static void inverse(float2* s, const float2* tw, LH&& load = LH()) {
    inv_pass<true>(s, tw, load);
    inv_pass<false>(s, tw);
  }

  // Apply a hook to every element of the natural-layout array (same task shape as step A).
  template <class H>
  __device__ static void elementwise(float2* s, H&& h) {
    const int tid = threadIdx.x;
#pragma unroll 1
    for (int i = 0; i < NA; ++i) {
      const int t = tid + i * T;
      const int c = t % N, n2 = t / N;
      float2 v[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) v[n1] = s[(R2 * n1 + n2) * RS + c];
      h.template operator()<R1>(n2, R2, c, v);
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) s[(R2 * n1 + n2) * RS + c] = v[n1];
    }
    __syncthreads();
  }
};

// tw[t] = exp(-2 pi i t / N) for t < N, written by the first N threads.
template <int N>
__device__ __forceinline__ void build_twiddles(float2* tw) {
  const int t = threadIdx.x;
  if (t < N) {
    float sn, cs;
    sincospif(2.0f * (float)t / (float)N, &sn, &cs);
    tw[t] = make_float2(cs, -sn);
  }
}

}  // namespace pty
