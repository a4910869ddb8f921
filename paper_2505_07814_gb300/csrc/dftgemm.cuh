// dftgemm.cuh -- the same pass with every per-slice 2D DFT computed as tensor-core GEMMs in split
// precision (pty_geom.fft_impl = PTY_FFT_SPLIT_BF16, _FP16 or SPLIT3_BF16), for N = 64 and 128.
//
// A 2D DFT of every wave of the batch is two row GEMMs over all waves at once: the first transforms
// along axis 1 and stores its result transposed per wave, the second transforms along the other axis.
// A complex row x times a complex matrix F is the real product [xr xi] [[Fr Fi]; [-Fi Fr]], and each
// real operand is cut into 16-bit pieces: with two pieces x F ~ xh Fh + xh Fl + xl Fh, evaluated as
// ONE GEMM with the terms concatenated along K (K = terms * 2N) and FP32 accumulation.  The DFT
// matrices are permuted so that k-space comes out in exactly the digit order of the shared-memory
// FFT (kbin0 / kbin1), so patterns, loss, hooks and finalisers are shared with the FP32 path.
// Elementwise work between transforms runs as per-wave pointwise kernels that apply the same hooks
// to the wave in global memory.  FP32 FFTs remain for the probe spectra and the probe-gradient
// finaliser (once per call, not per slice).
//
// fp16 has a 5-bit exponent, so before each fp16 GEMM the batch is scaled by a power of two that
// puts its largest magnitude near 2^14; bf16 keeps FP32's exponent range and needs no scaling.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gemm_mma.cuh"
#include "gemm_tc.cuh"

// column tile of the DFT GEMMs (0: all 2N columns in one CTA)
#ifndef PTY_DFT_BN
#define PTY_DFT_BN 0
#endif
#include "pipeline.cuh"

namespace pty {

// Split formats.  Each operand is cut into kPieces 16-bit pieces (piece 0 = the value rounded to 16
// bits, piece q = the remainder after pieces 0..q-1 rounded to 16 bits), and the product keeps the
// kTerms piece pairs (A piece, B piece) whose weight is above the format's rounding:
//   P = 1 (bf16, 2 pieces): h*h + h*l + l*h, 16 significant bits;
//   P = 2 (fp16, 2 pieces): h*h + h*l + l*h, 22 significant bits (after power-of-two scaling);
//   P = 3 (bf16, 3 pieces): h*h + h*m + m*h + h*l + l*h + m*m, 24 significant bits.
template <int P>
struct SplitType;
template <>
struct SplitType<PTY_FFT_SPLIT_BF16> {
  using H = __nv_bfloat16;
  static constexpr bool kScale = false;
  static constexpr int kPieces = 2, kTerms = 3;
  __host__ __device__ static constexpr int a_piece(int t) { return t == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int b_piece(int t) { return t == 1 ? 1 : 0; }
  __device__ static H to(float x) { return __float2bfloat16_rn(x); }
  __device__ static float from(H h) { return __bfloat162float(h); }
};
template <>
struct SplitType<PTY_FFT_SPLIT_FP16> {
  using H = __half;
  static constexpr bool kScale = true;
  static constexpr int kPieces = 2, kTerms = 3;
  __host__ __device__ static constexpr int a_piece(int t) { return t == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int b_piece(int t) { return t == 1 ? 1 : 0; }
  __device__ static H to(float x) { return __float2half_rn(x); }
  __device__ static float from(H h) { return __half2float(h); }
};
template <>
struct SplitType<PTY_FFT_SPLIT3_BF16> {
  using H = __nv_bfloat16;
  static constexpr bool kScale = false;
  static constexpr int kPieces = 3, kTerms = 6;
  // terms: hh, hm, mh, hl, lh, mm
  __host__ __device__ static constexpr int a_piece(int t) { return t == 2 ? 1 : t == 4 ? 2 : t == 5 ? 1 : 0; }
  __host__ __device__ static constexpr int b_piece(int t) { return t == 1 ? 1 : t == 3 ? 2 : t == 5 ? 1 : 0; }
  __device__ static H to(float x) { return __float2bfloat16_rn(x); }
  __device__ static float from(H h) { return __bfloat162float(h); }
};

// Piece q of x (FP32 remainders are exact: each piece removes the leading bits).
template <class S>
__device__ __forceinline__ typename S::H split_piece(float x, int q) {
  typename S::H h = S::to(x);
  for (int i = 0; i < q; ++i) {
    x -= S::from(h);
    h = S::to(x);
  }
  return h;
}

// Split DFT matrices B^T[mat][2N][kTerms * 2N] (rows: real and imaginary part of output position 0,
// then of position 1, ...; K: the split terms, each input real parts then imaginary parts).  mat 0: axis 1 forward (natural c ->
// position p1); 1: axis 0 forward (r -> p0); 2: axis 0 inverse (p0 -> r); 3: axis 1 inverse (p1 -> c).
template <int N, int P>
__global__ void k_init_dft_tables(typename SplitType<P>::H* Bt) {
  using S = SplitType<P>;
  constexpr int R = 2 * N, K = S::kTerms * 2 * N;
  const size_t n = (size_t)4 * R * K;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int mat = (int)(i / ((size_t)R * K));
    const int jp = (int)((i / K) % R), kp = (int)(i % K);
    const int t = kp / R, q = kp % R;
    const int qin = q % N, pin = q / N, jout = jp / 2, pout = jp % 2;  // output (re, im) interleaved
    int a, b;
    double sign;
    switch (mat) {
      case 0: a = qin; b = kbin1<N>(jout); sign = -1.0; break;
      case 1: a = qin; b = kbin0<N>(jout); sign = -1.0; break;
      case 2: a = kbin0<N>(qin); b = jout; sign = 1.0; break;
      default: a = kbin1<N>(qin); b = jout; sign = 1.0; break;
    }
    double sn, cs;
    sincospi(2.0 * (double)((a * b) % N) / N, &sn, &cs);
    const double fr = cs, fi = sign * sn;
    // [[Fr Fi]; [-Fi Fr]]: input part pin, output part pout
    double g = (pin == pout) ? fr : (pin == 0 ? fi : -fi);
    // pieces from the FP64 value (the FP32 rounding of g would cap the table at 24 bits)
    typename S::H h = S::to((float)g);
    for (int r = 0; r < S::b_piece(t); ++r) {
      g -= (double)S::from(h);
      h = S::to((float)g);
    }
    Bt[i] = h;
  }
}

// A operand: row m of the batch (N complex values) expanded to kTerms copies of [re | im], each
// holding the piece of x that its term pairs with.
template <int N, int P>
struct SplitLoader {
  using S = SplitType<P>;
  const float2* X;
  int M;               // valid rows; rows beyond are zero
  const float* scale;  // fp16: device scalar, else nullptr
  __device__ __forceinline__ uint4 operator()(int m, int k) const {
    union {
      uint4 u;
      typename S::H h[8];
    } out;
    if (m >= M) return make_uint4(0u, 0u, 0u, 0u);
    const int t = k / (2 * N), q = k % (2 * N), part = q / N, c = q % N;
    const int piece = S::a_piece(t);
    const float4* x = reinterpret_cast<const float4*>(X + (size_t)m * N + c);
    const float sc = S::kScale ? *scale : 1.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 v = x[i];
      out.h[2 * i] = split_piece<S>((part ? v.y : v.x) * sc, piece);
      out.h[2 * i + 1] = split_piece<S>((part ? v.w : v.z) * sc, piece);
    }
    return out.u;
  }
};

// C column 2c is the real part and 2c + 1 the imaginary part of output position c (the tables
// interleave them), so each (v0, v1) pair is one complex value; TRANSPOSE stores row a of wave w
// at position (w, c, a).
template <int N, bool TRANSPOSE>
struct DftEpilogue {
  float* out;  // interleaved complex
  int M;
  const float* scale;  // fp16: undo the input scaling
  __device__ __forceinline__ void operator()(int row, int col, float v0, float v1) const {
    if (row >= M) return;
    const float s = scale ? 1.0f / *scale : 1.0f;
    const int c = col >> 1;
    const int w = row / N, a = row % N;
    const size_t e = TRANSPOSE ? ((size_t)w * N + c) * N + a : (size_t)row * N + c;
    reinterpret_cast<float2*>(out)[e] = make_float2(v0 * s, v1 * s);
  }
};

// Pre-split operands for the tensor-core GEMMs: row r holds, for each piece q, the 2N reals
// (real parts then imaginary parts) of that piece: Xs[r][q][2N].  A K chunk (term t, position j) is
// then 16 contiguous bytes, Xs[r][a_piece(t)][j .. j + 7], copied global -> shared directly.
template <int N, int P>
struct PiecesLoader {
  using S = SplitType<P>;
  using H = typename S::H;
  static constexpr bool kDirect = true;
  const H* A;
  int rows;
  __device__ __forceinline__ const void* src(int r, int k) const {
    if (r >= rows) return nullptr;
    const int t = k / (2 * N), j = k % (2 * N);
    return A + ((size_t)r * S::kPieces + S::a_piece(t)) * (2 * N) + j;
  }
  __device__ __forceinline__ uint4 operator()(int r, int k) const {
    const void* g = src(r, k);
    return g ? *reinterpret_cast<const uint4*>(g) : make_uint4(0u, 0u, 0u, 0u);
  }
};

// Xs from complex rows X[rows][N] (times the fp16 scale when given): one thread per 8 columns of
// one row, both parts, every piece.
template <int N, int P>
__global__ void k_split(const float2* __restrict__ X, typename SplitType<P>::H* __restrict__ Xs, int rows,
                        const float* scale) {
  using S = SplitType<P>;
  using H = typename S::H;
  const size_t n = (size_t)rows * (N / 8);
  const float sc = scale ? *scale : 1.0f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t r = i / (N / 8);
    const int c0 = 8 * (int)(i % (N / 8));
    const float4* x = reinterpret_cast<const float4*>(X + r * N + c0);
    float re[8], im[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float4 v = x[e];
      re[2 * e] = v.x * sc;
      im[2 * e] = v.y * sc;
      re[2 * e + 1] = v.z * sc;
      im[2 * e + 1] = v.w * sc;
    }
#pragma unroll
    for (int q = 0; q < S::kPieces; ++q) {
      union {
        uint4 u;
        H h[8];
      } a, b;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        a.h[e] = split_piece<S>(re[e], q);
        b.h[e] = split_piece<S>(im[e], q);
      }
      H* row = Xs + (r * S::kPieces + q) * (2 * N);
      *reinterpret_cast<uint4*>(row + c0) = a.u;
      *reinterpret_cast<uint4*>(row + N + c0) = b.u;
    }
  }
}

// First GEMM of a 2D transform, unscaled formats: the result, transposed per wave, goes straight
// into the pieces of the second GEMM's operand (output row (w, c), position part * N + a).
template <int N, int P>
struct DftSplitEpilogue {
  using S = SplitType<P>;
  typename S::H* out;
  int M;
  __device__ __forceinline__ void put(size_t orow, int j, float v) const {
#pragma unroll
    for (int q = 0; q < S::kPieces; ++q) out[(orow * S::kPieces + q) * (2 * N) + j] = split_piece<S>(v, q);
  }
  __device__ __forceinline__ void operator()(int row, int col, float v0, float v1) const {
    if (row >= M) return;
    const int c = col >> 1;  // (v0, v1) = (re, im) of output position c
    const int w = row / N, a = row % N;
    put((size_t)w * N + c, a, v0);
    put((size_t)w * N + c, N + a, v1);
  }
};

// fp16 scaling: largest |re|, |im| of the batch, then the power of two that maps it near 2^14.
static __global__ void k_absmax(const float* __restrict__ x, size_t n, unsigned* out) {
  float m = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(x[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as ints
}
static __global__ void k_pow2_scale(const unsigned* amax, float* scale) {
  const float m = __uint_as_float(*amax);
  *scale = (m > 0.f && isfinite(m)) ? exp2f(14.0f - ceilf(log2f(m))) : 1.0f;
}

// ---------------------------------------------------------------------------------------------
// Pointwise stages on a wave in global memory (one CTA of 256 threads per wave)
// ---------------------------------------------------------------------------------------------
enum GemmStage { GS_SHIFT, GS_TRANS, GS_PROP, GS_FAR, GS_FARGRAD, GS_ADJTRANS, GS_ADJPROP, GS_PROBE };

struct StageArgs {
  FwdArgs f;     // geometry, parameters, checkpoint / far-field outputs (forward stages)
  AdjArgs a;     // adjoint inputs and accumulators
  float2* wave;  // [waves][N*N] current wave (natural or k-space layout)
  int sl;        // slice
};

template <int N>
__host__ __device__ constexpr size_t stage_smem_bytes() {
  return sizeof(float2) * 4 * N + sizeof(float) * 6 * N + sizeof(double) * 5 * 8;
}

template <int N, int ST>
__global__ void __launch_bounds__(256) k_stage(StageArgs g) {
  constexpr int T = 256, NN = N * N, STEP = T / N;
  extern __shared__ __align__(16) float2 sm[];
  float2* t0p = sm;  // forward: ra0 / ra1 / pm0 / pm1; adjoint: cm0 / cm1 / cr0 / cr1
  float2* t1p = t0p + N;
  float2* t2p = t1p + N;
  float2* t3p = t2p + N;
  float* e0 = reinterpret_cast<float*>(t3p + N);
  float* e1 = e0 + N;
  float* c0 = e1 + N;
  float* c1 = c0 + N;
  float* f0 = c1 + N;
  float* f1 = f0 + N;
  double* red = reinterpret_cast<double*>(f1 + N);
  const FwdArgs& a = g.f;
  const int tid = threadIdx.x, bm = blockIdx.x;
  const int b = bm / (a.M * a.Ko), m = (bm / a.Ko) % a.M;  // waves: (position, probe mode, object mode)
  const int j = checked_index(a.idx, b, a.Ntot, a.status);
  int i0, i1;
  float d0, d1, th0, th1;
  patch_corner<N>(a.pos, j, a.H, a.W, &i0, &i1, &d0, &d1, a.status);
  tilt_of(a.tilt, a.global_tilt, j, &th0, &th1);
  const float dz = a.dz[0];
  constexpr bool kAdj = ST >= GS_FARGRAD;
  if (kAdj) {
    adj_tables<N>(t0p, t1p, t2p, t3p, e0, e1, c0, c1, f0, f1, d0, d1, th0, th1, dz, a.dx, a.lam);
  } else {
    fwd_tables<N>(t0p, t1p, t2p, t3p, d0, d1, th0, th1, dz, a.dx, a.lam);
  }
  __syncthreads();
  const size_t plane = (size_t)a.H * a.W, patch = (size_t)(bm % a.Ko) * a.Nz * plane + (size_t)i0 * a.W + i1;
  float2* X = g.wave + (size_t)bm * NN;
  const int sl = g.sl;
  float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  constexpr int U = 8;
  // natural stages: thread owns column tid % N, rows tid / N + STEP i; k-space stages: row p0 = tid % N,
  // columns p1 = tid / N + STEP i (the buffer is stored p1 * N + p0)
  const int lo = tid % N, hi0 = tid / N;
  for (int i = 0; i < N / STEP; i += U) {
    float2 v[U];
    const int h = hi0 + i * STEP;
    if constexpr (ST != GS_SHIFT && ST != GS_FARGRAD) {  // those two replace the wave
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = X[(size_t)(h + u * STEP) * N + lo];
    }
    if constexpr (ST == GS_SHIFT) {
      ShiftLoad<N> hk{a.Phat + (size_t)m * NN, t0p, t1p};
      hk.template operator()<U>(lo, 0, h, STEP, v);
    } else if constexpr (ST == GS_TRANS) {
      TransLoad<N> hk{a.T + sl * plane + patch, a.W, a.ckpt ? a.ckpt + ((size_t)bm * a.Nz + sl) * NN : nullptr};
      hk.template operator()<U>(h, STEP, lo, 0, v);
    } else if constexpr (ST == GS_PROP) {
      PropStore<N> hk{t2p, t3p, a.vhat ? a.vhat + ((size_t)bm * (a.Nz - 1) + sl) * NN : nullptr};
      hk.template operator()<U>(lo, 0, h, STEP, v);
    } else if constexpr (ST == GS_FAR) {
      FarStore<N> hk{a.Psi ? a.Psi + (size_t)bm * NN : nullptr, a.Imode + (size_t)bm * NN};
      hk.template operator()<U>(lo, 0, h, STEP, v);
    } else if constexpr (ST == GS_FARGRAD) {
      FarGradLoad<N> hk{g.a.u + (size_t)b * NN, g.a.Psi + (size_t)bm * NN,
                        g.a.u_scaled ? 1.0f : (float)(2.0 * g.a.scal[0] / N)};
      hk.template operator()<U>(lo, 0, h, STEP, v);
    } else if constexpr (ST == GS_ADJTRANS) {
      const bool obj = (g.a.grad_mask & (PTY_GRAD_AMP | PTY_GRAD_PHASE)) != 0;
      AdjTransLoad<N> hk{a.T + sl * plane + patch, g.a.gT + sl * plane + patch,
                         obj ? g.a.ckpt + ((size_t)bm * a.Nz + sl) * NN : nullptr, a.W};
      hk.template operator()<U>(h, STEP, lo, 0, v);
    } else if constexpr (ST == GS_ADJPROP) {
      AdjPropStore<N> hk{t0p, t1p, g.a.vhat ? g.a.vhat + ((size_t)bm * (a.Nz - 1) + sl - 1) * NN : nullptr,
                         e0, e1, c0, c1, acc[4], acc[2], acc[3]};
      hk.template operator()<U>(lo, 0, h, STEP, v);
    } else {
      ProbeStore<N> hk{(g.a.grad_mask & PTY_GRAD_PROBE) ? g.a.gPhat + (size_t)m * NN : nullptr,
                       a.Phat + (size_t)m * NN, t2p, t3p, f0, f1, (g.a.grad_mask & PTY_GRAD_POS) != 0, acc[0], acc[1]};
      hk.template operator()<U>(lo, 0, h, STEP, v);
    }
    if constexpr (ST != GS_FAR && ST != GS_PROBE) {
#pragma unroll
      for (int u = 0; u < U; ++u) X[(size_t)(h + u * STEP) * N + lo] = v[u];
    }
  }
  if constexpr (ST == GS_ADJPROP || ST == GS_PROBE) {  // FP64 CTA sums into the per-wave partials
    double s5[5] = {acc[0], acc[1], acc[2], acc[3], acc[4]};
#pragma unroll
    for (int q = 0; q < 5; ++q)
      for (int o = 16; o > 0; o >>= 1) s5[q] += __shfl_down_sync(0xffffffffu, s5[q], o);
    if ((tid & 31) == 0) {
#pragma unroll
      for (int q = 0; q < 5; ++q) red[5 * (tid >> 5) + q] = s5[q];
    }
    __syncthreads();
    if (tid < 5) {
      double t = 0.0;
      for (int w = 0; w < T / 32; ++w) t += red[5 * w + tid];
      g.a.spart[(size_t)bm * 5 + tid] += t;
    }
  }
}

}  // namespace pty

namespace pty {

// Split DFT matrices of one device, built on the device on first use (one synchronous init per
// device and precision).
template <int N, int P>
__device__ __align__(256) typename SplitType<P>::H g_dft_tables[4 * 2 * N * SplitType<P>::kTerms * 2 * N];

template <int N, int P>
const typename SplitType<P>::H* dft_tables(cudaStream_t st) {
  static void* addr[256] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return nullptr;
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dft_tables<N, P>) != cudaSuccess || !p) return nullptr;
    k_init_dft_tables<N, P><<<152 * 4, 256, 0, st>>>(reinterpret_cast<typename SplitType<P>::H*>(p));
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return nullptr;
    note_launch();
    addr[dev] = p;
  }
  return reinterpret_cast<const typename SplitType<P>::H*>(addr[dev]);
}

// One pass with split-precision DFT-GEMMs in place of the shared-memory FFT (checkpoint every slice).
template <int N, int P>
struct GemmPass {
  using S = SplitType<P>;
  using H = typename S::H;
  static constexpr int NN = N * N;
  Pass<N> base;
  const Problem& pb;
  const Workspace& ws;
  cudaStream_t st;
  const H* tables = nullptr;

  explicit GemmPass(const Problem& p) : base(p), pb(p), ws(p.ws), st(p.stream) {}

  // out = rows of `src` times split DFT matrix `mat`; TRANSPOSE stores each wave transposed
  // fp16 batch scale of `src` into ws.gscal (returns the device scale pointer)
  int fp16_scale(const float2* src, const float** sc) {
    const int rows = pb.B * pb.M * pb.Ko * N;
    unsigned* amax = reinterpret_cast<unsigned*>(ws.gscal);
    float* scale = reinterpret_cast<float*>(ws.gscal) + 1;
    if (cudaMemsetAsync(amax, 0, sizeof(unsigned), st) != cudaSuccess) return base.memset_failed();
    k_absmax<<<152 * 4, 256, 0, st>>>(reinterpret_cast<const float*>(src), (size_t)rows * N * 2, amax);
    PTY_LAUNCH_CHECK("k_absmax", -1);
    k_pow2_scale<<<1, 1, 0, st>>>(amax, scale);
    PTY_LAUNCH_CHECK("k_pow2_scale", -1);
    *sc = scale;
    return PTY_OK;
  }
#if PTY_GEMM_LEGACY
  // out = rows of `src` times split DFT matrix `mat`; TRANSPOSE stores each wave transposed
  int gemm(int mat, const float2* src, float2* dst, bool transpose) {
    const int rows = pb.B * pb.M * pb.Ko * N;
    const int rows_pad = (rows + GB_M - 1) / GB_M * GB_M;
    const float* sc = nullptr;
    if (S::kScale) {
      int rc = fp16_scale(src, &sc);
      if (rc) return rc;
    }
    SplitLoader<N, P> ld{src, rows, sc};
    constexpr int K = S::kTerms * 2 * N;
    PlainLoader<H> lb{tables + (size_t)mat * 2 * N * K, (size_t)K, 2 * N};
    const dim3 grid(2 * N / GB_N, rows_pad / GB_M, 1);
    if (transpose) {
      k_gemm_tn<H, SplitLoader<N, P>, PlainLoader<H>, DftEpilogue<N, true>, true>
          <<<grid, GB_THREADS, 0, st>>>(ld, lb, K, K / GB_K, DftEpilogue<N, true>{(float*)dst, rows, sc});
    } else {
      k_gemm_tn<H, SplitLoader<N, P>, PlainLoader<H>, DftEpilogue<N, false>, true>
          <<<grid, GB_THREADS, 0, st>>>(ld, lb, K, K / GB_K, DftEpilogue<N, false>{(float*)dst, rows, sc});
    }
    PTY_LAUNCH_CHECK("k_gemm_tn", -1);
    return PTY_OK;
  }
  int transform(int mat_a, int mat_b) {
    int rc = gemm(mat_a, ws.wave, ws.tmp, true);
    return rc ? rc : gemm(mat_b, ws.tmp, ws.wave, false);
  }
#else
  // Tensor-core form: the wave is split once into pieces (k_split), the first GEMM writes its
  // transposed result either as pieces of the second GEMM's operand (bf16 formats) or, for fp16,
  // in FP32 to be rescaled and split again; both operands reach shared memory by cp.async.
  template <class Epi>
  int gemm_tc(int mat, const H* a_pieces, const Epi& epi) {
    const int rows = pb.B * pb.M * pb.Ko * N;
    constexpr int K = S::kTerms * 2 * N;
    PiecesLoader<N, P> la{a_pieces, rows};
    PlainLoader<H> lb{tables + (size_t)mat * 2 * N * K, (size_t)K, 2 * N};
    constexpr int BN = PTY_DFT_BN > 0 && PTY_DFT_BN < 2 * N ? PTY_DFT_BN : 2 * N;
    const cudaError_t e = launch_gemm_tc<H, BN, PTY_TC_PROMOTE>(la, lb, rows, 2 * N, K, epi, ws.status, st);
    if (e != cudaSuccess) {
      set_error("k_gemm_tc launch failed: %s", cudaGetErrorString(e));
      return PTY_ECUDA;
    }
    PTY_LAUNCH_CHECK("k_gemm_tc", -1);
    return PTY_OK;
  }
  int split(const float2* src, H* dst, const float* sc) {
    const int rows = pb.B * pb.M * pb.Ko * N;
    const size_t n = (size_t)rows * (N / 8);
    const unsigned blocks = (unsigned)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
    k_split<N, P><<<blocks, 256, 0, st>>>(src, dst, rows, sc);
    PTY_LAUNCH_CHECK("k_split", -1);
    return PTY_OK;
  }
  int transform(int mat_a, int mat_b) {
    const int rows = pb.B * pb.M * pb.Ko * N;
    H* pa = reinterpret_cast<H*>(ws.pieces0);
    H* pb_ = reinterpret_cast<H*>(ws.pieces1);
    const float* sc = nullptr;
    int rc;
    if (S::kScale) {
      if ((rc = fp16_scale(ws.wave, &sc))) return rc;
      if ((rc = split(ws.wave, pa, sc))) return rc;
      if ((rc = gemm_tc(mat_a, pa, DftEpilogue<N, true>{(float*)ws.tmp, rows, sc}))) return rc;
      if ((rc = fp16_scale(ws.tmp, &sc))) return rc;
      if ((rc = split(ws.tmp, pb_, sc))) return rc;
    } else {
      if ((rc = split(ws.wave, pa, nullptr))) return rc;
      if ((rc = gemm_tc(mat_a, pa, DftSplitEpilogue<N, P>{pb_, rows}))) return rc;
    }
    return gemm_tc(mat_b, pb_, DftEpilogue<N, false>{(float*)ws.wave, rows, sc});
  }
#endif
  // natural [w][r][c] -> k-space [w][p1][p0] and back
  int dft2() { return transform(0, 1); }
  int idft2() { return transform(2, 3); }
  template <int ST>
  int stage(const FwdArgs& fa, const AdjArgs& aa, int sl, int prof) {
    StageArgs g{fa, aa, ws.wave, sl};
    k_stage<N, ST><<<pb.B * pb.M * pb.Ko, 256, stage_smem_bytes<N>(), st>>>(g);
    PTY_LAUNCH_CHECK("k_stage", prof);
    return PTY_OK;
  }

  int forward(const float* I_meas) {
    tables = dft_tables<N, P>(st);
    if (!tables) {
      set_error("split DFT tables could not be set up: %s", cudaGetErrorString(cudaGetLastError()));
      return PTY_ECUDA;
    }
    int rc = base.forward_begin();
    if (rc || pb.B == 0) return rc;
    const FwdArgs fa = base.fwd_args_saved();
    const AdjArgs aa = base.adj_args();
    const int Nz = pb.Nz;
#define PTY_TRY(x)         \
  do {                     \
    int r_ = (x);          \
    if (r_) return r_;     \
  } while (0)
    PTY_TRY(stage<GS_SHIFT>(fa, aa, 0, -1));
    PTY_TRY(idft2());
    for (int sl = 0; sl < Nz; ++sl) {
      PTY_TRY(stage<GS_TRANS>(fa, aa, sl, -1));
      PTY_TRY(dft2());
      if (sl + 1 < Nz) {
        PTY_TRY(stage<GS_PROP>(fa, aa, sl, -1));
        PTY_TRY(idft2());
      } else {
        PTY_TRY(stage<GS_FAR>(fa, aa, sl, 2));
      }
    }
    return base.loss_phase(I_meas);
  }

  int adjoint() {
    PTY_TRY(base.adjoint_begin());
    if (pb.B > 0) {
      AdjArgs aa = base.adj_args();
      aa.ckpt = ws.ckpt;
      aa.vhat = base.want_prop ? ws.vhat : nullptr;
      const FwdArgs fa = base.fwd_args();
      const int Nz = pb.Nz;
      PTY_TRY(stage<GS_FARGRAD>(fa, aa, Nz - 1, -1));
      PTY_TRY(idft2());
      for (int sl = Nz - 1; sl >= 0; --sl) {
        PTY_TRY(stage<GS_ADJTRANS>(fa, aa, sl, -1));
        if (sl > 0) {
          PTY_TRY(dft2());
          PTY_TRY(stage<GS_ADJPROP>(fa, aa, sl, -1));
          PTY_TRY(idft2());
        } else if (base.want_probe || (pb.grad_mask & PTY_GRAD_POS)) {
          PTY_TRY(dft2());
          PTY_TRY(stage<GS_PROBE>(fa, aa, sl, -1));
        }
      }
      prof_mark(5, st);
    }
    return base.finalize();
#undef PTY_TRY
  }
};

template <int N, int P>
int run_pipeline_gemm(const Problem& pb) {
  GemmPass<N, P> ps(pb);
  int rc = ps.base.set_attributes();
  if (rc) return rc;
  switch (pb.mode) {
    case MODE_FORWARD:
    case MODE_FORWARD_SAVE:
      return ps.forward(nullptr);
    case MODE_GRAD:
      rc = ps.forward(pb.I_meas);
      if (rc) return rc;
      if (pb.B == 0 && pb.loss_out) {
        if (cudaMemsetAsync(pb.loss_out, 0, sizeof(double), pb.stream) != cudaSuccess) return ps.base.memset_failed();
      }
      return ps.adjoint();
    case MODE_STATS:
      if (pb.loss == PTY_LOSS_POISSON) return ps.base.stats();  // the measured patterns only
      rc = ps.forward(pb.I_meas);
      if (rc) return rc;
      return ps.base.stats_write();
    case MODE_BACKWARD:
      rc = ps.base.external_dldi(pb.dldi);
      if (rc) return rc;
      ps.tables = dft_tables<N, P>(pb.stream);
      if (!ps.tables) {
        set_error("split DFT tables could not be set up");
        return PTY_ECUDA;
      }
      return ps.adjoint();
    default:
      set_error("unknown pass mode %d", pb.mode);
      return PTY_EINVAL;
  }
}

}  // namespace pty
