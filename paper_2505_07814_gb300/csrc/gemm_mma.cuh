// gemm_mma.cuh -- tensor-core GEMM C = A * B^T with 16-bit operands (bf16 or fp16) and FP32
// accumulation, for the split-precision DFT passes and the CNN layers.
//
// A is M x K and B is N x K, both K-contiguous ("TN": the layout mma.sync reads directly).  Both are
// produced by loader functors (plain matrix, split-precision expansion of complex data, or an
// implicit-GEMM gather of convolution patches or of their gradients), and each finished 2-element
// pair of C goes to an epilogue functor.  K must be a multiple of 32 (the loaders pad with zeros).
//
// CTA tile 128 x 128 x 32, eight warps as 2 (M) x 4 (N), warp tile 64 x 32 = 4 x 4 mma.sync
// m16n8k16 tiles; A and B tiles double-buffered in shared memory with an 80-byte row pitch (the
// ldmatrix row addresses of one 8 x 8 matrix then fall in distinct bank groups).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace pty {

constexpr int GB_M = 128, GB_N = 128, GB_K = 32, GB_PITCH = 40, GB_THREADS = 256;

template <class H>
struct MmaOp;
template <>
struct MmaOp<__nv_bfloat16> {
  __device__ static void run(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  // d = a b (zero accumulator in)
  __device__ static void run0(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%10,%10,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(0.f));
  }
};
template <>
struct MmaOp<__half> {
  __device__ static void run(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  __device__ static void run0(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%10,%10,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(0.f));
  }
};

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
// Plain operand loader: 8 consecutive K elements of row r starting at k (16-byte aligned); rows at
// or beyond `rows` read as zero.
template <class H>
struct PlainLoader {
  static constexpr bool kDirect = true;  // src() gives the address: copies may go global -> shared directly
  const H* A;
  size_t ld;
  int rows;
  __device__ __forceinline__ uint4 operator()(int r, int k) const {
    if (r >= rows) return make_uint4(0u, 0u, 0u, 0u);
    return __ldg(reinterpret_cast<const uint4*>(A + (size_t)r * ld + k));
  }
  // address of the chunk, or nullptr where the loader reads zeros
  __device__ __forceinline__ const void* src(int r, int k) const {
    return r < rows ? (const void*)(A + (size_t)r * ld + k) : nullptr;
  }
  // cursor for gathers through registers: the chunk's address, stepped along the row
  struct Cursor {
    const H* p;
  };
  __device__ __forceinline__ Cursor cursor(int r, int k) const {
    return Cursor{r < rows ? A + (size_t)r * ld + k : nullptr};
  }
  __device__ __forceinline__ uint4 load(const Cursor& c) const {
    return c.p ? __ldg(reinterpret_cast<const uint4*>(c.p)) : make_uint4(0u, 0u, 0u, 0u);
  }
  __device__ __forceinline__ void advance(Cursor& c, int dk) const {
    if (c.p) c.p += dk;
  }
};

// Loaders without src() are gathered through registers.
template <class L, class = void>
struct loader_direct : std::false_type {};
template <class L>
struct loader_direct<L, std::void_t<decltype(L::kDirect)>> : std::bool_constant<L::kDirect> {};

// C[M x N] = A[M x K] * B[N x K]^T, A row m / B row n delivered 8 K-elements at a time by the
// loaders.  grid = (ceil(N / 128), ceil(M / 128), splits): blockIdx.z takes K tiles
// [z * kt_per, min((z + 1) * kt_per, K / 32)) (split-K; the epilogue then accumulates).  The loaders
// return zeros outside the matrices and the epilogue discards what lies outside C.
//
// The next K tile is fetched into registers while the tensor cores work on the current one and
// stored to the other shared-memory buffer afterwards (one barrier per K tile).
//
// PROMOTE: the tensor core's addition of each MMA's products into its FP32 accumulator does not
// round like an IEEE FP32 add, and over a long K the error compounds (measured on the split DFTs:
// it grew with K and with the number of split products).  With PROMOTE the products of each 32-wide
// K tile are summed by the MMAs into a fresh register tile that is then added to the running sum
// with an ordinary round-to-nearest FP32 add, so the long sum rounds like a plain FP32 dot product.
template <class H, class LoadA, class LoadB, class Epi, bool PROMOTE = false>
__global__ void __launch_bounds__(GB_THREADS) k_gemm_tn(LoadA la, LoadB lb, int K, int kt_per, Epi epi) {
  __shared__ __align__(16) H sA[2][GB_M * GB_PITCH];
  __shared__ __align__(16) H sB[2][GB_N * GB_PITCH];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp / 4, wn = warp % 4;  // warp position: 2 x 4
  const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
  const int kt_all = K / GB_K;
  const int kt0 = blockIdx.z * kt_per;
  const int kt1 = kt0 + kt_per < kt_all ? kt0 + kt_per : kt_all;
  float acc[4][4][4];
  [[maybe_unused]] float part[PROMOTE ? 4 : 1][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

  // each thread moves two 16-byte chunks of A and two of B per K tile (128 rows x 4 chunks)
  uint4 ra[2], rb[2];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = tid + h * GB_THREADS;  // 0..511
      const int r = c >> 2, kc = (c & 3) * 8;
      ra[h] = la(m0 + r, k0 + kc);
      rb[h] = lb(n0 + r, k0 + kc);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = tid + h * GB_THREADS;
      const int r = c >> 2, kc = (c & 3) * 8;
      *reinterpret_cast<uint4*>(&sA[buf][r * GB_PITCH + kc]) = ra[h];
      *reinterpret_cast<uint4*>(&sB[buf][r * GB_PITCH + kc]) = rb[h];
    }
  };

  if (kt0 < kt1) {
    fetch(kt0 * GB_K);
    stash(0);
  }
  __syncthreads();
  for (int kt = kt0; kt < kt1; ++kt) {
    const int buf = (kt - kt0) & 1;
    const bool more = kt + 1 < kt1;
    if (more) fetch((kt + 1) * GB_K);  // in flight during the MMAs below
#pragma unroll
    for (int kk = 0; kk < GB_K; kk += 16) {
      uint32_t af[4][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = wm * 64 + i * 16 + (lane & 7) + 8 * ((lane >> 3) & 1);
        ldsm_x4(af[i], &sA[buf][r * GB_PITCH + kk + 8 * (lane >> 4)]);
      }
#pragma unroll
      for (int j = 0; j < 4; j += 2) {
        const int r = wn * 32 + j * 8 + (lane & 7) + 8 * (lane >> 4);
        uint32_t t[4];
        ldsm_x4(t, &sB[buf][r * GB_PITCH + kk + 8 * ((lane >> 3) & 1)]);
        bf[j][0] = t[0];
        bf[j][1] = t[1];
        bf[j + 1][0] = t[2];
        bf[j + 1][1] = t[3];
      }
      if constexpr (PROMOTE) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (kk == 0) {
              MmaOp<H>::run0(part[i][j], af[i], bf[j]);
            } else {
              MmaOp<H>::run(part[i][j], af[i], bf[j]);
            }
          }
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) MmaOp<H>::run(acc[i][j], af[i], bf[j]);
      }
    }
    if constexpr (PROMOTE) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][j][q] += part[i][j][q];
    }
    // the other buffer was last read in the previous iteration, before this iteration's barrier
    if (more) stash(buf ^ 1);
    __syncthreads();
  }
  // epilogue: thread holds C(row, col..col+1) and C(row+8, col..col+1) of every 16 x 8 tile
  const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = m0 + wm * 64 + i * 16 + g, col = n0 + wn * 32 + j * 8 + 2 * t4;
      epi(row, col, acc[i][j][0], acc[i][j][1]);
      epi(row + 8, col, acc[i][j][2], acc[i][j][3]);
    }
}

}  // namespace pty
