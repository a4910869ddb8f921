// gemm_tc.cuh -- C = A * B^T on the 5th-generation tensor cores (tcgen05.mma, accumulator in TMEM),
// with the same loader / epilogue interface as k_gemm_tn (gemm_mma.cuh).
//
// CTA tile 128 x BN (BN = 64, 128 or 256), K in blocks of 64.  All 256 threads are producers: each
// K block's A (128 x 64) and B (BN x 64) tiles are gathered by the loader functors and written to
// shared memory in the tensor core's canonical K-major layout without swizzle (8-row x 16-byte core
// matrices; LBO = 128 B between core matrices along K, SBO = 1024 B between 8-row groups).  One
// thread issues four 128 x BN x 16 MMAs per block and commits them to the stage's mbarrier; the
// producers fill the next stages meanwhile and wait on a stage's mbarrier only before refilling it
// (STAGES-deep ring).  The FP32 accumulator lives in TMEM (BN columns x 128 lanes); at the end the
// eight warps read it back with tcgen05.ld (warp w: lanes 32 (w % 4) .., columns of half w / 4)
// and hand (row, col, v0, v1) pairs to the epilogue.
//
// PROMOTE: every block of 64 is accumulated into a fresh TMEM region and added to an FP32
// register accumulator with round-to-nearest adds (the tensor core's own accumulation drifts over
// long K; see k_gemm_tn), using two TMEM regions alternately.
//
// Every wait is bounded: on a timeout the kernel sets PTY_ETIMEOUT in *status, stops issuing,
// waits (bounded) for its MMAs, frees its TMEM and returns.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "gemm_mma.cuh"
#include "pty.h"

// 1: the legacy mma.sync GEMM (gemm_mma.cuh) instead, for comparisons
#ifndef PTY_GEMM_LEGACY
#define PTY_GEMM_LEGACY 0
#endif
#ifndef PTY_TC_PROMOTE
#define PTY_TC_PROMOTE true
#endif

namespace pty {

constexpr int TC_BM = 128, TC_BK = 64, TC_THREADS = 256;
constexpr int TC_LBO = 128, TC_SBO = 1024;
constexpr long TC_SPIN = PTY_WAIT_POLLS_DEFAULT;  // non-blocking mbarrier polls before a wait gives up (well under a second)

// Pipeline depth and CTAs per SM by tile width: a 128 x 256 tile with promotion holds 128 FP32
// accumulators per thread (one CTA per SM, three stages); narrower tiles run two CTAs per SM with
// two stages each, so one CTA's gathers overlap the other's waits.
#ifndef PTY_TC_MINB
#define PTY_TC_MINB 2
#endif
template <int BN>
struct TcShape {
  static constexpr int STAGES = BN == 256 ? 3 : 2, MINB = BN == 256 ? 1 : PTY_TC_MINB;
};
template <int BN>
__host__ __device__ constexpr size_t tc_smem_bytes() {
  return (size_t)TcShape<BN>::STAGES * (TC_BM + BN) * TC_BK * 2 + 1024 /* alignment */ + 64 /* barriers, TMEM slot */;
}

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), descriptor version 1,
// no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(TC_LBO >> 4) << 16) | ((uint64_t)(TC_SBO >> 4) << 32) |
         ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, A and B of type H (bf16 or fp16), both
// K-major, M = 128, N = BN.
template <class H, int BN>
__host__ __device__ constexpr uint32_t tc_idesc() {
  constexpr uint32_t ab = std::is_same<H, __nv_bfloat16>::value ? 1u : 0u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ bool tc_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait of at most `limit` polls; false on timeout.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity, long limit = TC_SPIN) {
  for (long i = 0; i < limit; ++i)
    if (tc_try_wait(bar, parity)) return true;
  return false;
}
// Poll limit of the pipeline's waits (the final drain before TMEM is released always takes
// TC_SPIN); pty_set_wait_limit changes it for tests that make a wait run out.
long stage_wait_limit();

__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}


// Loader cursors.  Each producer thread gathers the same rows in every K block, so a loader may
// define Cursor / cursor(m, k) / load(cursor) / advance(cursor, dk) to decode a row once and step
// through K incrementally; other loaders are called as loader(m, k).
template <class L, class = void>
struct loader_cursor : std::false_type {};
template <class L>
struct loader_cursor<L, std::void_t<typename L::Cursor>> : std::true_type {};

template <class L, bool = loader_cursor<L>::value>
struct CursorOf {
  struct T {
    int m, k;
  };
};
template <class L>
struct CursorOf<L, true> {
  using T = typename L::Cursor;
};
template <class L>
__device__ __forceinline__ typename CursorOf<L>::T cur_make(const L& l, int m, int k) {
  if constexpr (loader_cursor<L>::value) return l.cursor(m, k);
  else return typename CursorOf<L>::T{m, k};
}
template <class L>
__device__ __forceinline__ uint4 cur_load(const L& l, const typename CursorOf<L>::T& c) {
  if constexpr (loader_cursor<L>::value) return l.load(c);
  else return l(c.m, c.k);
}
template <class L>
__device__ __forceinline__ void cur_advance(const L& l, typename CursorOf<L>::T& c, int dk) {
  if constexpr (loader_cursor<L>::value) l.advance(c, dk);
  else c.k += dk;
}

// grid = (ceil(N / BN), ceil(M / 128), splits); blockIdx.z takes K blocks [z kb_per, (z + 1) kb_per).
// Dynamic shared memory: tc_smem_bytes<BN>().  K is a multiple of 64 (the loaders pad with zeros).
// spin: poll limit of the pipeline's waits (stage reuse, promotion, last block).
template <class H, class LoadA, class LoadB, class Epi, int BN, bool PROMOTE>
__global__ void __launch_bounds__(TC_THREADS, TcShape<BN>::MINB)
    k_gemm_tc(LoadA la, LoadB lb, int K, int kb_per, Epi epi, int* status, long spin) {
  static_assert(BN == 64 || BN == 128 || BN == 256, "BN");
  constexpr int TC_STAGES = TcShape<BN>::STAGES;
  constexpr int A_BYTES = TC_BM * TC_BK * 2, B_BYTES = BN * TC_BK * 2, STAGE = A_BYTES + B_BYTES;
  constexpr int A_CHUNKS = TC_BM * TC_BK / 8 / TC_THREADS, B_CHUNKS = BN * TC_BK / 8 / TC_THREADS;
  constexpr int COLS = PROMOTE ? 2 * BN : BN;  // TMEM columns (power of two, >= 32)
  constexpr int HALF = BN / 2;                 // epilogue columns per warp
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + TC_STAGES * STAGE);  // [TC_STAGES]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + TC_STAGES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * BN;
  const int kb_all = K / TC_BK;
  const int kb0 = blockIdx.z * kb_per;
  const int kb1 = kb0 + kb_per < kb_all ? kb0 + kb_per : kb_all;
  const int nkb = kb1 > kb0 ? kb1 - kb0 : 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(tslot)),
                 "r"(COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < TC_STAGES; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_u32(bars + i)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const int col_half = (warp >> 2) * HALF;

  [[maybe_unused]] float acc[PROMOTE ? HALF : 1];
  if constexpr (PROMOTE) {
#pragma unroll
    for (int j = 0; j < HALF; ++j) acc[j] = 0.f;
  }
  // Waits are per thread and bounded; their outcome is made uniform over the CTA with
  // __syncthreads_and before anything that needs every thread (barriers, .sync.aligned loads).
  bool ok = true;
  int issued = -1;  // last block whose MMAs were issued (uniform)
  auto wait_block = [&](int q, long limit) {  // block q's MMAs complete
    return tc_wait(tc_smem_u32(bars + q % TC_STAGES), (uint32_t)((q / TC_STAGES) & 1), limit);
  };
  // add block q (TMEM region q % 2, complete) to the register accumulator
  auto promote = [&](int q) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t region = tmem + (uint32_t)((q & 1) * BN) + lane_base + col_half;
#pragma unroll
    for (int c = 0; c < HALF; c += 32) {
      float v[32];
      tc_ld32(region + c, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[c + j] += v[j];
    }
  };

  // Loaders with src() (plain matrices) are copied global -> shared with cp.async; the others are
  // gathered through registers.
  constexpr bool kDirectA = loader_direct<LoadA>::value, kDirectB = loader_direct<LoadB>::value;
  [[maybe_unused]] uint4 ra[kDirectA ? 1 : A_CHUNKS];
  [[maybe_unused]] uint4 rb[kDirectB ? 1 : B_CHUNKS];
  // chunk c of a tile -> k group c / rows, row c % rows: a warp writes 32 rows of one k group
  // (four conflict-free 128-byte wavefronts).  A thread's rows are the same in every block, so its
  // loader cursors are set up once and advanced by 64 per block.
  [[maybe_unused]] typename CursorOf<LoadA>::T ca[kDirectA ? 1 : A_CHUNKS];
  [[maybe_unused]] typename CursorOf<LoadB>::T cb[kDirectB ? 1 : B_CHUNKS];
  if constexpr (!kDirectA) {
#pragma unroll
    for (int h = 0; h < A_CHUNKS; ++h) {
      const int c = tid + h * TC_THREADS;
      ca[h] = cur_make(la, m0 + c % TC_BM, kb0 * TC_BK + 8 * (c / TC_BM));
    }
  }
  if constexpr (!kDirectB) {
#pragma unroll
    for (int h = 0; h < B_CHUNKS; ++h) {
      const int c = tid + h * TC_THREADS;
      cb[h] = cur_make(lb, n0 + c % BN, kb0 * TC_BK + 8 * (c / BN));
    }
  }
  auto fetch = [&](int q) {  // the next block's register-path chunks
    (void)q;
    if constexpr (!kDirectA) {
#pragma unroll
      for (int h = 0; h < A_CHUNKS; ++h) {
        ra[h] = cur_load(la, ca[h]);
        cur_advance(la, ca[h], TC_BK);
      }
    }
    if constexpr (!kDirectB) {
#pragma unroll
      for (int h = 0; h < B_CHUNKS; ++h) {
        rb[h] = cur_load(lb, cb[h]);
        cur_advance(lb, cb[h], TC_BK);
      }
    }
  };
  // direct operands: asynchronous global -> shared copies of block q (zero-filled past the rows)
  auto copy_direct = [&](int q) {
    if constexpr (kDirectA || kDirectB) {
      unsigned char* st = base + (q % TC_STAGES) * STAGE;
      const int k0 = (kb0 + q) * TC_BK;
      if constexpr (kDirectA) {
#pragma unroll
        for (int h = 0; h < A_CHUNKS; ++h) {
          const int c = tid + h * TC_THREADS, r = c % TC_BM, kg = c / TC_BM;
          const void* g = la.src(m0 + r, k0 + 8 * kg);
          const uint32_t d = tc_smem_u32(st + (r >> 3) * TC_SBO + kg * TC_LBO + (r & 7) * 16);
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(g ? g : (const void*)la.A),
                       "r"(g ? 16 : 0)
                       : "memory");
        }
      }
      if constexpr (kDirectB) {
#pragma unroll
        for (int h = 0; h < B_CHUNKS; ++h) {
          const int c = tid + h * TC_THREADS, r = c % BN, kg = c / BN;
          const void* g = lb.src(n0 + r, k0 + 8 * kg);
          const uint32_t d = tc_smem_u32(st + A_BYTES + (r >> 3) * TC_SBO + kg * TC_LBO + (r & 7) * 16);
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(g ? g : (const void*)lb.A),
                       "r"(g ? 16 : 0)
                       : "memory");
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  };
  auto stash = [&](int q) {  // register-path chunks -> the block's stage
    unsigned char* sa = base + (q % TC_STAGES) * STAGE;
    if constexpr (!kDirectA) {
#pragma unroll
      for (int h = 0; h < A_CHUNKS; ++h) {
        const int c = tid + h * TC_THREADS, r = c % TC_BM, kg = c / TC_BM;
        *reinterpret_cast<uint4*>(sa + (r >> 3) * TC_SBO + kg * TC_LBO + (r & 7) * 16) = ra[h];
      }
    }
    if constexpr (!kDirectB) {
      unsigned char* sb = sa + A_BYTES;
#pragma unroll
      for (int h = 0; h < B_CHUNKS; ++h) {
        const int c = tid + h * TC_THREADS, r = c % BN, kg = c / BN;
        *reinterpret_cast<uint4*>(sb + (r >> 3) * TC_SBO + kg * TC_LBO + (r & 7) * 16) = rb[h];
      }
    }
  };

  // direct copies run D = STAGES - 1 blocks ahead of the MMAs
  constexpr int D = TC_STAGES - 1;
  if (nkb > 0) fetch(0);
#pragma unroll
  for (int d = 0; d < D; ++d)
    if (d < nkb) copy_direct(d);
  for (int q = 0; q < nkb; ++q) {
    const int s = q % TC_STAGES;
    unsigned char* sa = base + s * STAGE;
    unsigned char* sb = sa + A_BYTES;
    // the stage is free once the MMAs of block q - STAGES are done (already waited for, in
    // practice, by the promotion or the direct-B copy of an earlier iteration)
    bool mine = q < TC_STAGES || wait_block(q - TC_STAGES, spin);
    if (mine) stash(q);
    if constexpr (kDirectA || kDirectB) {  // block q's copies landed (newer ones may still fly)
      if (D >= 2 && q + 1 < nkb) {
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_all;" ::: "memory");
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok && mine) != 0;
    if (!ok) break;
    issued = q;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t d = tmem + (PROMOTE ? (uint32_t)((q & 1) * BN) : 0u);
      constexpr uint32_t id = tc_idesc<H, BN>();
#pragma unroll
      for (int kk = 0; kk < TC_BK; kk += 16) {
        const uint64_t da = tc_desc(tc_smem_u32(sa) + (kk / 8) * TC_LBO);
        const uint64_t db = tc_desc(tc_smem_u32(sb) + (kk / 8) * TC_LBO);
        const uint32_t accum = (PROMOTE ? kk > 0 : (q > 0 || kk > 0)) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
            "l"(da), "l"(db), "r"(id), "r"(accum));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tc_smem_u32(bars + s))
                   : "memory");
    }
    // the next block's register-path loads go out now and land while the tensor cores work
    if (q + 1 < nkb) fetch(q + 1);
    if constexpr (PROMOTE) {
      if (q > 0) {
        // block q - 1's region is refilled by block q + 1, issued only after the next barrier
        ok = __syncthreads_and(wait_block(q - 1, spin)) != 0;
        if (!ok) break;
        promote(q - 1);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      }
    }
    // direct copies of block q + D go to the stage block q - 1 read (finished once promoted)
    if constexpr (kDirectA || kDirectB) {
      if (q + D < nkb) {
        if (!PROMOTE && q >= 1) mine = wait_block(q - 1, spin);
        if (mine) copy_direct(q + D);
      }
    }
    if constexpr (!PROMOTE) ok = ok && mine;
  }
  if (nkb > 0 && ok) {
    ok = __syncthreads_and(wait_block(nkb - 1, spin)) != 0;
    if (ok) {
      if constexpr (PROMOTE) promote(nkb - 1);
      else asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
  }
  if (!ok) {
    if (tid == 0) atomicOr(status, PTY_ETIMEOUT);
    // let whatever was issued finish (bounded) before the accumulator is released
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (issued >= 0) wait_block(issued, TC_SPIN);
  } else if (nkb > 0) {
    const int row = m0 + 32 * (warp & 3) + lane;
    if constexpr (PROMOTE) {
#pragma unroll
      for (int j = 0; j < HALF; j += 2) epi(row, n0 + col_half + j, acc[j], acc[j + 1]);
    } else {
#pragma unroll 1
      for (int c = 0; c < HALF; c += 32) {
        float v[32];
        tc_ld32(tmem + lane_base + col_half + c, v);
#pragma unroll
        for (int j = 0; j < 32; j += 2) epi(row, n0 + col_half + c + j, v[j], v[j + 1]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS));
}


// Launch of k_gemm_tc for C[rows x cols] with reduction length K (rounded up to 64 here; the
// loaders return zeros past the real K) split over `splits` CTAs along K.
template <class H, int BN, bool PROMOTE, class LA, class LB, class Epi>
cudaError_t launch_gemm_tc(const LA& la, const LB& lb, int rows, int cols, int K, const Epi& epi, int* status,
                           cudaStream_t st, int splits = 1) {
  auto kern = k_gemm_tc<H, LA, LB, Epi, BN, PROMOTE>;
  static bool ready[256] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  if (!ready[dev]) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes<BN>());
    if (e != cudaSuccess) return e;
    ready[dev] = true;
  }
  const int kb_all = (K + TC_BK - 1) / TC_BK;
  if (splits > kb_all) splits = kb_all;
  if (splits < 1) splits = 1;
  const int kb_per = (kb_all + splits - 1) / splits;
  const dim3 grid((cols + BN - 1) / BN, (rows + TC_BM - 1) / TC_BM, (kb_all + kb_per - 1) / kb_per);
  kern<<<grid, TC_THREADS, tc_smem_bytes<BN>(), st>>>(la, lb, kb_all * TC_BK, kb_per, epi, status,
                                                       stage_wait_limit());
  return cudaGetLastError();
}

}  // namespace pty
