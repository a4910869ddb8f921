// constraints.cu -- the constraints applied after an optimiser step (pty_constrain, include/pty.h;
// Sec. "Physical constraints").
//
//   probe orthogonalisation  k_gram (FP64 Gram-matrix partials of the probe modes), k_ortho_eig
//                            (one warp: complex Jacobi eigensolver in FP64, modes sorted by power),
//                            k_ortho_apply (each pixel's modes mixed by the eigenvectors, in place);
//   k_z filter (Eq. 10-12)   the filter W_a is real and even in k, so one complex 3D DFT of
//                            z = amp + i phase filters both real arrays: k_lines along x, then y
//                            (forward), k_kz_columns (depth DFT, W_a / (Nz H W), inverse depth DFT
//                            per (k_y, k_x) column), k_lines along y, then x (inverse); the last
//                            pass writes amp and phase with the relaxation;
//   depth blur, positivity   k_constrain (Eq. 13 and the phase clip).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "pty_internal.h"

namespace pty {

// ---------------------------------------------------------------------------------------------
// Depth blur and positivity.  One CTA per (tile of T x V pixels of the plane, array): cp.async
// copies the tile's Nz slices to shared memory (each element is read from HBM once), each thread
// blurs its V pixel columns along depth with the Gaussian taps held in shared memory and writes
// every output once; the phase CTAs apply the relaxed positivity clip on the way out.
// HBM-bound: 8 bytes per element and array.
// ---------------------------------------------------------------------------------------------
constexpr int kMaxBlurSlices = 128;
constexpr int kConstrainSmem = 200 * 1024;

template <int V>
__global__ void k_constrain(float* __restrict__ x0, float* __restrict__ x1, int Nz, size_t plane, float sigma, int R,
                            float rz_relax, float pos_relax) {
  extern __shared__ __align__(16) unsigned char c_smem[];
  float* taps = reinterpret_cast<float*>(c_smem);  // w(d) = exp(-d^2 / (2 sigma^2)), d = 0 .. R
  float* rden = taps + kMaxBlurSlices;             // 1 / (sum of slice s's taps inside the volume)
  float* tile = rden + kMaxBlurSlices;             // [Nz][T * V]
  float* x = blockIdx.y ? x1 : x0;
  const float clip = x == x1 ? pos_relax : 0.f;  // x1 is the phase
  const int T = blockDim.x, tid = threadIdx.x;
  const size_t p = (blockIdx.x * (size_t)T + tid) * V;
  const bool in = p < plane;  // V = 4 needs plane % 4 == 0, so the whole vector is inside

  if (!(sigma > 0.f)) {  // positivity alone
    if (in) {
      for (int s = 0; s < Nz; ++s) {
        float* q = x + (size_t)s * plane + p;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const float y = q[v];
          if (y < 0.f) q[v] = y - clip * y;
        }
      }
    }
    return;
  }
  for (int s = 0; s < Nz; ++s) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(tile + ((size_t)s * T + tid) * V);
    const float* g = x + (size_t)s * plane + (in ? p : 0);
    if (V == 4)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(g), "r"(in ? 16 : 0) : "memory");
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(g), "r"(in ? 4 : 0) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int d = tid; d <= R; d += T) {
    const float u = (float)d / sigma;
    taps[d] = expf(-0.5f * u * u);
  }
  __syncthreads();
  for (int s = tid; s < Nz; s += T) {
    const int t0 = s - R > 0 ? s - R : 0, t1 = s + R < Nz - 1 ? s + R : Nz - 1;
    float den = 0.f;
    for (int t = t0; t <= t1; ++t) den += taps[t > s ? t - s : s - t];
    rden[s] = 1.f / den;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  if (!in) return;
  for (int s = 0; s < Nz; ++s) {
    const int t0 = s - R > 0 ? s - R : 0, t1 = s + R < Nz - 1 ? s + R : Nz - 1;
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.f;
    for (int t = t0; t <= t1; ++t) {
      const float w = taps[t > s ? t - s : s - t];
      const float* src = tile + ((size_t)t * T + tid) * V;
      if constexpr (V == 4) {
        const float4 q = *reinterpret_cast<const float4*>(src);
        acc[0] = fmaf(w, q.x, acc[0]);
        acc[1] = fmaf(w, q.y, acc[1]);
        acc[2] = fmaf(w, q.z, acc[2]);
        acc[3] = fmaf(w, q.w, acc[3]);
      } else {
        acc[0] = fmaf(w, src[0], acc[0]);
      }
    }
    const float* own = tile + ((size_t)s * T + tid) * V;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float v0 = own[v];
      float y = v0 + rz_relax * (acc[v] * rden[s] - v0);
      if (y < 0.f) y -= clip * y;
      acc[v] = y;
    }
    float* dst = x + (size_t)s * plane + p;
    if constexpr (V == 4)
      *reinterpret_cast<float4*>(dst) = make_float4(acc[0], acc[1], acc[2], acc[3]);
    else
      dst[0] = acc[0];
  }
}

template <int V>
static int launch_constrain(float* amp, float* phase, int Nz, size_t plane, float sigma, float rz_relax,
                            float pos_relax, cudaStream_t st) {
  const bool blur = sigma > 0.f;
  int T = 128;
  size_t smem = 0;
  if (blur) {
    const size_t fixed = 2 * kMaxBlurSlices * sizeof(float);
    T = (int)((kConstrainSmem - fixed) / ((size_t)Nz * V * sizeof(float)));
    T = T >= 128 ? 128 : T / 32 * 32;
    smem = fixed + (size_t)Nz * T * V * sizeof(float);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_constrain<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      set_error("cudaFuncSetAttribute(k_constrain) failed: %s", cudaGetErrorString(cudaGetLastError()));
      return PTY_ECUDA;
    }
  }
  const int R0 = (int)ceilf(4.0f * sigma);
  const int R = blur ? (R0 < Nz - 1 ? R0 : Nz - 1) : 0;
  const size_t per = (size_t)T * V;
  const dim3 grid((unsigned)((plane + per - 1) / per), blur ? 2 : 1);
  // without the blur only the phase is touched: the single row of CTAs takes x0 = phase
  k_constrain<V><<<grid, T, smem, st>>>(blur ? amp : phase, phase, Nz, plane, sigma, R, rz_relax, pos_relax);
  return PTY_OK;
}

// ---------------------------------------------------------------------------------------------
// k_z filter: line transforms.  One CTA transforms C lines of length L held in shared memory:
// radix-2 decimation in time (input stored bit-reversed, natural-order output) when L is a power
// of two, otherwise the direct O(L^2) DFT.  Neither direction normalises.  Lines along x are rows
// (element stride 1); lines along y are columns (stride W) taken C adjacent columns at a time, so
// global accesses stay in contiguous runs of C (axis 1) or L (axis 0) elements.
// ---------------------------------------------------------------------------------------------
constexpr int kLineElems = 8192;  // C * L per CTA
constexpr int kMaxLine = 8192;
constexpr int kLineThreads = 256;

enum LineIO { IO_Z = 0, IO_FROM_PAIR = 1, IO_TO_PAIR = 2 };

struct LineArgs {
  float2* z;     // complex volume [Nz][H][W]
  float* amp;    // IO_FROM_PAIR: real part source; IO_TO_PAIR: destination (relaxed)
  float* phase;  // imaginary part, likewise
  float relax;
  int axis;      // 0: lines along x, 1: lines along y
  int L, C, logL, pow2;
  int Nz, H, W;
  int tiles_per_slice;  // axis 1: ceil(W / C)
  long long lines;      // axis 0: Nz * H
};

// Global element of (line l of this CTA's tile, position j), or -1 when the line is past the end.
__device__ __forceinline__ long long line_elem(const LineArgs& a, long long tile, int l, int j) {
  if (a.axis == 0) {
    const long long g = tile * a.C + l;
    return g < a.lines ? g * a.W + j : -1;
  }
  const long long s = tile / a.tiles_per_slice;
  const int x = (int)(tile % a.tiles_per_slice) * a.C + l;
  return x < a.W ? (s * a.H + j) * a.W + x : -1;
}

__device__ __forceinline__ unsigned bitrev(unsigned j, int bits) { return bits ? __brev(j) >> (32 - bits) : 0u; }

template <bool INV, int IO>
__global__ void __launch_bounds__(kLineThreads) k_lines(LineArgs a) {
  extern __shared__ __align__(16) unsigned char l_smem[];
  const int L = a.L, C = a.C, tid = threadIdx.x;
  const int n = C * L;
  float2* buf = reinterpret_cast<float2*>(l_smem);  // [C][L]
  float2* out = buf + n;                              // direct DFT: [C][L]; power of two: unused
  float2* tw = a.pow2 ? buf + n : buf + 2 * n;        // exp(-+2 pi i t / L), t < L/2 (pow2) or < L
  const long long tile = blockIdx.x;
  const int ntw = a.pow2 ? L / 2 : L;
  for (int t = tid; t < ntw; t += kLineThreads) {
    float s, c;
    sincospif(-2.0f * (float)t / (float)L, &s, &c);
    tw[t] = make_float2(c, INV ? -s : s);
  }
  // load (contiguous runs: along j for axis 0, along l for axis 1)
  for (int f = tid; f < n; f += kLineThreads) {
    const int l = a.axis == 0 ? f / L : f % C;
    const int j = a.axis == 0 ? f % L : f / C;
    const long long e = line_elem(a, tile, l, j);
    float2 v = make_float2(0.f, 0.f);
    if (e >= 0) v = IO == IO_FROM_PAIR ? make_float2(a.amp[e], a.phase[e]) : a.z[e];
    buf[l * L + (a.pow2 ? (int)bitrev((unsigned)j, a.logL) : j)] = v;
  }
  __syncthreads();
  const float2* res = buf;
  if (a.pow2) {
    const int half = L >> 1;
    for (int h = 1, lh = 0; h < L; h <<= 1, ++lh) {
      for (int b = tid; b < C * half; b += kLineThreads) {
        const int l = b / half, q = b - l * half;
        const int r = q & (h - 1);
        const int i = ((q >> lh) << (lh + 1)) + r;
        const float2 w = tw[r << (a.logL - 1 - lh)];
        float2* row = buf + l * L;
        const float2 u = row[i], v0 = row[i + h];
        const float2 v = make_float2(fmaf(v0.x, w.x, -v0.y * w.y), fmaf(v0.x, w.y, v0.y * w.x));
        row[i] = make_float2(u.x + v.x, u.y + v.y);
        row[i + h] = make_float2(u.x - v.x, u.y - v.y);
      }
      __syncthreads();
    }
  } else {
    for (int f = tid; f < n; f += kLineThreads) {
      const int l = f / L, k = f - l * L;
      const float2* row = buf + l * L;
      float2 acc = make_float2(0.f, 0.f);
      int t = 0;  // (j * k) mod L
      for (int j = 0; j < L; ++j) {
        const float2 x = row[j], w = tw[t];
        acc.x = fmaf(x.x, w.x, fmaf(-x.y, w.y, acc.x));
        acc.y = fmaf(x.x, w.y, fmaf(x.y, w.x, acc.y));
        t += k;
        if (t >= L) t -= L;
      }
      out[f] = acc;
    }
    __syncthreads();
    res = out;
  }
  for (int f = tid; f < n; f += kLineThreads) {
    const int l = a.axis == 0 ? f / L : f % C;
    const int j = a.axis == 0 ? f % L : f / C;
    const long long e = line_elem(a, tile, l, j);
    if (e < 0) continue;
    const float2 v = res[l * L + j];
    if (IO == IO_TO_PAIR) {
      const float x0 = a.amp[e], y0 = a.phase[e];
      a.amp[e] = x0 + a.relax * (v.x - x0);
      a.phase[e] = y0 + a.relax * (v.y - y0);
    } else {
      a.z[e] = v;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// k_z filter: per (k_y, k_x) column of the laterally transformed volume, the depth DFT, the
// filter W_a (Eq. 10-11) with the 1 / (Nz H W) of the inverse 3D DFT, and the inverse depth DFT.
// One thread per column; the column and its spectrum sit in shared memory ([Nz][T] each).
// ---------------------------------------------------------------------------------------------
constexpr float kKzEps = 1e-3f;  // per square angstrom, the stabilising constant under Eq. 10

// DFT frequency of bin i of n samples spaced d, in cycles per unit of d (numpy's fftfreq)
__device__ __forceinline__ float fft_freq(int i, int n, float d) {
  return (float)(i < (n + 1) / 2 ? i : i - n) / ((float)n * d);
}

__global__ void k_kz_columns(float2* __restrict__ z, int Nz, int H, int W, float dx, const float* __restrict__ dz,
                             float beta, float alpha) {
  extern __shared__ __align__(16) unsigned char k_smem[];
  const int T = blockDim.x, tid = threadIdx.x;
  float2* tw = reinterpret_cast<float2*>(k_smem);  // exp(-2 pi i t / Nz)
  float2* col = tw + Nz;                           // [Nz][T]
  float2* spec = col + (size_t)Nz * T;             // [Nz][T]
  const size_t plane = (size_t)H * W;
  const size_t p = blockIdx.x * (size_t)T + tid;
  for (int t = tid; t < Nz; t += T) {
    float s, c;
    sincospif(-2.0f * (float)t / (float)Nz, &s, &c);
    tw[t] = make_float2(c, s);
  }
  const bool in = p < plane;
  if (in)
    for (int s = 0; s < Nz; ++s) col[(size_t)s * T + tid] = z[(size_t)s * plane + p];
  __syncthreads();
  if (!in) return;
  const float kx = fft_freq((int)(p % W), W, dx), ky = fft_freq((int)(p / W), H, dx);
  const float kr2 = kx * kx + ky * ky;
  const float dzv = *dz;
  const float lateral = expf(-alpha * kr2) / ((float)Nz * (float)plane);
  const float b2 = beta * beta, den = kr2 + kKzEps;
  for (int k = 0; k < Nz; ++k) {
    float2 acc = make_float2(0.f, 0.f);
    int t = 0;  // (s * k) mod Nz
    for (int s = 0; s < Nz; ++s) {
      const float2 x = col[(size_t)s * T + tid], w = tw[t];
      acc.x = fmaf(x.x, w.x, fmaf(-x.y, w.y, acc.x));
      acc.y = fmaf(x.x, w.y, fmaf(x.y, w.x, acc.y));
      t += k;
      if (t >= Nz) t -= Nz;
    }
    const float kz = fft_freq(k, Nz, dzv);
    const float wk = (1.0f - 0.63661977236758134f * atanf(b2 * kz * kz / den)) * lateral;  // 2 / pi
    spec[(size_t)k * T + tid] = make_float2(acc.x * wk, acc.y * wk);
  }
  for (int s = 0; s < Nz; ++s) {
    float2 acc = make_float2(0.f, 0.f);
    int t = 0;  // (s * k) mod Nz, conjugate twiddles
    for (int k = 0; k < Nz; ++k) {
      const float2 x = spec[(size_t)k * T + tid], w = tw[t];
      acc.x = fmaf(x.x, w.x, fmaf(x.y, w.y, acc.x));
      acc.y = fmaf(x.y, w.x, fmaf(-x.x, w.y, acc.y));
      t += s;
      if (t >= Nz) t -= Nz;
    }
    z[(size_t)s * plane + p] = acc;
  }
}

// ---------------------------------------------------------------------------------------------
// Probe orthogonalisation (mixed-state probe, Sec. "Physical constraints").  With the modes as the
// rows of A (M x N^2): G = A A^H = U diag(lambda) U^H, Q = U^H A, modes ordered by decreasing
// power lambda; each column of U is turned so that its largest-magnitude entry is real positive.
// ---------------------------------------------------------------------------------------------
constexpr int kMaxOrthoModes = 32;
constexpr int kGramChunk = 1024;   // pixels per k_gram CTA
constexpr int kJacobiSweeps = 60;  // cyclic sweeps at most (convergence is quadratic; a handful suffice)

__device__ __forceinline__ void pair_of(int pair, int M, int* m, int* n) {
  int r = pair, i = 0;
  while (r >= M - i) {  // row i holds the pairs (i, i .. M-1)
    r -= M - i;
    ++i;
  }
  *m = i;
  *n = i + r;
}

// partial[pair][chunk] = sum over the chunk's pixels of P_m conj(P_n), m <= n
__global__ void __launch_bounds__(256) k_gram(const float2* __restrict__ probe, int M, int NN,
                                              double2* __restrict__ partial) {
  __shared__ double2 red[256];
  int m, n;
  pair_of(blockIdx.y, M, &m, &n);
  const float2* pm = probe + (size_t)m * NN;
  const float2* pn = probe + (size_t)n * NN;
  double re = 0.0, im = 0.0;
  const int p1 = min(NN, (int)(blockIdx.x + 1) * kGramChunk);
  for (int p = blockIdx.x * kGramChunk + threadIdx.x; p < p1; p += 256) {
    const float2 a = pm[p], b = pn[p];
    re += (double)a.x * b.x + (double)a.y * b.y;
    im += (double)a.y * b.x - (double)a.x * b.y;
  }
  red[threadIdx.x] = make_double2(re, im);
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[threadIdx.x].x += red[threadIdx.x + h].x;
      red[threadIdx.x].y += red[threadIdx.x + h].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zlin(double a, double2 x, double2 b, double2 y) {  // a x + b y
  const double2 by = zmul(b, y);
  return make_double2(a * x.x + by.x, a * x.y + by.y);
}

// One warp: reduce the Gram partials, diagonalise with cyclic complex Jacobi rotations in FP64,
// sort, fix the phases; writes U (column k = eigenvector of the k-th largest power) and lambda.
__global__ void __launch_bounds__(32) k_ortho_eig(const double2* __restrict__ partial, int M, int chunks,
                                                   double2* __restrict__ Uout, double* __restrict__ lam_out) {
  __shared__ double2 G[kMaxOrthoModes][kMaxOrthoModes + 1];
  __shared__ double2 V[kMaxOrthoModes][kMaxOrthoModes + 1];
  __shared__ double lam[kMaxOrthoModes];
  const int lane = threadIdx.x;
  const int npairs = M * (M + 1) / 2;
  for (int pr = lane; pr < npairs; pr += 32) {
    int m, n;
    pair_of(pr, M, &m, &n);
    double re = 0.0, im = 0.0;
    for (int c = 0; c < chunks; ++c) {
      const double2 v = partial[(size_t)pr * chunks + c];
      re += v.x;
      im += v.y;
    }
    G[m][n] = make_double2(re, im);
    G[n][m] = make_double2(re, -im);
  }
  if (lane < M)
    for (int j = 0; j < M; ++j) V[lane][j] = make_double2(lane == j ? 1.0 : 0.0, 0.0);
  __syncwarp();
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = lane; i < M; i += 32) {
      diag += G[i][i].x * G[i][i].x;
      for (int j = i + 1; j < M; ++j) off += G[i][j].x * G[i][j].x + G[i][j].y * G[i][j].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      diag += __shfl_xor_sync(0xffffffffu, diag, o);
    }
    if (!(off > 1e-30 * diag)) break;  // also ends on an all-zero matrix
    for (int p = 0; p < M - 1; ++p) {
      for (int q = p + 1; q < M; ++q) {
        const double2 g = G[p][q];
        const double ag = sqrt(g.x * g.x + g.y * g.y);
        const double app = G[p][p].x, aqq = G[q][q].x;
        if (!(ag > 1e-290)) continue;  // already zero (or denormal)
        const double tau = (aqq - app) / (2.0 * ag);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        const double2 e = make_double2(g.x / ag, g.y / ag);    // e^{i phi}
        const double2 ec = make_double2(e.x, -e.y);              // e^{-i phi}
        const double2 mse = make_double2(-s * ec.x, -s * ec.y);  // -s e^{-i phi}
        const double2 cec = make_double2(c * ec.x, c * ec.y);    // c e^{-i phi}
        __syncwarp();
        // columns p, q of G and V: X <- X U with U_pp = c, U_pq = s, U_qp = -s e^{-i phi}, U_qq = c e^{-i phi}
        if (lane < M) {
          const double2 gp = G[lane][p], gq = G[lane][q];
          G[lane][p] = zlin(c, gp, mse, gq);
          G[lane][q] = zlin(s, gp, cec, gq);
          const double2 vp = V[lane][p], vq = V[lane][q];
          V[lane][p] = zlin(c, vp, mse, vq);
          V[lane][q] = zlin(s, vp, cec, vq);
        }
        __syncwarp();
        // rows p, q of G: G <- U^H G
        if (lane < M) {
          const double2 gp = G[p][lane], gq = G[q][lane];
          G[p][lane] = zlin(c, gp, make_double2(-s * e.x, -s * e.y), gq);
          G[q][lane] = zlin(s, gp, make_double2(c * e.x, c * e.y), gq);
        }
        __syncwarp();
        if (lane == 0) {
          G[p][q] = make_double2(0.0, 0.0);
          G[q][p] = make_double2(0.0, 0.0);
          G[p][p].y = 0.0;
          G[q][q].y = 0.0;
        }
        __syncwarp();
      }
    }
  }
  if (lane < M) lam[lane] = G[lane][lane].x;
  __syncwarp();
  if (lane < M) {
    // rank of this eigenpair by decreasing power (ties keep the index order)
    const double lk = lam[lane];
    int rank = 0;
    for (int j = 0; j < M; ++j) rank += (lam[j] > lk) || (lam[j] == lk && j < lane);
    int mstar = 0;
    double best = -1.0;
    for (int m = 0; m < M; ++m) {
      const double a = V[m][lane].x * V[m][lane].x + V[m][lane].y * V[m][lane].y;
      if (a > best) {
        best = a;
        mstar = m;
      }
    }
    const double2 vs = V[mstar][lane];
    const double av = sqrt(vs.x * vs.x + vs.y * vs.y);
    const double2 ph = av > 0.0 ? make_double2(vs.x / av, -vs.y / av) : make_double2(1.0, 0.0);
    for (int m = 0; m < M; ++m) Uout[(size_t)m * M + rank] = zmul(V[m][lane], ph);
    lam_out[rank] = lk;
  }
}

// Q_k[p] = sum_m conj(U[m][k]) P_m[p], in place; one thread per pixel, its M modes in shared memory.
__global__ void __launch_bounds__(128) k_ortho_apply(float2* __restrict__ probe, int M, int NN,
                                                      const double2* __restrict__ U) {
  extern __shared__ __align__(16) unsigned char o_smem[];
  double2* u = reinterpret_cast<double2*>(o_smem);                 // [M][M]
  float2* px = reinterpret_cast<float2*>(u + (size_t)M * M);     // [M][128]
  const int tid = threadIdx.x;
  for (int i = tid; i < M * M; i += 128) u[i] = U[i];
  const int p = blockIdx.x * 128 + tid;
  if (p < NN)
    for (int m = 0; m < M; ++m) px[m * 128 + tid] = probe[(size_t)m * NN + p];
  __syncthreads();
  if (p >= NN) return;
  for (int k = 0; k < M; ++k) {
    double re = 0.0, im = 0.0;
    for (int m = 0; m < M; ++m) {
      const double2 w = u[m * M + k];  // conj(w) * x
      const float2 x = px[m * 128 + tid];
      re += w.x * x.x + w.y * x.y;
      im += w.x * x.y - w.y * x.x;
    }
    probe[(size_t)k * NN + p] = make_float2((float)re, (float)im);
  }
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

static bool kz_on(const pty_constraints* c) { return c->kz_relax > 0.f && (c->kz_beta > 0.f || c->kz_alpha > 0.f); }

struct ConstrainLayout {
  size_t z, partial, U, lam, total;
};

static ConstrainLayout constrain_layout(const pty_geom* g, const pty_constraints* c) {
  ConstrainLayout L = {0, 0, 0, 0, 0};
  size_t off = 0;
  if (kz_on(c)) {
    L.z = off;
    off += round256(sizeof(float2) * (size_t)g->Nz * g->H * g->W);
  }
  if (c->probe_orthogonalize && g->M > 1) {
    const size_t NN = (size_t)g->N * g->N, chunks = (NN + kGramChunk - 1) / kGramChunk;
    L.partial = off;
    off += round256(sizeof(double2) * (size_t)g->M * (g->M + 1) / 2 * chunks);
    L.U = off;
    off += round256(sizeof(double2) * (size_t)g->M * g->M);
    L.lam = off;
    off += round256(sizeof(double) * g->M);
  }
  L.total = off;
  return L;
}

static int launched(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s launch failed: %s", what, cudaGetErrorString(e));
    return PTY_ECUDA;
  }
  note_launch();
  return PTY_OK;
}

static int check_constraints(const pty_geom* geom, const pty_constraints* c) {
  int rc = validate_geom(geom);
  if (rc) return rc;
  REQUIRE(c, "constraints are NULL");
  REQUIRE(c->phase_positivity >= 0.f && c->phase_positivity <= 1.f, "phase_positivity %g outside [0, 1]",
          c->phase_positivity);
  REQUIRE(c->rz_relax >= 0.f && c->rz_relax <= 1.f, "rz_relax %g outside [0, 1]", c->rz_relax);
  REQUIRE(c->rz_sigma >= 0.f && isfinite(c->rz_sigma), "rz_sigma %g must be finite and >= 0", c->rz_sigma);
  REQUIRE(c->kz_relax >= 0.f && c->kz_relax <= 1.f, "kz_relax %g outside [0, 1]", c->kz_relax);
  REQUIRE(c->kz_beta >= 0.f && isfinite(c->kz_beta) && c->kz_alpha >= 0.f && isfinite(c->kz_alpha),
          "kz_beta %g and kz_alpha %g must be finite and >= 0", c->kz_beta, c->kz_alpha);
  const bool blur = c->rz_sigma > 0.f && c->rz_relax > 0.f;
  REQUIRE(!blur || geom->Nz <= kMaxBlurSlices, "the depth blur supports Nz <= %d", kMaxBlurSlices);
  REQUIRE(!kz_on(c) || (geom->H <= kMaxLine && geom->W <= kMaxLine && geom->Nz <= kMaxBlurSlices),
          "the k_z filter supports H, W <= %d and Nz <= %d", kMaxLine, kMaxBlurSlices);
  REQUIRE(!c->probe_orthogonalize || geom->M <= kMaxOrthoModes, "orthogonalisation supports M <= %d modes",
          kMaxOrthoModes);
  return PTY_OK;
}

static int run_lines(LineArgs a, bool inverse, int io, cudaStream_t st) {
  a.pow2 = (a.L & (a.L - 1)) == 0;
  a.logL = 0;
  while ((1 << a.logL) < a.L) ++a.logL;
  int C = kLineElems / a.L;
  C = C < 1 ? 1 : C > 16 ? 16 : C;
  while (C & (C - 1)) C &= C - 1;  // a power of two
  a.C = C;
  const size_t n = (size_t)C * a.L;
  const size_t smem = sizeof(float2) * (a.pow2 ? n + a.L / 2 : 2 * n + a.L);
  long long tiles;
  if (a.axis == 0) {
    a.lines = (long long)a.Nz * a.H;
    tiles = (a.lines + C - 1) / C;
  } else {
    a.tiles_per_slice = (a.W + C - 1) / C;
    tiles = (long long)a.Nz * a.tiles_per_slice;
  }
  auto kern = io == IO_FROM_PAIR ? k_lines<false, IO_FROM_PAIR>
            : io == IO_TO_PAIR   ? k_lines<true, IO_TO_PAIR>
            : inverse            ? k_lines<true, IO_Z>
                                 : k_lines<false, IO_Z>;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                              cudaSuccess) {
    set_error("cudaFuncSetAttribute(k_lines) failed: %s", cudaGetErrorString(cudaGetLastError()));
    return PTY_ECUDA;
  }
  kern<<<(unsigned)tiles, kLineThreads, smem, st>>>(a);
  return launched("k_lines");
}

static int run_kz_filter(const pty_geom* g, float* amp, float* phase, const float* dz, const pty_constraints* c,
                         float2* z, cudaStream_t st) {
  LineArgs a;
  memset(&a, 0, sizeof(a));
  a.z = z;
  a.amp = amp;
  a.phase = phase;
  a.relax = c->kz_relax;
  a.Nz = g->Nz;
  a.H = g->H;
  a.W = g->W;
  int rc;
  a.axis = 0;
  a.L = g->W;
  if ((rc = run_lines(a, false, IO_FROM_PAIR, st))) return rc;
  a.axis = 1;
  a.L = g->H;
  if ((rc = run_lines(a, false, IO_Z, st))) return rc;
  const size_t plane = (size_t)g->H * g->W;
  int T = (int)((kConstrainSmem - sizeof(float2) * g->Nz) / (2 * sizeof(float2) * (size_t)g->Nz));
  T = T >= 128 ? 128 : T / 32 * 32;
  const size_t smem = sizeof(float2) * ((size_t)g->Nz + 2 * (size_t)g->Nz * T);
  if (smem > 48 * 1024 && cudaFuncSetAttribute(k_kz_columns, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem) != cudaSuccess) {
    set_error("cudaFuncSetAttribute(k_kz_columns) failed: %s", cudaGetErrorString(cudaGetLastError()));
    return PTY_ECUDA;
  }
  k_kz_columns<<<(unsigned)((plane + T - 1) / T), T, smem, st>>>(z, g->Nz, g->H, g->W, g->dx, dz, c->kz_beta,
                                                                 c->kz_alpha);
  if ((rc = launched("k_kz_columns"))) return rc;
  if ((rc = run_lines(a, true, IO_Z, st))) return rc;
  a.axis = 0;
  a.L = g->W;
  return run_lines(a, true, IO_TO_PAIR, st);
}

static int run_orthogonalize(const pty_geom* g, float* probe, const ConstrainLayout& L, char* ws, cudaStream_t st) {
  const int M = g->M, NN = g->N * g->N;
  const int chunks = (NN + kGramChunk - 1) / kGramChunk;
  double2* partial = reinterpret_cast<double2*>(ws + L.partial);
  double2* U = reinterpret_cast<double2*>(ws + L.U);
  double* lam = reinterpret_cast<double*>(ws + L.lam);
  float2* P = reinterpret_cast<float2*>(probe);
  int rc;
  k_gram<<<dim3(chunks, M * (M + 1) / 2), 256, 0, st>>>(P, M, NN, partial);
  if ((rc = launched("k_gram"))) return rc;
  k_ortho_eig<<<1, 32, 0, st>>>(partial, M, chunks, U, lam);
  if ((rc = launched("k_ortho_eig"))) return rc;
  const size_t smem = sizeof(double2) * M * M + sizeof(float2) * M * 128;
  k_ortho_apply<<<(NN + 127) / 128, 128, smem, st>>>(P, M, NN, U);
  return launched("k_ortho_apply");
}

}  // namespace pty

using namespace pty;

extern "C" {

size_t pty_constrain_workspace_size(const pty_geom* geom, const pty_constraints* c) {
  if (check_constraints(geom, c)) return 0;
  return constrain_layout(geom, c).total;
}

int pty_constrain(const pty_geom* geom, float* amp, float* phase, float* probe, const float* dz,
                  const pty_constraints* c, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_constraints(geom, c);
  if (rc) return rc;
  const bool blur = c->rz_sigma > 0.f && c->rz_relax > 0.f;
  const bool kz = kz_on(c), ortho = c->probe_orthogonalize != 0;
  REQUIRE(!(blur || kz || c->phase_positivity > 0.f) || (amp && phase), "amp or phase is NULL");
  REQUIRE(!amp || (aligned(amp, 4) && aligned(phase, 4)), "float arrays must be 4-byte aligned");
  REQUIRE(!kz || dz, "the k_z filter needs the slice spacing dz (device pointer)");
  REQUIRE(!ortho || (probe && aligned(probe, 8)), "probe is NULL or not 8-byte aligned");
  const ConstrainLayout L = constrain_layout(geom, c);
  REQUIRE(ws_bytes >= L.total, "workspace of %zu bytes is smaller than the %zu needed", ws_bytes, L.total);
  REQUIRE(L.total == 0 || (ws && aligned(ws, 256)), "workspace is NULL or not 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  char* w = static_cast<char*>(ws);
  if (ortho && geom->M > 1 && (rc = run_orthogonalize(geom, probe, L, w, st))) return rc;
  const size_t plane = (size_t)geom->H * geom->W, vol = (size_t)geom->Nz * plane;
  const int Ko = geom->obj_modes > 1 ? geom->obj_modes : 1;
  for (int n = 0; n < Ko; ++n) {  // each object mode is its own volume (the k_z workspace is reused)
    float* a = amp ? amp + n * vol : nullptr;
    float* p = phase ? phase + n * vol : nullptr;
    if (kz && (rc = run_kz_filter(geom, a, p, dz, c, reinterpret_cast<float2*>(w + L.z), st))) return rc;
    if (!blur && c->phase_positivity == 0.f) continue;
    const bool vec = plane % 4 == 0 && aligned(a, 16) && aligned(p, 16);
    const float sigma = blur ? c->rz_sigma : 0.f;
    rc = vec ? launch_constrain<4>(a, p, geom->Nz, plane, sigma, c->rz_relax, c->phase_positivity, st)
             : launch_constrain<1>(a, p, geom->Nz, plane, sigma, c->rz_relax, c->phase_positivity, st);
    if (rc || (rc = launched("k_constrain"))) return rc;
  }
  return PTY_OK;
}

}  // extern "C"
