// cnn.cu -- the learned initialiser of include/pty_cnn.h: bf16 implicit-GEMM convolutions on the
// tensor cores (tcgen05 with TMEM accumulators, gemm_tc.cuh: forward, input gradient, weight
// gradient), the two-channel output layer on the CUDA cores, the loss, Adam, training targets and
// stitching.
//
// Layout: activations channels-last [B][H][W][C] in bf16, so one 16-byte load gathers 8 channels of
// one tap.  GEMM views (rows x cols, reduction K):
//   forward    z[pixel][oc]   = sum_k col[pixel][k] W[oc][k],        k = (ky, kx, ic)
//   dgrad      du[pixel][ic]  = sum_k' dz[pixel'(k')][oc] Wt[ic][k'], k' = (ky, kx, oc), pixels of the
//                                (upsampled) input grid; pixel' is the output that reads it by tap
//   wgrad      dW[oc][k]      = sum_pixels dz[pixel][oc] col[pixel][k]: dz and the im2col matrix are
//                                first transposed to pixel-contiguous rows (chunks of at most 2^18
//                                pixels), then one plain GEMM per chunk, split over pixels with
//                                float atomics
// Layer 6 (upsampling x4, 2 output channels) would waste 126 of 128 GEMM columns, so it runs on the
// CUDA cores: nearest upsampling makes every output pixel read, for each tap, one low-resolution
// pixel, so the per-tap channel sums P[p][tap][o] = sum_c W[o][tap][c] a5[p][c] are formed once per
// low-resolution pixel and each output adds nine of them; the backward pass runs the same
// structure in reverse.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "gemm_mma.cuh"
#include "gemm_tc.cuh"
#include "pty_cnn.h"
#include "pty_internal.h"

namespace pty {
namespace cnn {

using bf16 = __nv_bfloat16;

struct LayerDef {
  int ic, oc, stride, up;
};
constexpr int kLayers = 6;
constexpr LayerDef kNet[kLayers] = {{1, 48, 2, 1}, {48, 96, 2, 1}, {96, 192, 2, 1},
                                    {192, 384, 2, 1}, {384, 256, 1, 2}, {256, 2, 1, 4}};
constexpr int kOut = 2;     // output channels
constexpr int kTaps6 = 18;  // layer 6: 9 taps x 2 output channels
constexpr int kC6 = 256;    // layer 6 input channels
constexpr int kPixChunk = 1 << 18;  // output pixels per weight-gradient chunk

__host__ __device__ constexpr int round64(int x) { return (x + 63) / 64 * 64; }

// ---------------------------------------------------------------------------------------------
// Plan: per-layer sizes and workspace offsets for patterns of S x S and batches of B
// ---------------------------------------------------------------------------------------------
struct Plan {
  int S, B;
  int hin[kLayers], hout[kLayers], hu[kLayers];  // input, output and upsampled-input sizes
  size_t woff[kLayers], boff[kLayers];           // offsets of weights / biases in the parameters
  int kp[kLayers], ktp[kLayers];                 // padded K of the forward and dgrad GEMMs
  // workspace pieces (byte offsets)
  size_t status, wp[kLayers], wt[kLayers], w6, act[kLayers], dz[kLayers + 1], p6, dp6, du5, lpart, colt, dzt,
      total;
  int pchunk[kLayers];  // pixels per weight-gradient chunk (multiple of 64)
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static bool make_plan(int S, int B, Plan* pl) {
  if (S < 16 || S > 512 || S % 16 != 0 || B < 0 || B > 1024) return false;
  Plan p;
  memset(&p, 0, sizeof(p));
  p.S = S;
  p.B = B;
  int h = S;
  size_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    p.hin[l] = h;
    p.hu[l] = h * kNet[l].up;
    p.hout[l] = (p.hu[l] + kNet[l].stride - 1) / kNet[l].stride;
    h = p.hout[l];
    p.woff[l] = o;
    o += (size_t)9 * kNet[l].ic * kNet[l].oc;
    p.boff[l] = o;
    o += kNet[l].oc;
    p.kp[l] = round64(9 * kNet[l].ic);
    p.ktp[l] = round64(9 * kNet[l].oc);
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t r = off;
    off += align256(bytes);
    return r;
  };
  p.status = take(sizeof(int) * 64);
  for (int l = 0; l < 5; ++l) {
    p.wp[l] = take(sizeof(bf16) * kNet[l].oc * p.kp[l]);
    if (l > 0) p.wt[l] = take(sizeof(bf16) * kNet[l].ic * p.ktp[l]);
  }
  p.w6 = take(sizeof(float) * kTaps6 * kC6);
  for (int l = 0; l < 5; ++l) p.act[l] = take(sizeof(bf16) * (size_t)B * p.hout[l] * p.hout[l] * kNet[l].oc);
  for (int l = 0; l < 5; ++l) p.dz[l] = take(sizeof(bf16) * (size_t)B * p.hout[l] * p.hout[l] * kNet[l].oc);
  p.dz[5] = take(sizeof(bf16) * (size_t)B * p.hout[5] * p.hout[5] * kOut);
  const size_t lowres = (size_t)B * p.hout[4] * p.hout[4];
  p.p6 = take(sizeof(float) * lowres * kTaps6);
  p.dp6 = take(sizeof(float) * lowres * kTaps6);
  p.du5 = take(sizeof(float) * (size_t)B * p.hu[4] * p.hu[4] * kNet[4].ic);
  p.lpart = take(sizeof(double) * 1024);
  // weight gradients run over chunks of at most kPixChunk output pixels, with the im2col matrix and
  // dL/dz transposed to pixel-contiguous rows
  size_t colt = 0, dzt = 0;
  for (int l = 0; l < 5; ++l) {
    const size_t pix = (size_t)B * p.hout[l] * p.hout[l];
    p.pchunk[l] = (int)((pix < (size_t)kPixChunk ? (pix + 63) / 64 * 64 : (size_t)kPixChunk));
    if (p.pchunk[l] < 64) p.pchunk[l] = 64;
    colt = colt > (size_t)9 * kNet[l].ic * p.pchunk[l] ? colt : (size_t)9 * kNet[l].ic * p.pchunk[l];
    dzt = dzt > (size_t)kNet[l].oc * p.pchunk[l] ? dzt : (size_t)kNet[l].oc * p.pchunk[l];
  }
  p.colt = take(sizeof(bf16) * colt);
  p.dzt = take(sizeof(bf16) * dzt);
  p.total = off;
  *pl = p;
  return true;
}

size_t param_count() {
  size_t n = 0;
  for (int l = 0; l < kLayers; ++l) n += (size_t)9 * kNet[l].ic * kNet[l].oc + kNet[l].oc;
  return n;
}


// ---------------------------------------------------------------------------------------------
// Weight packing: FP32 parameters -> bf16 GEMM operands (zero-padded K) and layer 6's table
// ---------------------------------------------------------------------------------------------
struct PackArgs {
  const float* params;
  bf16* wp[5];  // [OC][kp]
  bf16* wt[5];  // [IC][ktp] (layers 2..5)
  float* w6;    // [18][256]: row tap * 2 + o, bf16-rounded
  size_t woff[kLayers];
  int kp[kLayers], ktp[kLayers], ic[kLayers], oc[kLayers];
};

__global__ void k_pack(PackArgs a) {
  // segments: wp of layers 0..4, wt of layers 1..4, w6
  size_t seg[10];
  int n = 0;
  for (int l = 0; l < 5; ++l) seg[n++] = (size_t)a.oc[l] * a.kp[l];
  for (int l = 1; l < 5; ++l) seg[n++] = (size_t)a.ic[l] * a.ktp[l];
  seg[n++] = (size_t)kTaps6 * kC6;
  size_t total = 0;
  for (int q = 0; q < n; ++q) total += seg[q];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    size_t e = i;
    int q = 0;
    while (e >= seg[q]) e -= seg[q++];
    if (q < 5) {  // forward operand of layer q: W[oc][k], k = (ky, kx, ic)
      const int l = q, K9 = 9 * a.ic[l];
      const int oc = (int)(e / a.kp[l]), k = (int)(e % a.kp[l]);
      a.wp[l][e] = __float2bfloat16_rn(k < K9 ? a.params[a.woff[l] + (size_t)oc * K9 + k] : 0.f);
    } else if (q < 9) {  // dgrad operand of layer l: Wt[ic][k'] = W[oc][tap][ic], k' = tap * OC + oc
      const int l = q - 4, IC = a.ic[l], OC = a.oc[l];
      const int ic = (int)(e / a.ktp[l]), kk = (int)(e % a.ktp[l]);
      float w = 0.f;
      if (kk < 9 * OC) {
        const int tap = kk / OC, oc = kk % OC;
        w = a.params[a.woff[l] + ((size_t)oc * 9 + tap) * IC + ic];
      }
      a.wt[l][e] = __float2bfloat16_rn(w);
    } else {  // layer 6: w6[tap * 2 + o][c] = W[o][tap][c]
      const int j = (int)(e / kC6), c = (int)(e % kC6);
      const int tap = j / kOut, o = j % kOut;
      a.w6[e] = __bfloat162float(__float2bfloat16_rn(a.params[a.woff[5] + ((size_t)o * 9 + tap) * kC6 + c]));
    }
  }
}

// ---------------------------------------------------------------------------------------------
// GEMM operand loaders (8 consecutive reduction elements per call, zeros outside)
// ---------------------------------------------------------------------------------------------
union Pack8 {
  uint4 u;
  bf16 h[8];
};

__device__ __forceinline__ bf16 input_value(const float* I, float s_in, int S, int b, int y, int x) {
  return __float2bfloat16_rn(s_in * log1pf(__ldg(I + ((size_t)b * S + y) * S + x)));
}

// Forward of layer 1: rows = output pixels, k = tap (9 of 32 used); values from the FP32 patterns.
struct InputIm2col {
  const float* I;
  float s_in;
  int S, B, hout;
  __device__ __forceinline__ uint4 operator()(int m, int k) const {
    Pack8 r;
    r.u = make_uint4(0u, 0u, 0u, 0u);
    if (m >= B * hout * hout || k >= 9) return r.u;
    const int b = m / (hout * hout), rem = m % (hout * hout), oy = rem / hout, ox = rem % hout;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int tap = k + e;
      if (tap < 9) {
        const int y = 2 * oy + tap / 3 - 1, x = 2 * ox + tap % 3 - 1;
        if (y >= 0 && y < S && x >= 0 && x < S) r.h[e] = input_value(I, s_in, S, b, y, x);
      }
    }
    return r.u;
  }
};

// Forward of layers 2..5: 8 channels of one tap of the (upsampled) input, 16-byte loads.
struct Im2col {
  const bf16* a;  // [B][hin][hin][ic]
  int B, hin, hu, hout, ic, stride, up;
  __device__ __forceinline__ uint4 operator()(int m, int k) const {
    if (m >= B * hout * hout || k >= 9 * ic) return make_uint4(0u, 0u, 0u, 0u);
    const int b = m / (hout * hout), rem = m % (hout * hout), oy = rem / hout, ox = rem % hout;
    const int tap = k / ic, c0 = k - tap * ic;
    const int uy = stride * oy + tap / 3 - 1, ux = stride * ox + tap % 3 - 1;
    if (uy < 0 || uy >= hu || ux < 0 || ux >= hu) return make_uint4(0u, 0u, 0u, 0u);
    return __ldg(reinterpret_cast<const uint4*>(a + (((size_t)b * hin + uy / up) * hin + ux / up) * ic + c0));
  }
  // cursor: the output pixel decoded once, (tap, channel) stepped through K
  struct Cursor {
    const bf16* img;  // sample b of the input, or nullptr past the last row
    int y0, x0;       // stride * (oy, ox) - 1 on the upsampled grid
    int ky, kx, c0;
  };
  __device__ __forceinline__ Cursor cursor(int m, int k) const {
    Cursor c;
    c.img = nullptr;
    c.y0 = c.x0 = 0;
    if (m < B * hout * hout) {
      const int b = m / (hout * hout), rem = m % (hout * hout);
      c.img = a + (size_t)b * hin * hin * ic;
      c.y0 = stride * (rem / hout) - 1;
      c.x0 = stride * (rem % hout) - 1;
    }
    const int tap = k / ic;
    c.ky = tap / 3;
    c.kx = tap % 3;
    c.c0 = k - tap * ic;
    return c;
  }
  __device__ __forceinline__ uint4 load(const Cursor& c) const {
    const int uy = c.y0 + c.ky, ux = c.x0 + c.kx;
    if (!c.img || c.ky > 2 || uy < 0 || uy >= hu || ux < 0 || ux >= hu) return make_uint4(0u, 0u, 0u, 0u);
    const int sh = up == 2 ? 1 : 0;  // up is 1 or 2 for the layers that gather this way
    return __ldg(reinterpret_cast<const uint4*>(c.img + ((size_t)(uy >> sh) * hin + (ux >> sh)) * ic + c.c0));
  }
  __device__ __forceinline__ void advance(Cursor& c, int dk) const {
    c.c0 += dk;
    while (c.c0 >= ic) {
      c.c0 -= ic;
      if (++c.kx == 3) {
        c.kx = 0;
        ++c.ky;
      }
    }
  }
};

// Input gradient of layers 2..5: rows = pixels of the upsampled input grid, k' = (tap, oc); the
// output pixel that reads (uy, ux) through tap (ky, kx) is ((uy + 1 - ky) / s, (ux + 1 - kx) / s).
struct DgradGather {
  const bf16* dz;  // [B][hout][hout][oc]
  int B, hu, hout, oc, stride;
  __device__ __forceinline__ uint4 operator()(int m, int k) const {
    if (m >= B * hu * hu || k >= 9 * oc) return make_uint4(0u, 0u, 0u, 0u);
    const int b = m / (hu * hu), rem = m % (hu * hu), uy = rem / hu, ux = rem % hu;
    const int tap = k / oc, o0 = k - tap * oc;
    const int ty = uy + 1 - tap / 3, tx = ux + 1 - tap % 3;
    if (ty < 0 || tx < 0 || ty % stride || tx % stride) return make_uint4(0u, 0u, 0u, 0u);
    const int oy = ty / stride, ox = tx / stride;
    if (oy >= hout || ox >= hout) return make_uint4(0u, 0u, 0u, 0u);
    return __ldg(reinterpret_cast<const uint4*>(dz + (((size_t)b * hout + oy) * hout + ox) * oc + o0));
  }
  struct Cursor {
    const bf16* img;  // sample b of dz, or nullptr past the last row
    int y1, x1;       // (uy + 1, ux + 1)
    int ky, kx, o0;
  };
  __device__ __forceinline__ Cursor cursor(int m, int k) const {
    Cursor c;
    c.img = nullptr;
    c.y1 = c.x1 = 0;
    if (m < B * hu * hu) {
      const int b = m / (hu * hu), rem = m % (hu * hu);
      c.img = dz + (size_t)b * hout * hout * oc;
      c.y1 = rem / hu + 1;
      c.x1 = rem % hu + 1;
    }
    const int tap = k / oc;
    c.ky = tap / 3;
    c.kx = tap % 3;
    c.o0 = k - tap * oc;
    return c;
  }
  __device__ __forceinline__ uint4 load(const Cursor& c) const {
    const int ty = c.y1 - c.ky, tx = c.x1 - c.kx;
    const int sm = stride - 1, sh = stride == 2 ? 1 : 0;  // stride is 1 or 2
    if (!c.img || c.ky > 2 || ty < 0 || tx < 0 || ((ty | tx) & sm)) return make_uint4(0u, 0u, 0u, 0u);
    const int oy = ty >> sh, ox = tx >> sh;
    if (oy >= hout || ox >= hout) return make_uint4(0u, 0u, 0u, 0u);
    return __ldg(reinterpret_cast<const uint4*>(c.img + ((size_t)oy * hout + ox) * oc + c.o0));
  }
  __device__ __forceinline__ void advance(Cursor& c, int dk) const {
    c.o0 += dk;
    while (c.o0 >= oc) {
      c.o0 -= oc;
      if (++c.kx == 3) {
        c.kx = 0;
        ++c.ky;
      }
    }
  }
};

// ---------------------------------------------------------------------------------------------
// GEMM epilogues
// ---------------------------------------------------------------------------------------------
struct FwdEpi {  // a = bf16(relu(z + bias))
  bf16* out;
  const float* bias;
  int rows, oc;
  __device__ __forceinline__ void operator()(int row, int col, float v0, float v1) const {
    if (row >= rows || col >= oc) return;
    v0 = fmaxf(v0 + bias[col], 0.f);
    v1 = fmaxf(v1 + bias[col + 1], 0.f);
    *reinterpret_cast<__nv_bfloat162*>(out + (size_t)row * oc + col) = __floats2bfloat162_rn(v0, v1);
  }
};
struct DgradEpi {  // dz of the layer below = bf16(du * (a > 0)) (no upsampling between)
  bf16* dz;
  const bf16* a;
  int rows, ic;
  __device__ __forceinline__ void operator()(int row, int col, float v0, float v1) const {
    if (row >= rows || col >= ic) return;
    const size_t e = (size_t)row * ic + col;
    const __nv_bfloat162 av = *reinterpret_cast<const __nv_bfloat162*>(a + e);
    v0 = __low2float(av) > 0.f ? v0 : 0.f;
    v1 = __high2float(av) > 0.f ? v1 : 0.f;
    *reinterpret_cast<__nv_bfloat162*>(dz + e) = __floats2bfloat162_rn(v0, v1);
  }
};
struct StoreEpi {  // FP32 store (gradient on the upsampled grid)
  float* out;
  int rows, cols;
  __device__ __forceinline__ void operator()(int row, int col, float v0, float v1) const {
    if (row >= rows || col >= cols) return;
    *reinterpret_cast<float2*>(out + (size_t)row * cols + col) = make_float2(v0, v1);
  }
};
struct WgradEpi {  // split-K partial sums of dW[oc][k]
  float* g;
  int oc, k9;
  __device__ __forceinline__ void operator()(int row, int col, float v0, float v1) const {
    if (row >= oc) return;
    if (col < k9) atomicAdd(g + (size_t)row * k9 + col, v0);
    if (col + 1 < k9) atomicAdd(g + (size_t)row * k9 + col + 1, v1);
  }
};


// ---------------------------------------------------------------------------------------------
// Layer 6 on the CUDA cores
// ---------------------------------------------------------------------------------------------
// P[p][j] = sum_c w6[j][c] a5[p][c]: one warp per low-resolution pixel, 8 channels per lane.
__global__ void __launch_bounds__(256) k_l6_sums(const bf16* __restrict__ a5, const float* __restrict__ w6,
                                                 float* __restrict__ P, int npix) {
  __shared__ float w[kTaps6 * kC6];
  for (int i = threadIdx.x; i < kTaps6 * kC6; i += blockDim.x) w[i] = w6[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int p = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (p >= npix) return;
  Pack8 v;
  v.u = __ldg(reinterpret_cast<const uint4*>(a5 + (size_t)p * kC6 + lane * 8));
  float x[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) x[e] = __bfloat162float(v.h[e]);
  float acc[kTaps6];
#pragma unroll
  for (int j = 0; j < kTaps6; ++j) {
    float t = 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) t = fmaf(w[j * kC6 + lane * 8 + e], x[e], t);
    acc[j] = t;
  }
#pragma unroll
  for (int j = 0; j < kTaps6; ++j)
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < kTaps6; ++j) P[(size_t)p * kTaps6 + j] = acc[j];
  }
}

// out[b][y][x][o] = bias[o] + sum_tap P[b][(y + ky - 1) / 4][(x + kx - 1) / 4][tap][o] over taps
// inside the upsampled grid (hs = 4 * hl pixels per side).
__global__ void k_l6_out(const float* __restrict__ P, const float* __restrict__ bias, float* __restrict__ out, int B,
                         int hl) {
  const int hs = 4 * hl;
  const size_t n = (size_t)B * hs * hs * kOut;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(i % kOut);
    const size_t px = i / kOut;
    const int x = (int)(px % hs), y = (int)((px / hs) % hs), b = (int)(px / ((size_t)hs * hs));
    float acc = bias[o];
    for (int tap = 0; tap < 9; ++tap) {
      const int uy = y + tap / 3 - 1, ux = x + tap % 3 - 1;
      if (uy < 0 || uy >= hs || ux < 0 || ux >= hs) continue;
      acc += P[(((size_t)b * hl + uy / 4) * hl + ux / 4) * kTaps6 + tap * kOut + o];
    }
    out[i] = acc;
  }
}

// Loss partial sums (FP64 per block, fixed order) and dz6 = bf16(2 (pred - Y) / n).
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ pred, const float* __restrict__ Y,
                                              bf16* __restrict__ dz6, double* __restrict__ lpart, size_t n) {
  double acc = 0.0;
  const float g = (float)(2.0 / (double)n);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = pred[i] - Y[i];
    acc += (double)d * d;
    dz6[i] = __float2bfloat16_rn(g * d);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
}
__global__ void k_loss_final(const double* __restrict__ lpart, int nb, size_t n, double* loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nb; ++i) t += lpart[i];
    *loss = t / (double)n;
  }
}

// dP[p][tap][o] = sum of dz6 over the output pixels that read low-resolution pixel p through tap:
// y + ky - 1 in [4 sy, 4 sy + 3] and inside the grid.
__global__ void k_l6_dsums(const bf16* __restrict__ dz6, float* __restrict__ dP, int B, int hl) {
  const int hs = 4 * hl;
  const size_t n = (size_t)B * hl * hl * kTaps6;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % kTaps6), tap = j / kOut, o = j % kOut;
    const size_t p = i / kTaps6;
    const int sx = (int)(p % hl), sy = (int)((p / hl) % hl), b = (int)(p / ((size_t)hl * hl));
    const int ky = tap / 3, kx = tap % 3;
    float acc = 0.f;
    for (int dy = 0; dy < 4; ++dy) {
      const int y = 4 * sy + dy + 1 - ky;
      if (y < 0 || y >= hs) continue;
      for (int dx = 0; dx < 4; ++dx) {
        const int x = 4 * sx + dx + 1 - kx;
        if (x < 0 || x >= hs) continue;
        acc += __bfloat162float(dz6[(((size_t)b * hs + y) * hs + x) * kOut + o]);
      }
    }
    dP[i] = acc;
  }
}

// dz5[p][c] = bf16((a5[p][c] > 0) sum_j dP[p][j] w6[j][c]).
__global__ void __launch_bounds__(256) k_l6_dgrad(const float* __restrict__ dP, const float* __restrict__ w6,
                                                  const bf16* __restrict__ a5, bf16* __restrict__ dz5, int npix) {
  const int p = blockIdx.x, c = threadIdx.x;  // blockDim = 256 channels
  if (p >= npix) return;
  __shared__ float d[kTaps6];
  if (c < kTaps6) d[c] = dP[(size_t)p * kTaps6 + c];
  __syncthreads();
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < kTaps6; ++j) acc = fmaf(d[j], __ldg(w6 + j * kC6 + c), acc);
  const size_t e = (size_t)p * kC6 + c;
  dz5[e] = __float2bfloat16_rn(__bfloat162float(a5[e]) > 0.f ? acc : 0.f);
}

// dW6[o][tap][c] += sum over a chunk of pixels of dP[p][tap * 2 + o] a5[p][c].
__global__ void __launch_bounds__(256) k_l6_wgrad(const float* __restrict__ dP, const bf16* __restrict__ a5,
                                                  float* __restrict__ gW6, int npix, int chunk) {
  const int j = blockIdx.y, c = threadIdx.x, p0 = blockIdx.x * chunk;
  const int p1 = p0 + chunk < npix ? p0 + chunk : npix;
  float acc = 0.f;
  for (int p = p0; p < p1; ++p) acc = fmaf(__ldg(dP + (size_t)p * kTaps6 + j), __bfloat162float(a5[(size_t)p * kC6 + c]), acc);
  const int tap = j / kOut, o = j % kOut;
  atomicAdd(gW6 + ((size_t)o * 9 + tap) * kC6 + c, acc);
}

// ---------------------------------------------------------------------------------------------
// Bias gradients, upsampling adjoint, Adam
// ---------------------------------------------------------------------------------------------
// gb[c] += sum over a chunk of pixels of dz[p][c].
__global__ void k_bias_grad(const bf16* __restrict__ dz, float* __restrict__ gb, size_t npix, int C, int chunk) {
  const size_t p0 = (size_t)blockIdx.x * chunk;
  const size_t p1 = p0 + chunk < npix ? p0 + chunk : npix;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float acc = 0.f;
    for (size_t p = p0; p < p1; ++p) acc += __bfloat162float(dz[p * C + c]);
    atomicAdd(gb + c, acc);
  }
}

// dz[b][y][x][c] = bf16((a > 0) sum of the f x f block of du on the upsampled grid).
__global__ void k_upsample_grad(const float* __restrict__ du, const bf16* __restrict__ a, bf16* __restrict__ dz, int B,
                                int h, int C, int f) {
  const size_t n = (size_t)B * h * h * C;
  const int hu = h * f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const size_t px = i / C;
    const int x = (int)(px % h), y = (int)((px / h) % h), b = (int)(px / ((size_t)h * h));
    float acc = 0.f;
    for (int dy = 0; dy < f; ++dy)
      for (int dx = 0; dx < f; ++dx) acc += du[(((size_t)b * hu + f * y + dy) * hu + f * x + dx) * C + c];
    dz[i] = __float2bfloat16_rn(__bfloat162float(a[i]) > 0.f ? acc : 0.f);
  }
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       size_t n, float lr, float b1, float b2, float eps, float bc1, float bc2_sqrt) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= (lr / bc1) * mi / (sqrtf(vi) / bc2_sqrt + eps);
  }
}

// ---------------------------------------------------------------------------------------------
// Targets and stitching
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void window_corner(const float* pos, int j, int S, int H, int W, int* i0, int* i1) {
  float r0 = rintf(pos[2 * j]), r1 = rintf(pos[2 * j + 1]);  // half to even, as the forward model
  if (!isfinite(r0)) r0 = 0.f;
  if (!isfinite(r1)) r1 = 0.f;
  *i0 = (int)fminf(fmaxf(r0, 0.f), (float)(H - S));
  *i1 = (int)fminf(fmaxf(r1, 0.f), (float)(W - S));
}

__global__ void k_targets(int S, int Nz, int H, int W, const float* __restrict__ amp, const float* __restrict__ phase,
                          const float* __restrict__ pos, const int32_t* __restrict__ idx, int B, float* __restrict__ Y) {
  const int h = S / 2, q = S / 4;
  const size_t n = (size_t)B * h * h;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % h), y = (int)((i / h) % h), b = (int)(i / ((size_t)h * h));
    int i0, i1;
    window_corner(pos, idx[b], S, H, W, &i0, &i1);
    const size_t e = (size_t)(i0 + q + y) * W + (i1 + q + x);
    double ph = 0.0, la = 0.0;
    for (int s = 0; s < Nz; ++s) {
      ph += phase[(size_t)s * H * W + e];
      la += log((double)amp[(size_t)s * H * W + e]);
    }
    Y[2 * i] = (float)ph;
    Y[2 * i + 1] = (float)la;
  }
}

__global__ void k_stitch(int S, int H, int W, const float* __restrict__ pred, const float* __restrict__ pos,
                         const int32_t* __restrict__ idx, int B, const float* __restrict__ wgt, float* __restrict__ num,
                         float* __restrict__ den) {
  const int h = S / 2, q = S / 4;
  const size_t n = (size_t)B * h * h;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % h), y = (int)((i / h) % h), b = (int)(i / ((size_t)h * h));
    int i0, i1;
    window_corner(pos, idx[b], S, H, W, &i0, &i1);
    const size_t e = (size_t)(i0 + q + y) * W + (i1 + q + x);
    const float w = wgt[y * h + x];
    atomicAdd(num + 2 * e, w * pred[2 * i]);
    atomicAdd(num + 2 * e + 1, w * pred[2 * i + 1]);
    atomicAdd(den + e, w);
  }
}

__global__ void k_stitch_finish(int Nz, int H, int W, const float* __restrict__ num, const float* __restrict__ den,
                                float* __restrict__ amp, float* __restrict__ phase) {
  const size_t n = (size_t)H * W;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = den[i];
    const float ph = d > 0.f ? num[2 * i] / d / Nz : 0.f;
    const float am = d > 0.f ? expf(num[2 * i + 1] / d / Nz) : 1.f;
    for (int s = 0; s < Nz; ++s) {
      phase[(size_t)s * n + i] = ph;
      amp[(size_t)s * n + i] = am;
    }
  }
}


// ---------------------------------------------------------------------------------------------
// Weight-gradient operands with pixel-contiguous rows
// ---------------------------------------------------------------------------------------------
// colT[k][m - p0] = im2col[m][k] for k = (tap, ic) < 9 IC and output pixels m in [p0, p0 + P); zero
// past the last pixel (layers 2..5, ic a multiple of 8).  A thread takes one pixel and 8 channels:
// per tap one 16-byte load and 8 stores into 8 rows; consecutive threads take consecutive pixels, so
// every row is written 64 bytes per warp at a time.
__global__ void k_im2col_t(const bf16* __restrict__ a, bf16* __restrict__ colt, int B, int hin, int hu, int hout,
                           int ic, int stride, int up, int p0, int P) {
  const int hw = hout * hout, pixels = B * hw, groups = ic / 8;
  const size_t n = (size_t)groups * P;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int mm = (int)(i % P), c0 = 8 * (int)(i / P), m = p0 + mm;
    int b = 0, y0 = -1 << 20, x0 = -1 << 20;
    if (m < pixels) {
      b = m / hw;
      const int rem = m % hw;
      y0 = stride * (rem / hout) - 1;
      x0 = stride * (rem % hout) - 1;
    }
    const bf16* img = a + (size_t)b * hin * hin * ic + c0;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int uy = y0 + tap / 3, ux = x0 + tap % 3;
      union {
        uint4 u;
        bf16 h[8];
      } v;
      v.u = make_uint4(0u, 0u, 0u, 0u);
      if (uy >= 0 && uy < hu && ux >= 0 && ux < hu)
        v.u = __ldg(reinterpret_cast<const uint4*>(img + ((size_t)(uy / up) * hin + ux / up) * ic));
      bf16* row = colt + ((size_t)tap * ic + c0) * P + mm;
#pragma unroll
      for (int e = 0; e < 8; ++e) row[(size_t)e * P] = v.h[e];
    }
  }
}

// Layer 1 (one channel from the patterns): colT[tap][m - p0], threads along m.
__global__ void k_im2col_t1(const float* __restrict__ I, float s_in, bf16* __restrict__ colt, int B, int S, int hout,
                            int p0, int P) {
  const size_t n = (size_t)9 * P;
  const int hw = hout * hout, pixels = B * hw;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int m = p0 + (int)(i % P), tap = (int)(i / P);
    bf16 v = __float2bfloat16_rn(0.f);
    if (m < pixels) {
      const int b = m / hw, rem = m % hw, oy = rem / hout, ox = rem % hout;
      const int y = 2 * oy + tap / 3 - 1, x = 2 * ox + tap % 3 - 1;
      if (y >= 0 && y < S && x >= 0 && x < S) v = input_value(I, s_in, S, b, y, x);
    }
    colt[i] = v;
  }
}

// dzT[c][m - p0] = dz[m][c] for m in [p0, p0 + P) (zero past the last pixel), 32 x 32 tiles through
// shared memory, and the bias gradient: gb[c] += the tile's sum over its pixels.
__global__ void k_dz_t(const bf16* __restrict__ dz, bf16* __restrict__ dzt, float* __restrict__ gb, int pixels, int C,
                       int p0, int P) {
  __shared__ bf16 tile[32][34];
  __shared__ float colsum[8][32];
  const int mt = blockIdx.x * 32, ct = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  float acc = 0.f;
  for (int j = ty; j < 32; j += 8) {
    const int m = p0 + mt + j, c = ct + tx;
    const bf16 v = (m < pixels && mt + j < P && c < C) ? dz[(size_t)m * C + c] : __float2bfloat16_rn(0.f);
    tile[j][tx] = v;
    acc += __bfloat162float(v);
  }
  colsum[ty][tx] = acc;
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int c = ct + j, mm = mt + tx;
    if (c < C && mm < P) dzt[(size_t)c * P + mm] = tile[tx][j];
  }
  if (ty == 0 && ct + tx < C) {
    float t = 0.f;
#pragma unroll
    for (int r = 0; r < 8; ++r) t += colsum[r][tx];
    atomicAdd(gb + ct + tx, t);
  }
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
#define CNN_CHECK(what)                                                  \
  do {                                                                   \
    cudaError_t e_ = cudaGetLastError();                                 \
    if (e_ != cudaSuccess) {                                             \
      set_error("%s launch failed: %s", what, cudaGetErrorString(e_));   \
      return PTY_ECUDA;                                                  \
    }                                                                    \
    note_launch();                                                       \
  } while (0)

static unsigned blocks_for(size_t n, unsigned cap = 152 * 16) {
  const size_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <class LA, class LB, class Epi>
static int gemm(const LA& la, const LB& lb, int rows, int cols, int K, const Epi& epi, int* status, cudaStream_t st,
                int splits = 1) {
#if PTY_GEMM_LEGACY
  const int kt_all = (K + GB_K - 1) / GB_K;
  if (splits > kt_all) splits = kt_all;
  if (splits < 1) splits = 1;
  const int kt_per = (kt_all + splits - 1) / splits;
  const dim3 grid((cols + GB_N - 1) / GB_N, (rows + GB_M - 1) / GB_M, (kt_all + kt_per - 1) / kt_per);
  k_gemm_tn<bf16, LA, LB, Epi, true><<<grid, GB_THREADS, 0, st>>>(la, lb, kt_all * GB_K, kt_per, epi);
  (void)status;
  CNN_CHECK("k_gemm_tn");
#else
  // tcgen05 tiles of 128 x BN, BN matched to the column count; every 64-wide K block is promoted to
  // a round-to-nearest FP32 sum (see k_gemm_tc)
  cudaError_t e;
  if (cols <= 64) {
    e = launch_gemm_tc<bf16, 64, true>(la, lb, rows, cols, K, epi, status, st, splits);
  } else if (cols % 256 == 0) {
    e = launch_gemm_tc<bf16, 256, true>(la, lb, rows, cols, K, epi, status, st, splits);
  } else {
    e = launch_gemm_tc<bf16, 128, true>(la, lb, rows, cols, K, epi, status, st, splits);
  }
  if (e != cudaSuccess) {
    set_error("k_gemm_tc launch failed: %s", cudaGetErrorString(e));
    return PTY_ECUDA;
  }
  note_launch();
#endif
  return PTY_OK;
}

struct Buffers {
  int* status;
  bf16 *wp[5], *wt[5], *act[5], *dz[6];
  float *w6, *p6, *dp6, *du5;
  double* lpart;
  bf16 *colt, *dzt;
};

static Buffers carve(const Plan& pl, void* ws) {
  char* base = static_cast<char*>(ws);
  Buffers b;
  memset(&b, 0, sizeof(b));
  b.status = reinterpret_cast<int*>(base + pl.status);
  for (int l = 0; l < 5; ++l) {
    b.wp[l] = reinterpret_cast<bf16*>(base + pl.wp[l]);
    if (l > 0) b.wt[l] = reinterpret_cast<bf16*>(base + pl.wt[l]);
    b.act[l] = reinterpret_cast<bf16*>(base + pl.act[l]);
    b.dz[l] = reinterpret_cast<bf16*>(base + pl.dz[l]);
  }
  b.dz[5] = reinterpret_cast<bf16*>(base + pl.dz[5]);
  b.w6 = reinterpret_cast<float*>(base + pl.w6);
  b.p6 = reinterpret_cast<float*>(base + pl.p6);
  b.dp6 = reinterpret_cast<float*>(base + pl.dp6);
  b.du5 = reinterpret_cast<float*>(base + pl.du5);
  b.lpart = reinterpret_cast<double*>(base + pl.lpart);
  b.colt = reinterpret_cast<bf16*>(base + pl.colt);
  b.dzt = reinterpret_cast<bf16*>(base + pl.dzt);
  return b;
}

// Pack the weights and run layers 1..6; pred[B][S/2][S/2][2].
static int run_forward(const Plan& pl, const Buffers& bu, const float* params, const float* I, float s_in, float* pred,
                       cudaStream_t st) {
  PackArgs pa;
  pa.params = params;
  for (int l = 0; l < 5; ++l) {
    pa.wp[l] = bu.wp[l];
    pa.wt[l] = bu.wt[l];
  }
  pa.w6 = bu.w6;
  for (int l = 0; l < kLayers; ++l) {
    pa.woff[l] = pl.woff[l];
    pa.kp[l] = pl.kp[l];
    pa.ktp[l] = pl.ktp[l];
    pa.ic[l] = kNet[l].ic;
    pa.oc[l] = kNet[l].oc;
  }
  if (cudaMemsetAsync(bu.status, 0, sizeof(int), st) != cudaSuccess) {
    set_error("cudaMemsetAsync failed: %s", cudaGetErrorString(cudaGetLastError()));
    return PTY_ECUDA;
  }
  k_pack<<<152 * 4, 256, 0, st>>>(pa);
  CNN_CHECK("k_pack");
  const int B = pl.B;
  if (B == 0) return PTY_OK;
  for (int l = 0; l < 5; ++l) {
    const LayerDef& L = kNet[l];
    const int rows = B * pl.hout[l] * pl.hout[l];
    PlainLoader<bf16> lb{bu.wp[l], (size_t)pl.kp[l], L.oc};
    FwdEpi epi{bu.act[l], params + pl.boff[l], rows, L.oc};
    int rc;
    if (l == 0) {
      rc = gemm(InputIm2col{I, s_in, pl.S, B, pl.hout[0]}, lb, rows, L.oc, pl.kp[l], epi, bu.status, st);
    } else {
      rc = gemm(Im2col{bu.act[l - 1], B, pl.hin[l], pl.hu[l], pl.hout[l], L.ic, L.stride, L.up}, lb, rows, L.oc,
                pl.kp[l], epi, bu.status, st);
    }
    if (rc) return rc;
  }
  const int hl = pl.hout[4], npix = B * hl * hl;
  k_l6_sums<<<(npix + 7) / 8, 256, 0, st>>>(bu.act[4], bu.w6, bu.p6, npix);
  CNN_CHECK("k_l6_sums");
  k_l6_out<<<blocks_for((size_t)B * 16 * hl * hl * kOut), 256, 0, st>>>(bu.p6, params + pl.boff[5], pred, B, hl);
  CNN_CHECK("k_l6_out");
  return PTY_OK;
}

// Loss, then gradients of every layer (grad zeroed here).
static int run_backward(const Plan& pl, const Buffers& bu, const float* I, float s_in, const float* pred, const float* Y,
                        double* loss, float* grad, cudaStream_t st) {
  const int B = pl.B;
  if (cudaMemsetAsync(grad, 0, sizeof(float) * param_count(), st) != cudaSuccess) {
    set_error("cudaMemsetAsync failed");
    return PTY_ECUDA;
  }
  if (B == 0) {
    if (cudaMemsetAsync(loss, 0, sizeof(double), st) != cudaSuccess) {
      set_error("cudaMemsetAsync failed");
      return PTY_ECUDA;
    }
    return PTY_OK;
  }
  const int hs = pl.hout[5], hl = pl.hout[4];
  const size_t nout = (size_t)B * hs * hs * kOut;
  const unsigned lb = blocks_for(nout, 1024);
  k_loss<<<lb, 256, 0, st>>>(pred, Y, bu.dz[5], bu.lpart, nout);
  CNN_CHECK("k_loss");
  k_loss_final<<<1, 32, 0, st>>>(bu.lpart, (int)lb, nout, loss);
  CNN_CHECK("k_loss_final");
  // layer 6
  const int npix = B * hl * hl;
  k_l6_dsums<<<blocks_for((size_t)npix * kTaps6), 256, 0, st>>>(bu.dz[5], bu.dp6, B, hl);
  CNN_CHECK("k_l6_dsums");
  k_l6_dgrad<<<npix, kC6, 0, st>>>(bu.dp6, bu.w6, bu.act[4], bu.dz[4], npix);
  CNN_CHECK("k_l6_dgrad");
  const int chunk = 256;
  k_l6_wgrad<<<dim3((npix + chunk - 1) / chunk, kTaps6), kC6, 0, st>>>(bu.dp6, bu.act[4], grad + pl.woff[5], npix,
                                                                       chunk);
  CNN_CHECK("k_l6_wgrad");
  const size_t pix6 = (size_t)B * hs * hs;
  k_bias_grad<<<(unsigned)((pix6 + 1023) / 1024), 256, 0, st>>>(bu.dz[5], grad + pl.boff[5], pix6, kOut, 1024);
  CNN_CHECK("k_bias_grad");
  // layers 5..1
  for (int l = 4; l >= 0; --l) {
    const LayerDef& L = kNet[l];
    const int pixels = B * pl.hout[l] * pl.hout[l];
    const int k9 = 9 * L.ic;
    // dW[oc][k] = sum over pixels of dz[m][oc] im2col[m][k], chunk by chunk, both operands
    // transposed to pixel-contiguous rows first (plain 16-byte loads in the GEMM)
    const int P = pl.pchunk[l];
    for (int p0 = 0; p0 < pixels; p0 += P) {
      if (l == 0) {
        k_im2col_t1<<<blocks_for((size_t)9 * P), 256, 0, st>>>(I, s_in, bu.colt, B, pl.S, pl.hout[0], p0, P);
      } else {
        k_im2col_t<<<blocks_for((size_t)L.ic / 8 * P), 256, 0, st>>>(bu.act[l - 1], bu.colt, B, pl.hin[l], pl.hu[l],
                                                                     pl.hout[l], L.ic, L.stride, L.up, p0, P);
      }
      CNN_CHECK("k_im2col_t");
      k_dz_t<<<dim3((P + 31) / 32, (L.oc + 31) / 32), dim3(32, 8), 0, st>>>(bu.dz[l], bu.dzt, grad + pl.boff[l], pixels,
                                                                          L.oc, p0, P);
      CNN_CHECK("k_dz_t");
      const int tiles = ((k9 + 127) / 128) * ((L.oc + 127) / 128);
      const int splits = 2 * 152 / tiles > 1 ? 2 * 152 / tiles : 1;
      int rc = gemm(PlainLoader<bf16>{bu.dzt, (size_t)P, L.oc}, PlainLoader<bf16>{bu.colt, (size_t)P, k9}, L.oc, k9,
                    P, WgradEpi{grad + pl.woff[l], L.oc, k9}, bu.status, st, splits);
      if (rc) return rc;
    }
    if (l == 0) break;
    const int rows = B * pl.hu[l] * pl.hu[l];
    DgradGather ga{bu.dz[l], B, pl.hu[l], pl.hout[l], L.oc, L.stride};
    PlainLoader<bf16> wt{bu.wt[l], (size_t)pl.ktp[l], L.ic};
    int rc;
    if (L.up == 1) {
      rc = gemm(ga, wt, rows, L.ic, pl.ktp[l], DgradEpi{bu.dz[l - 1], bu.act[l - 1], rows, L.ic}, bu.status, st);
    } else {
      rc = gemm(ga, wt, rows, L.ic, pl.ktp[l], StoreEpi{bu.du5, rows, L.ic}, bu.status, st);
      if (rc) return rc;
      k_upsample_grad<<<blocks_for((size_t)B * pl.hin[l] * pl.hin[l] * L.ic), 256, 0, st>>>(
          bu.du5, bu.act[l - 1], bu.dz[l - 1], B, pl.hin[l], L.ic, L.up);
      CNN_CHECK("k_upsample_grad");
    }
    if (rc) return rc;
  }
  return PTY_OK;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

static int check(int S, int B, const void* ws, size_t ws_bytes, Plan* pl) {
  if (!make_plan(S, B, pl)) {
    set_error("S = %d, B = %d not supported (S a multiple of 16 in [16, 512], 0 <= B <= 1024)", S, B);
    return PTY_EINVAL;
  }
  if (!ws || ((uintptr_t)ws & 255)) {
    set_error("workspace is NULL or not 256-byte aligned");
    return PTY_EINVAL;
  }
  if (ws_bytes < pl->total) {
    set_error("workspace has %zu bytes, %zu needed", ws_bytes, pl->total);
    return PTY_EWORKSPACE;
  }
  return PTY_OK;
}

__global__ void k_to_f32(const bf16* __restrict__ x, float* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __bfloat162float(x[i]);
}

}  // namespace cnn
}  // namespace pty

using namespace pty;
using namespace pty::cnn;

extern "C" {

size_t pty_cnn_param_count(void) { return param_count(); }

size_t pty_cnn_workspace_size(int S, int B) {
  Plan pl;
  if (!make_plan(S, B, &pl)) {
    set_error("S = %d, B = %d not supported (S a multiple of 16 in [16, 512], 0 <= B <= 1024)", S, B);
    return 0;
  }
  return pl.total;
}

int pty_cnn_forward(int S, int B, const float* params, const float* I, float s_in, float* pred, void* ws,
                    size_t ws_bytes, void* stream) {
  Plan pl;
  int rc = check(S, B, ws, ws_bytes, &pl);
  if (rc) return rc;
  if (!params || !aligned16(params) || (B > 0 && (!I || !pred || !aligned16(I) || !aligned16(pred)))) {
    set_error("params, I and pred must be non-NULL and 16-byte aligned");
    return PTY_EINVAL;
  }
  return run_forward(pl, carve(pl, ws), params, I, s_in, pred, (cudaStream_t)stream);
}

int pty_cnn_loss_grad(int S, int B, const float* params, const float* I, const float* Y, float s_in, double* loss,
                      float* grad, float* pred, void* ws, size_t ws_bytes, void* stream) {
  Plan pl;
  int rc = check(S, B, ws, ws_bytes, &pl);
  if (rc) return rc;
  if (!params || !grad || !loss || !aligned16(params) || !aligned16(grad) ||
      (B > 0 && (!I || !Y || !aligned16(I) || !aligned16(Y))) || (pred && !aligned16(pred))) {
    set_error("params, grad, loss, I and Y must be non-NULL and 16-byte aligned");
    return PTY_EINVAL;
  }
  const Buffers bu = carve(pl, ws);
  float* out = pred ? pred : bu.du5;  // du5 is free until layer 5's input gradient
  if ((size_t)B * pl.hout[5] * pl.hout[5] * kOut > (size_t)B * pl.hu[4] * pl.hu[4] * kNet[4].ic && !pred) {
    set_error("internal: prediction scratch too small");
    return PTY_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  rc = run_forward(pl, bu, params, I, s_in, out, st);
  if (rc) return rc;
  return run_backward(pl, bu, I, s_in, out, Y, loss, grad, st);
}

int pty_cnn_adam(float* params, float* m, float* v, const float* grad, int step, float lr, float beta1, float beta2,
                 float eps, void* stream) {
  if (!params || !m || !v || !grad || step < 1 || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f)) {
    set_error("bad Adam arguments");
    return PTY_EINVAL;
  }
  const double bc1 = 1.0 - pow((double)beta1, step), bc2 = 1.0 - pow((double)beta2, step);
  const size_t n = param_count();
  k_adam<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(params, m, v, grad, n, lr, beta1, beta2, eps, (float)bc1,
                                                          (float)sqrt(bc2));
  CNN_CHECK("k_adam");
  return PTY_OK;
}

int pty_cnn_train_step(int S, int B, float* params, float* m, float* v, float* grad, int step, float lr,
                       const float* I, const float* Y, float s_in, double* loss, void* ws, size_t ws_bytes,
                       void* stream) {
  int rc = pty_cnn_loss_grad(S, B, params, I, Y, s_in, loss, grad, nullptr, ws, ws_bytes, stream);
  if (rc) return rc;
  return pty_cnn_adam(params, m, v, grad, step, lr, 0.9f, 0.999f, 1e-8f, stream);
}

int pty_cnn_targets(int S, int Nz, int H, int W, const float* amp, const float* phase, const float* pos,
                    const int32_t* idx, int B, float* Y, void* stream) {
  if (S < 16 || S % 16 || Nz < 1 || H < S || W < S || B < 0 || (B > 0 && (!amp || !phase || !pos || !idx || !Y))) {
    set_error("bad target arguments");
    return PTY_EINVAL;
  }
  if (B == 0) return PTY_OK;
  k_targets<<<blocks_for((size_t)B * S * S / 4), 256, 0, (cudaStream_t)stream>>>(S, Nz, H, W, amp, phase, pos, idx, B,
                                                                                Y);
  CNN_CHECK("k_targets");
  return PTY_OK;
}

int pty_cnn_stitch(int S, int H, int W, const float* pred, const float* pos, const int32_t* idx, int B,
                   const float* weight, float* num, float* den, void* stream) {
  if (S < 16 || S % 16 || H < S || W < S || B < 0 || !weight || !num || !den || (B > 0 && (!pred || !pos || !idx))) {
    set_error("bad stitch arguments");
    return PTY_EINVAL;
  }
  if (B == 0) return PTY_OK;
  k_stitch<<<blocks_for((size_t)B * S * S / 4), 256, 0, (cudaStream_t)stream>>>(S, H, W, pred, pos, idx, B, weight,
                                                                               num, den);
  CNN_CHECK("k_stitch");
  return PTY_OK;
}

int pty_cnn_stitch_finish(int Nz, int H, int W, const float* num, const float* den, float* amp, float* phase,
                          void* stream) {
  if (Nz < 1 || H < 1 || W < 1 || !num || !den || !amp || !phase) {
    set_error("bad stitch arguments");
    return PTY_EINVAL;
  }
  k_stitch_finish<<<blocks_for((size_t)H * W), 256, 0, (cudaStream_t)stream>>>(Nz, H, W, num, den, amp, phase);
  CNN_CHECK("k_stitch_finish");
  return PTY_OK;
}

int pty_cnn_read_state(int S, int B, const void* ws, size_t ws_bytes, int layer, int what, float* out,
                       void* stream) {
  Plan pl;
  int rc = check(S, B, ws, ws_bytes, &pl);
  if (rc) return rc;
  if (layer < 1 || layer > kLayers || what < 0 || what > 1 || (what == 0 && layer == kLayers) || (B > 0 && !out)) {
    set_error("bad state request: layer %d, what %d", layer, what);
    return PTY_EINVAL;
  }
  const Buffers bu = carve(pl, const_cast<void*>(ws));
  const int l = layer - 1;
  const size_t n = (size_t)B * pl.hout[l] * pl.hout[l] * kNet[l].oc;
  if (n == 0) return PTY_OK;
  k_to_f32<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(what == 0 ? bu.act[l] : bu.dz[l], out, n);
  CNN_CHECK("k_to_f32");
  return PTY_OK;
}

}  // extern "C"
