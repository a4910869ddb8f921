// Host stand-ins for the few CUDA names the shared-memory FFT header uses, so that the header can
// be compiled with a host C++ compiler and its steps run one "thread" at a time (test use only).
#pragma once
#include <cmath>

struct float2 {
  float x, y;
};
inline float2 make_float2(float x, float y) { return float2{x, y}; }
#define __device__
#define __host__
#define __forceinline__ inline
struct HostThreadIdx {
  int x = 0, y = 0, z = 0;
};
inline HostThreadIdx threadIdx;  // set by the caller before each emulated thread's call
inline HostThreadIdx blockDim;   // the emulated CTA's thread count, set by the caller
inline void __syncthreads() {}
inline void sincospif(float x, float* s, float* c) {
  const double a = 3.14159265358979323846 * (double)x;
  *s = (float)std::sin(a);
  *c = (float)std::cos(a);
}
