// The shared-memory 2D FFT steps of fft_smem.cuh (N = 64, 128: one CTA) and fft_cluster.cuh
// (N = 256: four CTAs of a cluster, each holding 64 rows), compiled for the host and run one
// emulated thread at a time (every thread of every CTA finishes a step before any starts the next,
// as the barriers after each step guarantee on the GPU), against a direct double-precision DFT.
//
// Prints one line per case: N, threads, and the relative L2 errors of
//   fwd   the forward transform, read through the k-space digit layout (kbin0 / kbin1);
//   inv   the inverse of that spectrum back to N^2 times the input;
//   fused the fused steps (inverse end + forward start, forward end + inverse start) in a
//         forward-then-inverse and an inverse-then-forward chain.
#include <complex>
#include <cstdio>
#include <random>
#include <vector>

#include "fft_cluster.cuh"

using cd = std::complex<double>;

template <class F>
static void each_thread(int T, F&& f) {
  blockDim.x = T;
  for (int t = 0; t < T; ++t) {
    threadIdx.x = t;
    f();
  }
}

static double rel(const std::vector<cd>& a, const std::vector<cd>& b) {
  double n = 0, d = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    n += std::norm(a[i] - b[i]);
    d += std::norm(b[i]);
  }
  return std::sqrt(n / d);
}

template <int N, int T>
static void run(unsigned seed) {
  using F = pty::Fft2<N, T>;
  constexpr int RS = F::RS;
  std::vector<float2> s(N * RS), tw(N);
  each_thread(T, [&] { pty::build_twiddles<N>(tw.data()); });
  std::mt19937 g(seed);
  std::normal_distribution<float> nd;
  std::vector<cd> x(N * N);
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < N; ++c) {
      const float2 v = make_float2(nd(g), nd(g));
      s[r * RS + c] = v;
      x[r * N + c] = cd(v.x, v.y);
    }
  // direct DFT (separable, sign -1, unnormalised)
  std::vector<cd> tmp(N * N), X(N * N);
  for (int r = 0; r < N; ++r)
    for (int k = 0; k < N; ++k) {
      cd a = 0;
      for (int c = 0; c < N; ++c) a += x[r * N + c] * std::polar(1.0, -2.0 * M_PI * (double)(k * c % N) / N);
      tmp[r * N + k] = a;
    }
  for (int k1 = 0; k1 < N; ++k1)
    for (int k0 = 0; k0 < N; ++k0) {
      cd a = 0;
      for (int r = 0; r < N; ++r) a += tmp[r * N + k1] * std::polar(1.0, -2.0 * M_PI * (double)(k0 * r % N) / N);
      X[k0 * N + k1] = a;
    }
  pty::NoHook none;
  auto read = [&](bool kspace) {
    std::vector<cd> out(N * N);
    for (int p0 = 0; p0 < N; ++p0)
      for (int p1 = 0; p1 < N; ++p1) {
        const float2 v = s[p0 * RS + p1];
        const int i = kspace ? pty::kbin0<N>(p0) * N + pty::kbin1<N>(p1) : p0 * N + p1;
        out[i] = cd(v.x, v.y);
      }
    return out;
  };
  auto scaled = [&](const std::vector<cd>& v, double f) {
    std::vector<cd> o(v);
    for (auto& z : o) z *= f;
    return o;
  };
  // forward: col, block, row
  each_thread(T, [&] { F::col_fwd(s.data(), tw.data(), none); });
  each_thread(T, [&] { F::block_fwd(s.data(), tw.data()); });
  each_thread(T, [&] { F::template row_fwd<true>(s.data(), none); });
  const double e_fwd = rel(read(true), X);
  // inverse: row, block, col
  each_thread(T, [&] { F::row_inv(s.data(), tw.data(), none); });
  each_thread(T, [&] { F::block_inv(s.data(), tw.data()); });
  each_thread(T, [&] { F::col_inv(s.data(), tw.data()); });
  const double e_inv = rel(read(false), scaled(x, (double)N * N));
  // fused chains on the natural-layout array now holding N^2 x:
  // forward with its last step fused into the next inverse's first (row_fwd_inv), then the inverse
  each_thread(T, [&] { F::col_fwd(s.data(), tw.data(), none); });
  each_thread(T, [&] { F::block_fwd(s.data(), tw.data()); });
  each_thread(T, [&] { F::row_fwd_inv(s.data(), tw.data(), none); });
  each_thread(T, [&] { F::block_inv(s.data(), tw.data()); });
  each_thread(T, [&] { F::col_inv(s.data(), tw.data()); });
  const double e_f1 = rel(read(false), scaled(x, std::pow((double)N, 4)));
  // back to x: scale, then an inverse whose last step is fused into the next forward's first
  // (col_inv_fwd), then the forward's remaining steps: the spectrum of x again
  for (auto& v : s) v = make_float2(v.x / (float)std::pow((double)N, 4), v.y / (float)std::pow((double)N, 4));
  each_thread(T, [&] { F::col_fwd(s.data(), tw.data(), none); });
  each_thread(T, [&] { F::block_fwd(s.data(), tw.data()); });
  each_thread(T, [&] { F::template row_fwd<true>(s.data(), none); });
  each_thread(T, [&] { F::row_inv(s.data(), tw.data(), none); });
  each_thread(T, [&] { F::block_inv(s.data(), tw.data()); });
  each_thread(T, [&] { F::template col_inv_fwd<true>(s.data(), tw.data(), none); });
  each_thread(T, [&] { F::block_fwd(s.data(), tw.data()); });
  each_thread(T, [&] { F::template row_fwd<true>(s.data(), none); });
  const double e_f2 = rel(read(true), scaled(X, (double)N * N));
  std::printf("N %d T %d fwd %.3e inv %.3e fused %.3e\n", N, T, e_fwd, e_inv, std::max(e_f1, e_f2));
}

// N = 256 on C emulated CTAs (PTY_N256_CTAS: 4 of 512 threads or 8 of 128): CTA q holds rows
// [L q, L q + L) as float2 [L][257]; k-space row p0 = L q + local row.  The cluster FFT's
// sub-steps are each one barrier-delimited step.
static void run256(unsigned seed) {
  constexpr int N = 256, C = PTY_N256_CTAS, T = C == 8 ? 128 : 512, L = N / C;
  using F = pty::Fft2<N, T>;
  static_assert(F::C == C && F::L == L, "cluster shape");
  constexpr int RS = F::RS;
  std::vector<float2> cta[C];
  for (int q = 0; q < C; ++q) {
    cta[q].assign(L * RS, make_float2(0.f, 0.f));
    host_cta_base[q] = reinterpret_cast<char*>(cta[q].data());
  }
  std::vector<float2> tw(N);
  each_thread(T, [&] { pty::build_twiddles<N>(tw.data()); });
  std::mt19937 g(seed);
  std::normal_distribution<float> nd;
  std::vector<cd> x(N * N);
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < N; ++c) {
      const float2 v = make_float2(nd(g), nd(g));
      cta[r / L][(r % L) * RS + c] = v;
      x[r * N + c] = cd(v.x, v.y);
    }
  std::vector<cd> tmp(N * N), X(N * N);
  for (int r = 0; r < N; ++r)
    for (int k = 0; k < N; ++k) {
      cd a = 0;
      for (int c = 0; c < N; ++c) a += x[r * N + c] * std::polar(1.0, -2.0 * M_PI * (double)(k * c % N) / N);
      tmp[r * N + k] = a;
    }
  for (int k1 = 0; k1 < N; ++k1)
    for (int k0 = 0; k0 < N; ++k0) {
      cd a = 0;
      for (int r = 0; r < N; ++r) a += tmp[r * N + k1] * std::polar(1.0, -2.0 * M_PI * (double)(k0 * r % N) / N);
      X[k0 * N + k1] = a;
    }
  pty::NoHook none;
  // one barrier-delimited step on every thread of every CTA
  auto step = [&](auto&& f) {
    for (int q = 0; q < C; ++q) {
      host_cluster_rank = q;
      each_thread(T, [&] { f(cta[q].data()); });
    }
  };
  auto fwd = [&] {
    step([&](float2* s) { F::x1_step<false, true, true>(s, tw.data(), none); });
    step([&](float2* s) { F::x2_step<false>(s); });
    step([&](float2* s) { F::ra_fwd(s, tw.data()); });
    step([&](float2* s) { F::rb_step<true, false, true>(s, nullptr, none); });
  };
  auto inv = [&] {
    step([&](float2* s) { F::rb_step<false, true, true>(s, tw.data(), none); });
    step([&](float2* s) { F::ra_inv(s, tw.data()); });
    step([&](float2* s) { F::x2_step<true>(s); });
    step([&](float2* s) { F::x1_step<true, false, true>(s, tw.data(), none); });
  };
  auto read = [&](bool kspace) {
    std::vector<cd> out(N * N);
    for (int p0 = 0; p0 < N; ++p0)
      for (int p1 = 0; p1 < N; ++p1) {
        const float2 v = cta[p0 / L][(p0 % L) * RS + p1];
        const int i = kspace ? pty::kbin0<N>(p0) * N + pty::kbin1<N>(p1) : p0 * N + p1;
        out[i] = cd(v.x, v.y);
      }
    return out;
  };
  auto scaled = [&](const std::vector<cd>& v, double f) {
    std::vector<cd> o(v);
    for (auto& z : o) z *= f;
    return o;
  };
  fwd();
  const double e_fwd = rel(read(true), X);
  inv();
  const double e_inv = rel(read(false), scaled(x, (double)N * N));
  // fused: forward ending in RB -> RB^-1 (row_fwd_inv), then the rest of the inverse
  step([&](float2* s) { F::x1_step<false, true, true>(s, tw.data(), none); });
  step([&](float2* s) { F::x2_step<false>(s); });
  step([&](float2* s) { F::ra_fwd(s, tw.data()); });
  step([&](float2* s) { F::row_fwd_inv(s, tw.data(), none); });
  step([&](float2* s) { F::ra_inv(s, tw.data()); });
  step([&](float2* s) { F::x2_step<true>(s); });
  step([&](float2* s) { F::x1_step<true, false, true>(s, tw.data(), none); });
  const double e_f1 = rel(read(false), scaled(x, std::pow((double)N, 4)));
  for (auto& c : cta)
    for (auto& v : c) v = make_float2(v.x / (float)std::pow((double)N, 4), v.y / (float)std::pow((double)N, 4));
  // fused: inverse ending in X1^-1 -> X1 (col_inv_fwd), then the rest of the forward
  fwd();
  step([&](float2* s) { F::rb_step<false, true, true>(s, tw.data(), none); });
  step([&](float2* s) { F::ra_inv(s, tw.data()); });
  step([&](float2* s) { F::x2_step<true>(s); });
  step([&](float2* s) { F::col_inv_fwd<true>(s, tw.data(), none); });
  step([&](float2* s) { F::x2_step<false>(s); });
  step([&](float2* s) { F::ra_fwd(s, tw.data()); });
  step([&](float2* s) { F::rb_step<true, false, true>(s, nullptr, none); });
  const double e_f2 = rel(read(true), scaled(X, (double)N * N));
  std::printf("N %d T %d fwd %.3e inv %.3e fused %.3e\n", N, T, e_fwd, e_inv, std::max(e_f1, e_f2));
}

int main() {
  run<64, 128>(1);
  run<128, 256>(2);
  run<128, 512>(3);
  run256(4);
  return 0;
}
