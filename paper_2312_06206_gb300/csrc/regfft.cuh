// regfft.cuh -- register-resident two-level FFT of length L = TT * E (L <= 2048).
//
// A vector of length L is owned by TT threads; thread t holds E elements in
// registers.  Forward transform (natural input x[q] = v[t + TT q]):
//   1. E-point DFT over q in registers            -> A[t][k1]
//   2. twiddle A[t][k1] *= exp(-2 pi i t k1 / L)
//   3. transpose through shared memory (padded rows of TT + 1 elements)
//   4. TT-point DFT over t in registers           -> X[k1 + E k2]
// so one shared-memory round trip per transform.  After step 4 thread t holds
// X[k1 + E brev_TT(p)] in register j TT + p for k1 = t + TT j (j < E / TT):
// the "frequency layout".  Pointwise spectral multiplies act on that layout
// in registers with natural-order tables; the inverse transform runs the
// four steps backwards (unnormalised, it returns L * ifft).
//
// All DFT constants are compile-time: the radix-2 cascades are generated by
// static_for over template indices, and cos/sin of 2 pi j / n come from a
// constexpr Taylor evaluation after quadrant reduction.
#pragma once

#include <type_traits>
#include <utility>

#include "fft.cuh"

namespace sadi {
namespace rf {

constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 16; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 16; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
// cos and sin of 2 pi j / n (n a multiple of 4, or j = 0)
constexpr double cos2pi(int j, int n) {
  j = ((j % n) + n) % n;
  if (j == 0) return 1.0;
  const int q = (4 * j) / n;
  const double r = 2.0 * kPi * (double)(j - q * (n / 4)) / (double)n;
  return q == 0 ? taylor_cos(r) : q == 1 ? -taylor_sin(r) : q == 2 ? -taylor_cos(r) : taylor_sin(r);
}
constexpr double sin2pi(int j, int n) {
  j = ((j % n) + n) % n;
  if (j == 0) return 0.0;
  const int q = (4 * j) / n;
  const double r = 2.0 * kPi * (double)(j - q * (n / 4)) / (double)n;
  return q == 0 ? taylor_sin(r) : q == 1 ? taylor_cos(r) : q == 2 ? -taylor_sin(r) : -taylor_cos(r);
}

constexpr int clog2(int n) { return n <= 1 ? 0 : 1 + clog2(n >> 1); }
constexpr int cbrev(int p, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((p >> b) & 1) << (bits - 1 - b);
  return r;
}

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// x * exp(-2 pi i J / S) (FWD) or x * exp(+2 pi i J / S), J and S compile-time.
template <typename T, bool FWD, int J, int S>
__device__ __forceinline__ cx<T> rot(cx<T> x) {
  constexpr int j = ((J % S) + S) % S;
  if constexpr (j == 0) {
    return x;
  } else if constexpr (2 * j == S) {
    return mkc(-x.x, -x.y);
  } else if constexpr (4 * j == S) {
    return FWD ? cmul_mi(x) : cmul_pi(x);
  } else if constexpr (4 * j == 3 * S) {
    return FWD ? cmul_pi(x) : cmul_mi(x);
  } else {
    constexpr T c = (T)cos2pi(j, S);
    constexpr T s = (T)sin2pi(j, S);
    // forward: x * (c - i s); inverse: x * (c + i s)
    return FWD ? mkc(x.x * c + x.y * s, x.y * c - x.x * s) : mkc(x.x * c - x.y * s, x.y * c + x.x * s);
  }
}

// N-point DFT in registers.  fwd: natural in, x[p] = X[brev(p)] out.
template <typename T, int N>
__device__ __forceinline__ void dft_fwd(cx<T>* x) {
  constexpr int LG = clog2(N);
  static_for<0, LG>([&](auto lc) {
    constexpr int span = N >> decltype(lc)::value;
    constexpr int half = span >> 1;
    static_for<0, N / span>([&](auto gc) {
      constexpr int g = decltype(gc)::value * span;
      static_for<0, half>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        const cx<T> a = x[g + j], b = x[g + j + half];
        x[g + j] = cadd(a, b);
        x[g + j + half] = rot<T, true, j, span>(csub(a, b));
      });
    });
  });
}

// Inverse: x[p] = X[brev(p)] in, natural out (unnormalised).
template <typename T, int N>
__device__ __forceinline__ void dft_inv(cx<T>* x) {
  constexpr int LG = clog2(N);
  static_for<0, LG>([&](auto lc) {
    constexpr int span = 2 << decltype(lc)::value;
    constexpr int half = span >> 1;
    static_for<0, N / span>([&](auto gc) {
      constexpr int g = decltype(gc)::value * span;
      static_for<0, half>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        const cx<T> a = x[g + j];
        const cx<T> b = rot<T, false, j, span>(x[g + j + half]);
        x[g + j] = cadd(a, b);
        x[g + j + half] = csub(a, b);
      });
    });
  });
}

template <typename T, int LOGL>
struct RegFFT {
  static constexpr int L = 1 << LOGL;
  static constexpr int LOGT = LOGL / 2;
  static constexpr int LOGE = LOGL - LOGT;
  static constexpr int TT = 1 << LOGT;
  static constexpr int E = 1 << LOGE;
  static constexpr int KPT = E / TT;       // 1 or 2
  static constexpr int ROW = TT + 1;       // padded transpose row

  // natural index held in register q: t + TT q
  // frequency index held in register j TT + p: (t + TT j) + E brev_TT(p)
  template <int R>
  __device__ static __forceinline__ int freq_index(int t) {
    constexpr int j = R / TT, p = R % TT;
    return (t + TT * j) + E * cbrev(p, LOGT);
  }

  // Barrier between the transpose's writes and reads: the whole block, or
  // (WARP) only the warp, when every vector's TT threads lie in one warp and
  // no other warp touches its buffer.
  template <bool WARP>
  __device__ static __forceinline__ void sync() {
    if constexpr (WARP) __syncwarp();
    else __syncthreads();
  }

  // Forward transform; ends with the buffer free (after a barrier).
  // tw1 may point to global or shared memory.
  template <bool WARP = false>
  __device__ static __forceinline__ void fwd(cx<T>* x, cx<T>* sm, int t, const cx<T>* __restrict__ tw1) {
    dft_fwd<T, E>(x);
    static_for<0, E>([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      constexpr int k1 = cbrev(p, LOGE);
      sm[k1 * ROW + t] = cmul(x[p], tw1[k1 * TT + t]);
    });
    sync<WARP>();
    static_for<0, KPT>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      static_for<0, TT>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        x[j * TT + s] = sm[(t + TT * j) * ROW + s];
      });
    });
    sync<WARP>();
    static_for<0, KPT>([&](auto jc) { dft_fwd<T, TT>(x + decltype(jc)::value * TT); });
  }

  // Inverse of fwd (times L); ends with the buffer free.
  template <bool WARP = false>
  __device__ static __forceinline__ void inv(cx<T>* x, cx<T>* sm, int t, const cx<T>* __restrict__ tw1) {
    static_for<0, KPT>([&](auto jc) { dft_inv<T, TT>(x + decltype(jc)::value * TT); });
    static_for<0, KPT>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      static_for<0, TT>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        sm[(t + TT * j) * ROW + s] = x[j * TT + s];
      });
    });
    sync<WARP>();
    static_for<0, E>([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      constexpr int k1 = cbrev(p, LOGE);
      x[p] = cmulc(sm[k1 * ROW + t], tw1[k1 * TT + t]);
    });
    sync<WARP>();
    dft_inv<T, E>(x);
  }
};

}  // namespace rf
}  // namespace sadi
