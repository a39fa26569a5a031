// fft.cuh -- shared-memory FFT building blocks for the S-ADI kernels.
//
// Every transform in the library is a complex FFT of one power-of-two length
// L (the "FFT length" N' of a context) held in shared memory:
//   * forward = in-place decimation-in-frequency (DIF): natural-order input,
//     bit-reversed output (position p holds frequency brev(p));
//   * inverse = in-place decimation-in-time (DIT): bit-reversed input,
//     natural-order output, unnormalised (it returns L * ifft).
// Because every pointwise spectral operation of the method (the symbol of the
// block-circulant embedding of L_h, Sec. 3; the circulant/skew-circulant
// spectra lambda_c, lambda_s of Algorithm 1) is stored in the same bit-reversed
// order, no reordering pass is ever needed.
//
// Stages: radix 8 (three radix-2 levels fused in registers), plus one radix-2
// or radix-4 stage for log2 L not divisible by 3 (outermost span in DIF,
// innermost-last in DIT).  The radix-2 cascade inside a butterfly leaves
// register p holding the DFT output brev_R(p), so storing register p to slot p
// makes the whole DIF produce exactly the bit-reversal permutation.
//
// Shared-memory layout: element i of a vector lives at i + (i >> 3) (one pad
// slot per 8 elements), which spreads the stride-8 accesses of the last DIF /
// first DIT stage over all banks.  A buffer of nvec vectors uses
// nvec * vec_stride(L) elements.
//
// Twiddles come from one table tw[k] = exp(-2 pi i k / P), 0 <= k < P, with
// P = 2L (the same table provides the exp(-i pi k / L) twist of Algorithm 1
// and the exp(-2 pi i k / 2L) factors of the real/complex packing).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sadi {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { typedef float2 type; };
template <> struct cplx_of<double> { typedef double2 type; };
template <typename T> using cx = typename cplx_of<T>::type;

__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mkc(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mkc(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  return mkc(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return mkc(a.x, -a.y); }
template <typename V, typename T> __device__ __forceinline__ V cscale(V a, T s) { return mkc(a.x * s, a.y * s); }
// multiply by -i
template <typename V> __device__ __forceinline__ V cmul_mi(V a) { return mkc(a.y, -a.x); }
// multiply by +i
template <typename V> __device__ __forceinline__ V cmul_pi(V a) { return mkc(-a.y, a.x); }

__host__ __device__ __forceinline__ int padi(int i) { return i + (i >> 3); }
__host__ __device__ __forceinline__ int vec_stride(int L) { return L + (L >> 3) + 2; }

__device__ __forceinline__ int brev(int p, int logL) {
  return (int)(__brev((unsigned)p) >> (32 - logL));
}

template <typename T> __device__ __forceinline__ T rsqrt2();
template <> __device__ __forceinline__ float rsqrt2<float>() { return 0.70710678118654752440f; }
template <> __device__ __forceinline__ double rsqrt2<double>() { return 0.70710678118654752440; }

// x * exp(-i pi / 4) (forward) or x * exp(+i pi / 4) (inverse)
template <typename T, bool FWD>
__device__ __forceinline__ cx<T> mul_w8(cx<T> a) {
  const T c = rsqrt2<T>();
  return FWD ? mkc((a.x + a.y) * c, (a.y - a.x) * c) : mkc((a.x - a.y) * c, (a.x + a.y) * c);
}
// x * exp(-3 i pi / 4) (forward) or x * exp(+3 i pi / 4) (inverse)
template <typename T, bool FWD>
__device__ __forceinline__ cx<T> mul_w8_3(cx<T> a) {
  const T c = rsqrt2<T>();
  return FWD ? mkc((a.y - a.x) * c, -(a.x + a.y) * c) : mkc(-(a.x + a.y) * c, (a.x - a.y) * c);
}

// ---------------------------------------------------------------------------
// Register butterflies.  Forward: natural-order inputs x[q]; on return x[p]
// holds DFT_R output brev_R(p).  Inverse: x[p] holds input frequency
// brev_R(p); on return x[q] holds the (unnormalised) inverse DFT sample q.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void bfly2(cx<T>* x) {
  cx<T> a = x[0], b = x[1];
  x[0] = cadd(a, b);
  x[1] = csub(a, b);
}

template <typename T, bool FWD>
__device__ __forceinline__ void bfly4(cx<T>* x) {
  if (FWD) {
    cx<T> a0 = cadd(x[0], x[2]), a1 = cadd(x[1], x[3]);
    cx<T> b0 = csub(x[0], x[2]), b1 = cmul_mi(csub(x[1], x[3]));
    x[0] = cadd(a0, a1); x[1] = csub(a0, a1);
    x[2] = cadd(b0, b1); x[3] = csub(b0, b1);
  } else {
    cx<T> a0 = cadd(x[0], x[1]), a1 = csub(x[0], x[1]);
    cx<T> b0 = cadd(x[2], x[3]), b1 = cmul_pi(csub(x[2], x[3]));
    x[0] = cadd(a0, b0); x[2] = csub(a0, b0);
    x[1] = cadd(a1, b1); x[3] = csub(a1, b1);
  }
}

template <typename T, bool FWD>
__device__ __forceinline__ void bfly8(cx<T>* x) {
  if (FWD) {
    // level 1: span 8
    cx<T> t0 = cadd(x[0], x[4]), t4 = csub(x[0], x[4]);
    cx<T> t1 = cadd(x[1], x[5]), t5 = mul_w8<T, true>(csub(x[1], x[5]));
    cx<T> t2 = cadd(x[2], x[6]), t6 = cmul_mi(csub(x[2], x[6]));
    cx<T> t3 = cadd(x[3], x[7]), t7 = mul_w8_3<T, true>(csub(x[3], x[7]));
    // level 2: span 4 on (t0..t3) and (t4..t7)
    cx<T> u0 = cadd(t0, t2), u2 = csub(t0, t2);
    cx<T> u1 = cadd(t1, t3), u3 = cmul_mi(csub(t1, t3));
    cx<T> u4 = cadd(t4, t6), u6 = csub(t4, t6);
    cx<T> u5 = cadd(t5, t7), u7 = cmul_mi(csub(t5, t7));
    // level 3: span 2
    x[0] = cadd(u0, u1); x[1] = csub(u0, u1);
    x[2] = cadd(u2, u3); x[3] = csub(u2, u3);
    x[4] = cadd(u4, u5); x[5] = csub(u4, u5);
    x[6] = cadd(u6, u7); x[7] = csub(u6, u7);
  } else {
    // level 3 inverse
    cx<T> u0 = cadd(x[0], x[1]), u1 = csub(x[0], x[1]);
    cx<T> u2 = cadd(x[2], x[3]), u3 = cmul_pi(csub(x[2], x[3]));
    cx<T> u4 = cadd(x[4], x[5]), u5 = csub(x[4], x[5]);
    cx<T> u6 = cadd(x[6], x[7]), u7 = cmul_pi(csub(x[6], x[7]));
    // level 2 inverse
    cx<T> t0 = cadd(u0, u2), t2 = csub(u0, u2);
    cx<T> t1 = cadd(u1, u3), t3 = csub(u1, u3);
    cx<T> t4 = cadd(u4, u6), t6 = csub(u4, u6);
    cx<T> t5 = cadd(u5, u7), t7 = csub(u5, u7);
    // level 1 inverse: x[q] = t_q + w^-q t_{q+4}
    t5 = mul_w8<T, false>(t5);
    t6 = cmul_pi(t6);
    t7 = mul_w8_3<T, false>(t7);
    x[0] = cadd(t0, t4); x[4] = csub(t0, t4);
    x[1] = cadd(t1, t5); x[5] = csub(t1, t5);
    x[2] = cadd(t2, t6); x[6] = csub(t2, t6);
    x[3] = cadd(t3, t7); x[7] = csub(t3, t7);
  }
}

__device__ __forceinline__ int brev_small(int p, int logR) {
  // bit reversal of p in logR bits (logR <= 3)
  return logR == 1 ? p : logR == 2 ? (((p & 1) << 1) | (p >> 1))
                                   : (((p & 1) << 2) | (p & 2) | (p >> 2));
}

template <typename T, int R>
__device__ __forceinline__ void bfly(cx<T>* x, bool fwd) {
  if (R == 2) bfly2<T>(x);
  else if (R == 4) { if (fwd) bfly4<T, true>(x); else bfly4<T, false>(x); }
  else { if (fwd) bfly8<T, true>(x); else bfly8<T, false>(x); }
}

// One radix-R stage over nvec vectors of length L (span S, stride m = S/R).
// tw: table of exp(-2 pi i k / P); twshift = log2(P / S).
template <typename T, int R, bool FWD>
__device__ __forceinline__ void fft_stage(cx<T>* __restrict__ buf, int logL, int logS, int nvec, int vstride,
                                          const cx<T>* __restrict__ tw, int logP) {
  constexpr int logR = (R == 2) ? 1 : (R == 4) ? 2 : 3;
  const int logm = logS - logR;
  const int m = 1 << logm;
  const int lognb = logL - logR;           // butterflies per vector = L / R
  const int total = nvec << lognb;
  const int twshift = logP - logS;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int v = t >> lognb;
    const int u = t & ((1 << lognb) - 1);
    const int j = u & (m - 1);
    const int base = ((u - j) << logR) + j;
    cx<T>* p = buf + v * vstride;
    cx<T> x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = p[padi(base + (q << logm))];
    if (!FWD && j != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) x[q] = cmulc(x[q], __ldg(&tw[(j * brev_small(q, logR)) << twshift]));
    }
    if (FWD) bfly<T, R>(x, true); else bfly<T, R>(x, false);
    if (FWD && j != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) x[q] = cmul(x[q], __ldg(&tw[(j * brev_small(q, logR)) << twshift]));
    }
#pragma unroll
    for (int q = 0; q < R; ++q) p[padi(base + (q << logm))] = x[q];
  }
}

// Forward DIF FFT (natural -> bit-reversed) of nvec vectors; ends with a
// __syncthreads().  Must be called by every thread of the block, with the
// input already visible (caller synchronised).
template <typename T>
__device__ void fft_dif(cx<T>* buf, int logL, int nvec, int vstride, const cx<T>* tw, int logP) {
  int logS = logL;
  const int rem = logL % 3;
  if (rem == 1) { fft_stage<T, 2, true>(buf, logL, logS, nvec, vstride, tw, logP); logS -= 1; __syncthreads(); }
  else if (rem == 2) { fft_stage<T, 4, true>(buf, logL, logS, nvec, vstride, tw, logP); logS -= 2; __syncthreads(); }
  while (logS >= 3) {
    fft_stage<T, 8, true>(buf, logL, logS, nvec, vstride, tw, logP);
    logS -= 3;
    __syncthreads();
  }
}

// Inverse DIT FFT (bit-reversed -> natural), unnormalised; ends with a
// __syncthreads().
template <typename T>
__device__ void fft_dit(cx<T>* buf, int logL, int nvec, int vstride, const cx<T>* tw, int logP) {
  const int rem = logL % 3;
  int logS = 3;
  while (logS <= logL - rem) {
    fft_stage<T, 8, false>(buf, logL, logS, nvec, vstride, tw, logP);
    logS += 3;
    __syncthreads();
  }
  if (rem == 1) { fft_stage<T, 2, false>(buf, logL, logL, nvec, vstride, tw, logP); __syncthreads(); }
  else if (rem == 2) { fft_stage<T, 4, false>(buf, logL, logL, nvec, vstride, tw, logP); __syncthreads(); }
}

}  // namespace sadi
