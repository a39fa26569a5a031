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
// Stages (the "plan"): radix 8 (three radix-2 levels fused in registers),
// plus one radix-2 or radix-4 stage when log2 L is not a multiple of 3; in the
// DIF order the odd stage comes first (span L), then radix-8 stages down to
// span 8; DIT runs the same stages in reverse.  The radix-2 cascade inside a
// butterfly leaves register p holding DFT output brev_R(p), so storing
// register p to slot p makes the whole DIF produce the bit-reversal
// permutation.
//
// Fusion: the last DIF stage (span 8) and the first DIT stage (span 8) act on
// the same 8 consecutive elements, and so do the last DIT stage and the first
// DIF stage (span L); a pointwise multiply between a forward and an inverse
// transform (or between an inverse and a forward one) is therefore done in
// registers by one thread with no shared-memory round trip (fused8 / fusedL).
//
// Twiddles: per-stage tables, laid out [(q-1) * (S/R) + j] for register q of
// butterfly j of the stage with span S, so that the threads of a warp read
// consecutive addresses.  A separate table tw[k] = exp(-2 pi i k / P), P = 2L,
// provides the exp(-i pi k / L) twist of Algorithm 1 and the packing factors.
//
// Shared-memory layout (sidx, vstride): a half-warp of 16 threads reads 16
// elements per access, at stride 1 (spans >= 128 and all staging loops), in
// two blocks of 8 (span 64) or at stride 8 (span 8).
//   * FP32 (8-byte elements, 16 per 128-byte bank row): element i lives at
//     i ^ h(i >> 4) with h(x) = (x & 7) | ((x & 4) << 1), an XOR of its low
//     four bits: every aligned run of 16 stays a permutation of itself, the two
//     8-runs 64 apart land in different halves, and the stride-8 set spreads
//     over all 16 positions, so none of these accesses conflicts; no padding.
//   * FP64 (16-byte elements, accessed per quarter-warp of 8): element i lives
//     at i + (i >> 3), one pad slot per 8 elements.
// A buffer of nvec vectors uses nvec * vstride<T>(L) elements.
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

// multiply by a real or a complex factor
__device__ __forceinline__ float2 cmulany(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cmulany(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmulany(float2 a, float2 b) { return cmul(a, b); }
__device__ __forceinline__ double2 cmulany(double2 a, double2 b) { return cmul(a, b); }

__host__ __device__ __forceinline__ int padi(int i) { return i + (i >> 3); }
__host__ __device__ __forceinline__ int vec_stride(int L) { return L + (L >> 3) + 2; }

// Shared-memory position of element i (see the layout note above).
template <typename T> __host__ __device__ __forceinline__ int sidx(int i);
template <> __host__ __device__ __forceinline__ int sidx<double>(int i) { return padi(i); }
template <> __host__ __device__ __forceinline__ int sidx<float>(int i) {
  const int x = i >> 4;
  return i ^ ((x & 7) | ((x & 4) << 1));
}
// Elements per vector buffer.
template <typename T> __host__ __device__ __forceinline__ int vstride(int L);
template <> __host__ __device__ __forceinline__ int vstride<double>(int L) { return vec_stride(L); }
template <> __host__ __device__ __forceinline__ int vstride<float>(int L) { return L + 2; }

__device__ __forceinline__ int brev(int p, int logL) {
  return (int)(__brev((unsigned)p) >> (32 - logL));
}

// Stage plan of a length-2^logL transform in DIF order.
struct FftPlan {
  int n;          // number of stages
  int logS[8];    // log2 span
  int logR[8];    // log2 radix (1, 2 or 3)
  int off[8];     // offset of the stage's twiddle sub-table
  int total;      // twiddle entries
};

__host__ __device__ inline FftPlan fft_plan(int logL) {
  FftPlan p;
  p.n = 0;
  int logS = logL, off = 0;
  const int rem = logL % 3;
  if (rem) {
    p.logS[0] = logL;
    p.logR[0] = rem;
    p.off[0] = 0;
    off += ((1 << rem) - 1) << (logL - rem);
    p.n = 1;
    logS -= rem;
  }
  while (logS >= 3) {
    p.logS[p.n] = logS;
    p.logR[p.n] = 3;
    p.off[p.n] = off;
    off += 7 << (logS - 3);
    p.n++;
    logS -= 3;
  }
  p.total = off;
  return p;
}

// Stage s of the plan, computed arithmetically (no local arrays):
// the odd stage (if any) first, then radix-8 stages k = 0, 1, ... with span
// 2^(logL - rem - 3k) and twiddle offset base + 2^(logL-rem) - 2^(logL-rem-3k).
struct Stage {
  int logS, logR, off;
};
__host__ __device__ __forceinline__ int plan_stages(int logL) {
  const int rem = logL % 3;
  return (rem ? 1 : 0) + (logL - rem) / 3;
}
__host__ __device__ __forceinline__ Stage plan_stage(int logL, int s) {
  const int rem = logL % 3;
  Stage st;
  if (rem && s == 0) {
    st.logS = logL;
    st.logR = rem;
    st.off = 0;
    return st;
  }
  const int k = s - (rem ? 1 : 0);
  const int base = rem ? (((1 << rem) - 1) << (logL - rem)) : 0;
  st.logS = logL - rem - 3 * k;
  st.logR = 3;
  st.off = base + (1 << (logL - rem)) - (1 << (logL - rem - 3 * k));
  return st;
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

template <typename T, int R, bool FWD>
__device__ __forceinline__ void bfly(cx<T>* x) {
  if (R == 2) bfly2<T>(x);
  else if (R == 4) bfly4<T, FWD>(x);
  else bfly8<T, FWD>(x);
}

// ---------------------------------------------------------------------------
// One radix-R stage over nvec vectors of length L (span S, stride m = S/R).
// stw: this stage's twiddle sub-table.
// ---------------------------------------------------------------------------
template <typename T, int R, bool FWD>
__device__ __forceinline__ void fft_stage(cx<T>* __restrict__ buf, int logL, int logS, int nvec, int vstride,
                                          const cx<T>* __restrict__ stw) {
  constexpr int logR = (R == 2) ? 1 : (R == 4) ? 2 : 3;
  const int logm = logS - logR;
  const int m = 1 << logm;
  const int lognb = logL - logR;           // butterflies per vector = L / R
  const int total = nvec << lognb;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int v = t >> lognb;
    const int u = t & ((1 << lognb) - 1);
    const int j = u & (m - 1);
    const int base = ((u - j) << logR) + j;
    cx<T>* p = buf + v * vstride;
    cx<T> x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = p[sidx<T>(base + (q << logm))];
    if (!FWD && j != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) x[q] = cmulc(x[q], __ldg(&stw[((q - 1) << logm) + j]));
    }
    bfly<T, R, FWD>(x);
    if (FWD && j != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) x[q] = cmul(x[q], __ldg(&stw[((q - 1) << logm) + j]));
    }
#pragma unroll
    for (int q = 0; q < R; ++q) p[sidx<T>(base + (q << logm))] = x[q];
  }
}

template <typename T, bool FWD>
__device__ __forceinline__ void run_stage(int logL, int s, cx<T>* buf, int nvec, int vs, const cx<T>* stw) {
  const Stage st = plan_stage(logL, s);
  if (st.logR == 3) fft_stage<T, 8, FWD>(buf, logL, st.logS, nvec, vs, stw + st.off);
  else if (st.logR == 2) fft_stage<T, 4, FWD>(buf, logL, st.logS, nvec, vs, stw + st.off);
  else fft_stage<T, 2, FWD>(buf, logL, st.logS, nvec, vs, stw + st.off);
  __syncthreads();
}

// Forward DIF FFT stages [s0, s1) of the plan; every stage ends with a
// __syncthreads().  Must be called by every thread of the block.
template <typename T>
__device__ void dif_stages(cx<T>* buf, int logL, int nvec, int vs, const cx<T>* stw, int s0, int s1) {
  for (int s = s0; s < s1; ++s) run_stage<T, true>(logL, s, buf, nvec, vs, stw);
}
// Inverse DIT FFT stages, DIF-order indices s1-1 down to s0.
template <typename T>
__device__ void dit_stages(cx<T>* buf, int logL, int nvec, int vs, const cx<T>* stw, int s0, int s1) {
  for (int s = s1 - 1; s >= s0; --s) run_stage<T, false>(logL, s, buf, nvec, vs, stw);
}

template <typename T>
__device__ void fft_dif(cx<T>* buf, int logL, int nvec, int vs, const cx<T>* stw) {
  dif_stages<T>(buf, logL, nvec, vs, stw, 0, plan_stages(logL));
}
template <typename T>
__device__ void fft_dit(cx<T>* buf, int logL, int nvec, int vs, const cx<T>* stw) {
  dit_stages<T>(buf, logL, nvec, vs, stw, 0, plan_stages(logL));
}

// ---------------------------------------------------------------------------
// fused8: last DIF stage (span 8) -> multiply by mult[v * mstride + p] ->
// first DIT stage (span 8), in registers (span-8 stages have no twiddles).
// Requires a plan with >= 2 stages (L >= 16).  Ends with __syncthreads().
// ---------------------------------------------------------------------------
template <typename T, typename M>
__device__ void fused8(cx<T>* __restrict__ buf, int logL, int nvec, int vs, const M* __restrict__ mult,
                       int mstride) {
  const int lognb = logL - 3;
  const int total = nvec << lognb;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int v = t >> lognb;
    const int base = (t & ((1 << lognb) - 1)) << 3;
    cx<T>* p = buf + v * vs;
    const M* mm = mult + (size_t)v * mstride + base;
    cx<T> x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = p[sidx<T>(base + q)];
    bfly8<T, true>(x);
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = cmulany(x[q], __ldg(&mm[q]));
    bfly8<T, false>(x);
#pragma unroll
    for (int q = 0; q < 8; ++q) p[sidx<T>(base + q)] = x[q];
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// fusedL: last DIT stage (span L) -> multiply natural position k by
// conj(tw[k]) -> first DIF stage (span L), in registers.  Requires >= 2 stages.
// Ends with __syncthreads().
// ---------------------------------------------------------------------------
template <typename T, int R>
__device__ void fusedL_impl(cx<T>* __restrict__ buf, int logL, int nvec, int vs, const cx<T>* __restrict__ stw,
                            const cx<T>* __restrict__ tw) {
  constexpr int logR = (R == 2) ? 1 : (R == 4) ? 2 : 3;
  const int logm = logL - logR;
  const int m = 1 << logm;
  const int total = nvec << logm;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int v = t >> logm;
    const int j = t & (m - 1);
    cx<T>* p = buf + v * vs;
    cx<T> x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = p[sidx<T>(j + (q << logm))];
    cx<T> w[R];
    w[0] = mkc(T(1), T(0));
#pragma unroll
    for (int q = 1; q < R; ++q) w[q] = __ldg(&stw[((q - 1) << logm) + j]);
    if (j != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) x[q] = cmulc(x[q], w[q]);
    }
    bfly<T, R, false>(x);
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = cmulc(x[q], __ldg(&tw[j + (q << logm)]));
    bfly<T, R, true>(x);
    if (j != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) x[q] = cmul(x[q], w[q]);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) p[sidx<T>(j + (q << logm))] = x[q];
  }
  __syncthreads();
}

template <typename T>
__device__ void fusedL(cx<T>* buf, int logL, int nvec, int vs, const cx<T>* stw, const cx<T>* tw) {
  const int lr = plan_stage(logL, 0).logR;
  if (lr == 3) fusedL_impl<T, 8>(buf, logL, nvec, vs, stw, tw);
  else if (lr == 2) fusedL_impl<T, 4>(buf, logL, nvec, vs, stw, tw);
  else fusedL_impl<T, 2>(buf, logL, nvec, vs, stw, tw);
}

}  // namespace sadi
