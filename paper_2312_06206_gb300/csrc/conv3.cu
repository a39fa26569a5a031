// conv3.cu -- the column convolution of the FP32 forms for FFT lengths
// N' = 2048 .. 8192 as three passes of a four-step FFT.
//
// The step applies L_h through the block-circulant embedding (Sec. 3): after
// the row transforms, every spectrum column (one x frequency) is transformed
// along y with length P = 2N' (N nonzero rows), multiplied by the symbol and
// transformed back.  As on the other paths the length-P transform is split
// into its even and odd frequency halves, two length-N' transforms of the
// column and of the column times w^j, w = exp(-i pi / N').
//
// Here N' = R1 x 64, row j = j1 + R1 j2, frequency m = m2 + 64 m1:
//   pass A (block: one j1, 16 columns): 64-point DFTs over j2 (rows R1
//           apart), times exp(-2 pi i j1 m2 / N'), stored at row j1 + R1 m2;
//   pass B (block: one m2, 16 columns): R1-point DFT over j1 (R1 adjacent
//           rows), times the symbol at y frequency 2m + h, inverse R1-point
//           DFT, times exp(+2 pi i j1 m2 / N');
//   pass C (block: one j1, 16 columns): inverse 64-point DFT over m2, then
//           even half + conj(w^j) odd half -> rows j < N of the spectrum.
// Every global access of a block covers 16 adjacent columns of a row (128
// bytes), where the single-pass shared-memory kernel gathers one 8-byte
// element per row; the two halves' intermediates (N' x (N' + 16) complex
// each) live in HBM between the passes.  The small transforms are the
// register FFT of regfft.cuh, one vector per TT threads of a warp.
//
// Columns: 0 = the real part of slot 0 (x frequency 0), N' = its imaginary
// part (x frequency N'), 1 .. N'-1 the other slots (bit-reversed x
// frequencies, as the shared-memory engine stores them); N' + 1 .. N' + 15
// pad the last group.  The symbol is the shared-memory engine's table,
// re-laid once so that a pass-B block reads it contiguously.
#include <cuda_runtime.h>

#include "regfft.cuh"
#include "sadi_internal.h"

namespace sadi {
namespace {

using rf::static_for;

constexpr int kGroup = 16;           // columns per block
constexpr int kR2 = 64;              // length of the strided transforms (passes A, C)
constexpr int kTP = kGroup + 1;      // padded tile row (float2)
constexpr int kThreadsAC = 32 * 8;   // 32 vectors x 8 threads (RegFFT<6>: TT = 8)

template <int LOGL>
constexpr int vec_elems() {
  return rf::RegFFT<float, LOGL>::E * rf::RegFFT<float, LOGL>::ROW;
}

__device__ __forceinline__ float2 column_input(const float2* __restrict__ S, int Np, int N, int j, int gc) {
  if (j >= N || gc > Np) return make_float2(0.f, 0.f);
  if (gc == 0) return make_float2(S[(size_t)j * Np].x, 0.f);
  if (gc == Np) return make_float2(S[(size_t)j * Np].y, 0.f);
  return S[(size_t)j * Np + gc];
}

// shared memory of passes A and C: tiles (input / two halves), 32 transform
// buffers and the 64-point twiddles
constexpr size_t kSmemAC = (size_t)(3 * kR2 * kTP + 32 * vec_elems<6>() + 64) * sizeof(float2);
template <int LOGR1>
constexpr size_t smem_b() {
  return (size_t)(2 * (1 << LOGR1) * kTP + 32 * vec_elems<LOGR1>() + (1 << LOGR1)) * sizeof(float2);
}

__global__ void __launch_bounds__(kThreadsAC) k_conv3_a(const float2* __restrict__ S, const float2* __restrict__ tw,
                                                        Conv3 c, int N, int Np) {
  using F = rf::RegFFT<float, 6>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s_in = reinterpret_cast<float2*>(smem_raw);
  float2* s_out = s_in + kR2 * kTP;                 // [2][kR2 * kTP]
  float2* s_fft = s_out + 2 * kR2 * kTP;
  float2* s_tw1 = s_fft + 32 * vec_elems<6>();
  const int grp = blockIdx.x, j1 = blockIdx.y, R1 = c.R1, tid = threadIdx.x;
  if (tid < 64) s_tw1[tid] = c.tw1a[tid];
  for (int e = tid; e < kR2 * kGroup; e += kThreadsAC) {
    const int r = e / kGroup, cc = e % kGroup;
    s_in[r * kTP + cc] = column_input(S, Np, N, j1 + R1 * r, kGroup * grp + cc);
  }
  __syncthreads();
  const int v = tid / F::TT, t = tid % F::TT, cl = v >> 1, h = v & 1;
  float2 x[F::E];
  static_for<0, F::E>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const int j2 = t + F::TT * q;
    const float2 val = s_in[j2 * kTP + cl];
    x[q] = h ? cmul(val, __ldg(&tw[j1 + R1 * j2])) : val;
  });
  F::template fwd<true>(x, s_fft + v * vec_elems<6>(), t, s_tw1);
  static_for<0, F::E>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    const int m2 = F::template freq_index<r>(t);
    s_out[h * kR2 * kTP + m2 * kTP + cl] = cmul(x[r], __ldg(&c.twM[j1 * m2]));
  });
  __syncthreads();
  for (int e = tid; e < 2 * kR2 * kGroup; e += kThreadsAC) {
    const int hh = e / (kR2 * kGroup), r = (e / kGroup) % kR2, cc = e % kGroup;
    float2* Z = hh ? c.ZO : c.ZE;
    Z[(size_t)(j1 + R1 * r) * c.CW + kGroup * grp + cc] = s_out[hh * kR2 * kTP + r * kTP + cc];
  }
}

template <int LOGR1>
__global__ void __launch_bounds__(32 * rf::RegFFT<float, LOGR1>::TT) k_conv3_b(Conv3 c) {
  using F = rf::RegFFT<float, LOGR1>;
  constexpr int R1 = 1 << LOGR1;
  constexpr int NT = 32 * F::TT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s_t = reinterpret_cast<float2*>(smem_raw);   // [2][R1 * kTP]
  float2* s_fft = s_t + 2 * R1 * kTP;
  float2* s_tw1 = s_fft + 32 * vec_elems<LOGR1>();
  const int grp = blockIdx.x, m2 = blockIdx.y, tid = threadIdx.x;
  for (int e = tid; e < R1; e += NT) s_tw1[e] = c.tw1b[e];
  for (int e = tid; e < 2 * R1 * kGroup; e += NT) {
    const int hh = e / (R1 * kGroup), r = (e / kGroup) % R1, cc = e % kGroup;
    const float2* Z = hh ? c.ZO : c.ZE;
    s_t[hh * R1 * kTP + r * kTP + cc] = Z[(size_t)(r + R1 * m2) * c.CW + kGroup * grp + cc];
  }
  __syncthreads();
  const int v = tid / F::TT, t = tid % F::TT, cl = v >> 1, h = v & 1;
  float2* tile = s_t + h * R1 * kTP;
  float2 x[F::E];
  // each element of the vector's column is read and later written by the same
  // thread (natural layout before the forward and after the inverse transform)
  static_for<0, F::E>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    x[q] = tile[(t + F::TT * q) * kTP + cl];
  });
  F::template fwd<true>(x, s_fft + v * vec_elems<LOGR1>(), t, s_tw1);
  const float* lam = c.Lt + ((size_t)(m2 * c.CW + kGroup * grp + cl) * 2 + h) * R1;
  static_for<0, F::E>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    x[r] = cscale(x[r], __ldg(lam + F::template freq_index<r>(t)));
  });
  F::template inv<true>(x, s_fft + v * vec_elems<LOGR1>(), t, s_tw1);
  static_for<0, F::E>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const int j1 = t + F::TT * q;
    tile[j1 * kTP + cl] = cmulc(x[q], __ldg(&c.twM[j1 * m2]));
  });
  __syncthreads();
  for (int e = tid; e < 2 * R1 * kGroup; e += NT) {
    const int hh = e / (R1 * kGroup), r = (e / kGroup) % R1, cc = e % kGroup;
    float2* Z = hh ? c.ZO : c.ZE;
    Z[(size_t)(r + R1 * m2) * c.CW + kGroup * grp + cc] = s_t[hh * R1 * kTP + r * kTP + cc];
  }
}

__global__ void __launch_bounds__(kThreadsAC) k_conv3_c(float2* __restrict__ S, const float2* __restrict__ tw,
                                                        Conv3 c, int N, int Np) {
  using F = rf::RegFFT<float, 6>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s_t = reinterpret_cast<float2*>(smem_raw);   // [2][kR2 * kTP]
  float2* s_fft = s_t + 3 * kR2 * kTP;
  float2* s_tw1 = s_fft + 32 * vec_elems<6>();
  const int grp = blockIdx.x, j1 = blockIdx.y, R1 = c.R1, tid = threadIdx.x;
  if (tid < 64) s_tw1[tid] = c.tw1a[tid];
  for (int e = tid; e < 2 * kR2 * kGroup; e += kThreadsAC) {
    const int hh = e / (kR2 * kGroup), r = (e / kGroup) % kR2, cc = e % kGroup;
    const float2* Z = hh ? c.ZO : c.ZE;
    s_t[hh * kR2 * kTP + r * kTP + cc] = Z[(size_t)(j1 + R1 * r) * c.CW + kGroup * grp + cc];
  }
  __syncthreads();
  const int v = tid / F::TT, t = tid % F::TT, cl = v >> 1, h = v & 1;
  float2* tile = s_t + h * kR2 * kTP;
  float2 x[F::E];
  static_for<0, F::E>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    x[r] = tile[F::template freq_index<r>(t) * kTP + cl];
  });
  // the transform's internal warp barriers order every read of the vector's
  // column before the writes below
  F::template inv<true>(x, s_fft + v * vec_elems<6>(), t, s_tw1);
  static_for<0, F::E>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    tile[(t + F::TT * q) * kTP + cl] = x[q];
  });
  __syncthreads();
  for (int e = tid; e < kR2 * kGroup; e += kThreadsAC) {
    const int r = e / kGroup, cc = e % kGroup;
    const int j = j1 + R1 * r, gc = kGroup * grp + cc;
    if (j >= N || gc > Np) continue;
    const float2 y = cadd(s_t[r * kTP + cc], cmulc(s_t[kR2 * kTP + r * kTP + cc], __ldg(&tw[j])));
    if (gc == 0) reinterpret_cast<float*>(S + (size_t)j * Np)[0] = y.x;
    else if (gc == Np) reinterpret_cast<float*>(S + (size_t)j * Np)[1] = y.x;
    else S[(size_t)j * Np + gc] = y;
  }
}

// Tables: the symbol re-laid as Lt[((m2 * CW + col) * 2 + h) * R1 + m1] =
// lpb[(col * 2 + h) * N' + brev(m2 + 64 m1)] (zero for pad columns), and the
// twiddles exp(-2 pi i k / N') and those of the two register transforms
// (tw1[k1 TT + t] = exp(-2 pi i t k1 / L)), evaluated in FP64.
__global__ void k_conv3_symbol(const float* __restrict__ lpb, Conv3 c, int Np, int logNp) {
  const size_t total = (size_t)kR2 * c.CW * 2 * c.R1;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int m1 = (int)(idx % c.R1);
  const int h = (int)((idx / c.R1) % 2);
  const int col = (int)((idx / (2 * (size_t)c.R1)) % c.CW);
  const int m2 = (int)(idx / (2 * (size_t)c.R1 * c.CW));
  const unsigned m = (unsigned)(m2 + kR2 * m1);
  const int p = (int)(__brev(m) >> (32 - logNp));
  c.Lt[idx] = col <= Np ? lpb[((size_t)col * 2 + h) * Np + p] : 0.f;
}

__device__ float2 unit_root(int k, int n) {
  double s, co;
  sincospi(-2.0 * (double)k / (double)n, &s, &co);
  return make_float2((float)co, (float)s);
}

template <int LOGL>
__device__ float2 regfft_twiddle(int i) {
  using F = rf::RegFFT<float, LOGL>;
  const int k1 = i / F::TT, t = i % F::TT;
  return unit_root(t * k1, F::L);
}

__global__ void k_conv3_twiddles(Conv3 c, int Np) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Np) c.twM[i] = unit_root(i, Np);
  if (i < 64) c.tw1a[i] = regfft_twiddle<6>(i);
  if (i < c.R1) {
    if (c.logR1 == 5) c.tw1b[i] = regfft_twiddle<5>(i);
    else if (c.logR1 == 6) c.tw1b[i] = regfft_twiddle<6>(i);
    else c.tw1b[i] = regfft_twiddle<7>(i);
  }
}

template <int LOGR1>
cudaError_t launch_b(const Conv3& c, int groups, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_conv3_b<LOGR1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b<LOGR1>());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_conv3_b<LOGR1><<<dim3(groups, kR2), 32 * rf::RegFFT<float, LOGR1>::TT, smem_b<LOGR1>(), st>>>(c);
  return cudaGetLastError();
}

}  // namespace

// Used where it measured faster than the single-pass kernel: N' = 8192
// (2.71 against 3.45 ms per step at N = 8191; at N' = 4096 it took 0.61
// against 0.41 ms).  The kernels themselves serve N' = 2048 .. 8192.
bool conv3_supported(int logNp) { return logNp == 13; }

cudaError_t conv3_setup(int Np, int logNp, const float* lpb32, Conv3* c, cudaStream_t st) {
  if (!conv3_supported(logNp) || Np != (1 << logNp)) return cudaErrorInvalidValue;
  Conv3 z{};
  z.logR1 = logNp - 6;
  z.R1 = 1 << z.logR1;
  z.CW = Np + kGroup;
  const size_t nz = (size_t)Np * z.CW;
  const size_t nlt = (size_t)kR2 * z.CW * 2 * z.R1;
  cudaError_t e;
  if ((e = cudaMalloc(&z.ZE, nz * sizeof(float2))) || (e = cudaMalloc(&z.ZO, nz * sizeof(float2))) ||
      (e = cudaMalloc(&z.Lt, nlt * sizeof(float))) || (e = cudaMalloc(&z.twM, (size_t)Np * sizeof(float2))) ||
      (e = cudaMalloc(&z.tw1a, 64 * sizeof(float2))) || (e = cudaMalloc(&z.tw1b, (size_t)z.R1 * sizeof(float2)))) {
    conv3_free(&z);
    return e;
  }
  k_conv3_symbol<<<(unsigned)((nlt + 255) / 256), 256, 0, st>>>(lpb32, z, Np, logNp);
  k_conv3_twiddles<<<(Np + 255) / 256, 256, 0, st>>>(z, Np);
  if ((e = cudaGetLastError())) {
    conv3_free(&z);
    return e;
  }
  static bool attr = false;
  if (!attr) {
    if ((e = cudaFuncSetAttribute(k_conv3_a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemAC)) ||
        (e = cudaFuncSetAttribute(k_conv3_c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemAC))) {
      conv3_free(&z);
      return e;
    }
    attr = true;
  }
  *c = z;
  return cudaSuccess;
}

void conv3_free(Conv3* c) {
  void* p[] = {c->ZE, c->ZO, c->Lt, c->twM, c->tw1a, c->tw1b};
  for (void* q : p)
    if (q) cudaFree(q);
  *c = Conv3{};
}

cudaError_t launch_conv3(const Conv3& c, int N, int Np, void* Sv, const void* twv, cudaStream_t st) {
  float2* S = static_cast<float2*>(Sv);
  const float2* tw = static_cast<const float2*>(twv);
  const int groups = c.CW / kGroup;
  k_conv3_a<<<dim3(groups, c.R1), kThreadsAC, kSmemAC, st>>>(S, tw, c, N, Np);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c.logR1 == 5) e = launch_b<5>(c, groups, st);
  else if (c.logR1 == 6) e = launch_b<6>(c, groups, st);
  else if (c.logR1 == 7) e = launch_b<7>(c, groups, st);
  else e = cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  k_conv3_c<<<dim3(groups, c.R1), kThreadsAC, kSmemAC, st>>>(S, tw, c, N, Np);
  return cudaGetLastError();
}

}  // namespace sadi
