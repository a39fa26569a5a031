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
// Every global access covers 16 adjacent columns of a row (128 bytes),
// where the single-pass shared-memory kernel gathers one 8-byte element per
// row; the two halves' intermediates (N' x (N' + 16) complex each) live in
// HBM between the passes.  The small transforms are the register FFT of
// regfft.cuh, one vector per TT threads of a warp.  Each pass is a
// persistent loop over its work items whose next item's tiles arrive by
// cp.async while the current one is transformed and stored.
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

constexpr int kGroup = 16;           // columns per work item
constexpr int kR2 = 64;              // length of the strided transforms (passes A, C)
constexpr int kTP = kGroup + 2;      // tile row pitch (float2): 16-byte rows, spread banks
constexpr int kThreadsAC = 32 * 8;   // 32 vectors x 8 threads (RegFFT<6>: TT = 8)

template <int LOGL>
constexpr int vec_elems() {
  return rf::RegFFT<float, LOGL>::E * rf::RegFFT<float, LOGL>::ROW;
}

// Asynchronous copies global -> shared; a false predicate zero-fills.
__device__ __forceinline__ void cp16(void* dst, const void* src, bool pred) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(pred ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp8(void* dst, const void* src, bool pred) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(pred ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Copy `rows` rows of 16 columns (starting at column 16 grp of row row0 +
// stride r) of a CW-column array into a tile, 16 bytes per copy.
__device__ __forceinline__ void load_tile(float2* tile, const float2* Z, int CW, int row0, int stride, int rows,
                                          int grp, int nthreads) {
  for (int e = threadIdx.x; e < rows * (kGroup / 2); e += nthreads) {
    const int r = e / (kGroup / 2), p = e % (kGroup / 2);
    cp16(tile + r * kTP + 2 * p, Z + (size_t)(row0 + stride * r) * CW + kGroup * grp + 2 * p, true);
  }
}

// Pass A input: column gc of spectrum rows j1 + R1 r (zero from row N on).
// The copies are raw; column 0 keeps only its real part and column N' (slot
// 0 again) only its imaginary part, fixed when the tile is read.
__device__ __forceinline__ void load_columns(float2* tile, const float2* S, int N, int Np, int j1, int R1,
                                             int grp) {
  const bool last = kGroup * grp == Np;
  for (int e = threadIdx.x; e < kR2 * (kGroup / 2); e += kThreadsAC) {
    const int r = e / (kGroup / 2), p = e % (kGroup / 2);
    const int j = j1 + R1 * r;
    const bool in = j < N;
    const float2* row = S + (size_t)(in ? j : 0) * Np;
    if (!last) {
      cp16(tile + r * kTP + 2 * p, row + kGroup * grp + 2 * p, in);
    } else {
      cp8(tile + r * kTP + 2 * p, row, in && p == 0);
      cp8(tile + r * kTP + 2 * p + 1, row, false);
    }
  }
}

__device__ __forceinline__ float2 column_value(float2 v, int gc, int Np) {
  if (gc == 0) return make_float2(v.x, 0.f);
  if (gc == Np) return make_float2(v.y, 0.f);
  return gc > Np ? make_float2(0.f, 0.f) : v;
}

// shared memory: passes A and C hold two buffers of two tiles each, 32
// transform buffers and the 64-point twiddles; pass B the same with R1-row tiles
constexpr size_t kSmemAC = (size_t)(4 * kR2 * kTP + 32 * vec_elems<6>() + 64) * sizeof(float2);
template <int LOGR1>
constexpr size_t smem_b() {
  return (size_t)(4 * (1 << LOGR1) * kTP + 32 * vec_elems<LOGR1>() + (1 << LOGR1)) * sizeof(float2);
}

// Each block walks the work items t = blockIdx.x, + gridDim.x, ...; the
// copies of the next item are in flight while the current one is computed
// and stored.  Barriers: (1) after the wait, the item's tiles are complete;
// (2) after the compute, the results are in shared memory; (3) after the
// stores, the buffer may be refilled.
__global__ void __launch_bounds__(kThreadsAC) k_conv3_a(const float2* __restrict__ S, const float2* __restrict__ tw,
                                                        Conv3 c, int N, int Np) {
  pdl_entry();
  using F = rf::RegFFT<float, 6>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s_buf = reinterpret_cast<float2*>(smem_raw);   // [2 buffers][2 tiles][kR2 * kTP]
  float2* s_fft = s_buf + 4 * kR2 * kTP;
  float2* s_tw1 = s_fft + 32 * vec_elems<6>();
  const int groups = c.CW / kGroup, R1 = c.R1, total = groups * R1, tid = threadIdx.x;
  if (tid < 64) s_tw1[tid] = c.tw1a[tid];
  int it = blockIdx.x;
  if (it < total) load_columns(s_buf, S, N, Np, it / groups, R1, it % groups);
  cp_commit();
  const int v = tid / F::TT, t = tid % F::TT, cl = v >> 1, h = v & 1;
  for (int b = 0; it < total; it += gridDim.x, b ^= 1) {
    const int next = it + gridDim.x;
    if (next < total) load_columns(s_buf + (b ^ 1) * 2 * kR2 * kTP, S, N, Np, next / groups, R1, next % groups);
    cp_commit();
    cp_wait<1>();
    __syncthreads();
    const int j1 = it / groups, grp = it % groups, gc = kGroup * grp + cl;
    float2* in = s_buf + b * 2 * kR2 * kTP;   // tile 0: input; tiles 0 / 1 then hold the halves
    float2 x[F::E];
    static_for<0, F::E>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const int j2 = t + F::TT * q;
      const float2 val = column_value(in[j2 * kTP + cl], gc, Np);
      x[q] = h ? cmul(val, __ldg(&tw[j1 + R1 * j2])) : val;
    });
    __syncthreads();   // every vector has read the input tile
    F::template fwd<true>(x, s_fft + v * vec_elems<6>(), t, s_tw1);
    static_for<0, F::E>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      const int m2 = F::template freq_index<r>(t);
      in[h * kR2 * kTP + m2 * kTP + cl] = cmul(x[r], __ldg(&c.twM[j1 * m2]));
    });
    __syncthreads();
    for (int e = tid; e < 2 * kR2 * (kGroup / 2); e += kThreadsAC) {
      const int hh = e / (kR2 * (kGroup / 2)), r = (e / (kGroup / 2)) % kR2, p = e % (kGroup / 2);
      float2* Z = hh ? c.ZO : c.ZE;
      const float4 val = *reinterpret_cast<const float4*>(in + hh * kR2 * kTP + r * kTP + 2 * p);
      *reinterpret_cast<float4*>(Z + (size_t)(j1 + R1 * r) * c.CW + kGroup * grp + 2 * p) = val;
    }
    __syncthreads();
  }
  cp_wait<0>();
}

template <int LOGR1>
__global__ void __launch_bounds__(32 * rf::RegFFT<float, LOGR1>::TT) k_conv3_b(Conv3 c) {
  pdl_entry();
  using F = rf::RegFFT<float, LOGR1>;
  constexpr int R1 = 1 << LOGR1;
  constexpr int NT = 32 * F::TT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s_buf = reinterpret_cast<float2*>(smem_raw);   // [2 buffers][2 halves][R1 * kTP]
  float2* s_fft = s_buf + 4 * R1 * kTP;
  float2* s_tw1 = s_fft + 32 * vec_elems<LOGR1>();
  const int groups = c.CW / kGroup, total = groups * kR2, tid = threadIdx.x;
  for (int e = tid; e < R1; e += NT) s_tw1[e] = c.tw1b[e];
  auto load = [&](float2* buf, int item) {
    const int m2 = item / groups, grp = item % groups;
    load_tile(buf, c.ZE, c.CW, R1 * m2, 1, R1, grp, NT);
    load_tile(buf + R1 * kTP, c.ZO, c.CW, R1 * m2, 1, R1, grp, NT);
  };
  int it = blockIdx.x;
  if (it < total) load(s_buf, it);
  cp_commit();
  const int v = tid / F::TT, t = tid % F::TT, cl = v >> 1, h = v & 1;
  for (int b = 0; it < total; it += gridDim.x, b ^= 1) {
    const int next = it + gridDim.x;
    if (next < total) load(s_buf + (b ^ 1) * 2 * R1 * kTP, next);
    cp_commit();
    const int m2 = it / groups, grp = it % groups;
    // the symbol values of this thread (frequency layout), loaded under the wait
    const float* lam = c.Lt + ((size_t)(m2 * c.CW + kGroup * grp + cl) * 2 + h) * R1;
    float lv[F::E];
    static_for<0, F::E>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      lv[r] = __ldg(lam + F::template freq_index<r>(t));
    });
    cp_wait<1>();
    __syncthreads();
    // each element of the vector's column is read and later written by the
    // same thread (natural layout before the forward, after the inverse)
    float2* tile = s_buf + b * 2 * R1 * kTP + h * R1 * kTP;
    float2 x[F::E];
    static_for<0, F::E>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      x[q] = tile[(t + F::TT * q) * kTP + cl];
    });
    F::template fwd<true>(x, s_fft + v * vec_elems<LOGR1>(), t, s_tw1);
    static_for<0, F::E>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      x[r] = cscale(x[r], lv[r]);
    });
    F::template inv<true>(x, s_fft + v * vec_elems<LOGR1>(), t, s_tw1);
    static_for<0, F::E>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const int j1 = t + F::TT * q;
      tile[j1 * kTP + cl] = cmulc(x[q], __ldg(&c.twM[j1 * m2]));
    });
    __syncthreads();
    const float2* buf = s_buf + b * 2 * R1 * kTP;
    for (int e = tid; e < 2 * R1 * (kGroup / 2); e += NT) {
      const int hh = e / (R1 * (kGroup / 2)), r = (e / (kGroup / 2)) % R1, p = e % (kGroup / 2);
      float2* Z = hh ? c.ZO : c.ZE;
      const float4 val = *reinterpret_cast<const float4*>(buf + hh * R1 * kTP + r * kTP + 2 * p);
      *reinterpret_cast<float4*>(Z + (size_t)(r + R1 * m2) * c.CW + kGroup * grp + 2 * p) = val;
    }
    __syncthreads();
  }
  cp_wait<0>();
}

__global__ void __launch_bounds__(kThreadsAC) k_conv3_c(float2* __restrict__ S, const float2* __restrict__ tw,
                                                        Conv3 c, int N, int Np) {
  pdl_entry();
  using F = rf::RegFFT<float, 6>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s_buf = reinterpret_cast<float2*>(smem_raw);   // [2 buffers][2 halves][kR2 * kTP]
  float2* s_fft = s_buf + 4 * kR2 * kTP;
  float2* s_tw1 = s_fft + 32 * vec_elems<6>();
  const int groups = c.CW / kGroup, R1 = c.R1, total = groups * R1, tid = threadIdx.x;
  if (tid < 64) s_tw1[tid] = c.tw1a[tid];
  auto load = [&](float2* buf, int item) {
    const int j1 = item / groups, grp = item % groups;
    load_tile(buf, c.ZE, c.CW, j1, R1, kR2, grp, kThreadsAC);
    load_tile(buf + kR2 * kTP, c.ZO, c.CW, j1, R1, kR2, grp, kThreadsAC);
  };
  int it = blockIdx.x;
  if (it < total) load(s_buf, it);
  cp_commit();
  const int v = tid / F::TT, t = tid % F::TT, cl = v >> 1, h = v & 1;
  for (int b = 0; it < total; it += gridDim.x, b ^= 1) {
    const int next = it + gridDim.x;
    if (next < total) load(s_buf + (b ^ 1) * 2 * kR2 * kTP, next);
    cp_commit();
    cp_wait<1>();
    __syncthreads();
    const int j1 = it / groups, grp = it % groups;
    float2* buf = s_buf + b * 2 * kR2 * kTP;
    float2* tile = buf + h * kR2 * kTP;
    float2 x[F::E];
    static_for<0, F::E>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      x[r] = tile[F::template freq_index<r>(t) * kTP + cl];
    });
    // the transform's internal warp barriers order every read of the
    // vector's column before the writes below
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
      const float2 y = cadd(buf[r * kTP + cc], cmulc(buf[kR2 * kTP + r * kTP + cc], __ldg(&tw[j])));
      if (gc == 0) reinterpret_cast<float*>(S + (size_t)j * Np)[0] = y.x;
      else if (gc == Np) reinterpret_cast<float*>(S + (size_t)j * Np)[1] = y.x;
      else S[(size_t)j * Np + gc] = y;
    }
    __syncthreads();
  }
  cp_wait<0>();
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

// Persistent grid: as many blocks as are resident at once (at most one per
// work item).
template <typename K>
cudaError_t resident_grid(K kernel, int threads, size_t smem, int items, int* grid) {
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  const int g = sms * (per > 0 ? per : 1);
  *grid = g < items ? g : items;
  return cudaSuccess;
}

template <int LOGR1>
cudaError_t launch_b(const Conv3& c, int groups, cudaStream_t st) {
  constexpr int NT = 32 * rf::RegFFT<float, LOGR1>::TT;
  static LaunchCache grids[kLauncherDevices];
  const int dev = device_slot();
  if (dev < 0) return cudaErrorInvalidDevice;
  int grid = grids[dev].load(std::memory_order_acquire);
  if (!grid) {
    cudaError_t e =
        cudaFuncSetAttribute(k_conv3_b<LOGR1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b<LOGR1>());
    if (e == cudaSuccess) e = resident_grid(k_conv3_b<LOGR1>, NT, smem_b<LOGR1>(), 1 << 30, &grid);
    if (e != cudaSuccess) return e;
    grids[dev].store(grid, std::memory_order_release);
  }
  const int items = groups * kR2;
  return launch_dependent(k_conv3_b<LOGR1>, dim3(grid < items ? grid : items), dim3(NT), smem_b<LOGR1>(), st, c);
}

}  // namespace

// The kernels serve N' = 2048 .. 8192; the step's default uses them at 8192,
// where they measured faster than the single-pass kernel (1.83 against 3.45
// ms per step at N = 8191; at N' = 4096 0.44 against 0.41 ms).
bool conv3_supported(int logNp) { return logNp >= 11 && logNp <= 13; }

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
  static LaunchCache attrs[kLauncherDevices];
  const int dev = device_slot();
  if (dev < 0) {
    conv3_free(&z);
    return cudaErrorInvalidDevice;
  }
  if (!attrs[dev].load(std::memory_order_acquire)) {
    if ((e = cudaFuncSetAttribute(k_conv3_a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemAC)) ||
        (e = cudaFuncSetAttribute(k_conv3_c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemAC))) {
      conv3_free(&z);
      return e;
    }
    attrs[dev].store(1, std::memory_order_release);
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
  const int groups = c.CW / kGroup, items = groups * c.R1;
  static LaunchCache grids_ac[kLauncherDevices];
  const int dev = device_slot();
  if (dev < 0) return cudaErrorInvalidDevice;
  int grid_ac = grids_ac[dev].load(std::memory_order_acquire);
  if (!grid_ac) {
    const cudaError_t e = resident_grid(k_conv3_a, kThreadsAC, kSmemAC, 1 << 30, &grid_ac);
    if (e != cudaSuccess) return e;
    grids_ac[dev].store(grid_ac, std::memory_order_release);
  }
  const int gac = grid_ac < items ? grid_ac : items;
  // the three passes are programmatic dependents, each of the one before it
  cudaError_t e = launch_dependent(k_conv3_a, dim3(gac), dim3(kThreadsAC), kSmemAC, st, static_cast<const float2*>(S),
                                   tw, c, N, Np);
  if (e != cudaSuccess) return e;
  if (c.logR1 == 5) e = launch_b<5>(c, groups, st);
  else if (c.logR1 == 6) e = launch_b<6>(c, groups, st);
  else if (c.logR1 == 7) e = launch_b<7>(c, groups, st);
  else e = cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  return launch_dependent(k_conv3_c, dim3(gac), dim3(kThreadsAC), kSmemAC, st, S, tw, c, N, Np);
}

}  // namespace sadi
