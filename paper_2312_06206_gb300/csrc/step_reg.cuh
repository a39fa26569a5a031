// step_reg.cuh -- the S-ADI step (Sec. 3, eq. "ADI scheme equivalent") for
// FFT lengths N' <= 1024 (both FP32 forms) and N' = 2048 (the dense-inverse
// form's FFT part) with the register-resident two-level FFT of regfft.cuh.
// Same four kernels and the same mathematics as step_kernels.cu:
//   kr_rows_r2c    rows of the increment d^n = u^n - u^{n-1} -> half spectrum
//                  along x (natural slots)
//   kr_cols_conv   per x frequency: y FFT (even/odd halves) x symbol, inverse
//   kr_rows_solve  inverse real FFT, remainder C += conv(d^n), B^n epilogue,
//                  x sweep (Algorithm 1)
//   kr_cols_solve  y sweep (Algorithm 1) + leapfrog
// Spectra are in natural order here (slot k holds x-frequency k, slot 0 holds
// X[0] + i X[N']); all spectral tables are natural-order copies of the FP64
// setup products.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>

#include "bf16split.cuh"
#include "regfft.cuh"
#include "sadi_internal.h"

namespace sadi {
namespace regk {

using rf::static_for;

// g(u) of the FP32 register path.  -sin u uses the hardware approximation:
// its absolute error (about 2^-21 on [-pi, pi], growing slowly with |u|) is
// scaled by tau^2 in B^n, far below the FP32 rounding of B^n itself.
__device__ __forceinline__ float g_of_r(const RegInst& I, float u) {
  if (I.gkind == 1) return -u * u * u;
  if (I.gkind == 2) return -__sinf(u);
  if (I.gkind == 3) return (I.gc1 + I.gc3 * u * u) * u + I.gcs * __sinf(u);
  return 0.f;
}

__host__ __device__ constexpr int pad32(int k) { return k + (k >> 5); }


// elements of one vector's shared buffer, rounded so that buffers of
// consecutive vectors start on staggered banks (8-byte elements, 16 per 128 B)
template <int LOGL>
__host__ __device__ constexpr int vec_smem(int res) {
  using F = rf::RegFFT<float, LOGL>;
  int n = F::E * F::ROW;
  if (n < pad32(F::L) + 1) n = pad32(F::L) + 1;
  while ((n & 15) != res) ++n;
  return n;
}
template <int LOGL, int BLOCK>
struct RowCfg {
  using F = rf::RegFFT<float, LOGL>;
  static constexpr int VB = BLOCK / F::TT;                    // vectors (rows) per block
  // transform buffer (float2).  The spectrum moves between global and shared
  // memory with the block's rows fastest (slot-major spectrum): 16 threads
  // then cover 16/VB slots x VB rows (narrow blocks) or 16 consecutive rows of
  // one slot, and a vector stride of 16/VB resp. 1 (mod 16) float2 gives them
  // 16 distinct bank pairs
  static constexpr int SMV = vec_smem<LOGL>(VB < 16 ? (16 / VB) & 15 : 1);
  static constexpr size_t tw_bytes = 2 * (size_t)F::L * sizeof(float2);   // tw1 and tw[0 .. L) staged
  static constexpr size_t bytes_r2c = (size_t)VB * SMV * sizeof(float2) + tw_bytes;
  static constexpr size_t bytes_solve = (size_t)VB * SMV * sizeof(float2) + tw_bytes;
  // resident blocks per SM promised to the compiler (its register budget):
  // four narrow blocks (two at N' = 2048, whose 64 elements per lane need
  // the full 255 registers), or one wide block of up to 2048 threads
  static constexpr int kMinBlocks = BLOCK >= 512 ? 1 : (LOGL >= 11 ? 2 : 4);
};
// The convolution kernel: vectors owned by warps (as in the row kernels), CT
// per block; the FFT buffers and the staged table tw1 (the symbol rows are
// read from global memory: without them four blocks of 128 threads fit an
// SM, against three).
template <int LOGL, int BLOCK>
struct ConvCfg {
  using F = rf::RegFFT<float, LOGL>;
  static constexpr int CT = BLOCK / F::TT;
  static_assert(CT >= 4 && CT % 2 == 0, "item 0 reads item 1's vectors: two items per block at least");
  // the staging copies of a half-warp cover CT/2 items (even vectors, 2 SMV
  // apart) x 32/CT rows: a vector stride of 16/CT (mod 16) float2 puts them
  // in distinct bank pairs
  static constexpr int SMV = vec_smem<LOGL>(CT >= 16 ? 1 : 16 / CT);
  // the half-angle twiddles tw[0 .. L) are staged too when the shared memory
  // still admits the block count of the launch bounds
  static constexpr size_t bytes_base = (size_t)CT * SMV * sizeof(float2) + (size_t)F::L * sizeof(float2);
  static constexpr int kBlocksPerSm = BLOCK >= 256 || LOGL >= 11 ? 2 : 4;
  static constexpr bool STAGE_TW =
      kBlocksPerSm * (bytes_base + F::L * sizeof(float2) + 1024) <= (size_t)228 * 1024;
  static constexpr size_t bytes = bytes_base + (STAGE_TW ? F::L * sizeof(float2) : 0);
};
template <int LOGL, int BLOCK>
struct ColCfg {
  using F = rf::RegFFT<float, LOGL>;
  static constexpr int CT = BLOCK / F::TT;                    // vectors (columns) per block
  // 8-byte accesses are served per half-warp (16 threads = CT columns x 16/CT
  // consecutive t): a column stride of 16/CT (mod 16) float2 makes the 16
  // bank pairs of a half-warp distinct
  static constexpr int SMV = vec_smem<LOGL>(CT >= 16 ? 1 : 16 / CT);
  static constexpr int STG = F::L;                            // staged state column (floats)
  // FFT buffers, staged state columns and the twiddle tables tw1 and
  // tw[0 .. L) staged once per block
  static constexpr size_t bytes_solve =
      (size_t)CT * (SMV * sizeof(float2) + 3 * STG * sizeof(float)) + 2 * (size_t)F::L * sizeof(float2);
};

// Asynchronous global -> shared copies (Ampere+ cp.async); a false predicate
// zero-fills the destination without reading global memory.
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  const int n = pred ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  const int n = pred ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  const int n = pred ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Programmatic dependent launch.  The step's kernels are launched with
// programmatic stream serialisation: a kernel may start once every block of
// the kernel before it has started (each signals that at its beginning),
// stages its constant tables, and waits for the earlier kernel to have
// completed, its writes visible, before it reads anything that kernel (or an
// earlier one) writes.  Launched without that attribute both are no-ops.
__device__ __forceinline__ void pdl_allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_prerequisites() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The twiddle tables tw1 (two-level FFT) and tw[0 .. L) staged into shared
// memory (one cp.async group): the transforms read them in their inner
// stages, where global (L1) loads would stall the few resident warps.
template <int LOGL, int BLOCK>
__device__ __forceinline__ void stage_twiddles(const RegInst& I, float2* s_tw1, float2* s_tw) {
  constexpr int L = 1 << LOGL;
  for (int e = threadIdx.x; e < L; e += BLOCK) {
    cp_async8(&s_tw1[e], I.tw1 + e, true);
    cp_async8(&s_tw[e], I.tw + e, true);
  }
}

// Gohberg-Semencul core (Algorithm 1 on the bordered matrix): x natural
// (x[q] = Q v1 at t + TT q) -> x natural (vhat).  lam tables natural order
// (global memory); tw1 and tw may be in global or shared memory.
template <int LOGL, bool WARP = false>
__device__ __forceinline__ void gs_reg(float2* x, float2* sm, int t, const float2* __restrict__ tw1,
                                       const float2* __restrict__ tw, const float2* __restrict__ lam_s,
                                       const float2* __restrict__ lam_c) {
  using F = rf::RegFFT<float, LOGL>;
  // first pass: x lambda_s then Q^H; second pass: x lambda_c.  Rolled so that the
  // kernel holds one forward and one inverse transform body.
#pragma unroll 1
  for (int round = 0; round < 2; ++round) {
    const float2* lam = round == 0 ? lam_s : lam_c;
    F::template fwd<WARP>(x, sm, t, tw1);
    static_for<0, F::E>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      x[r] = cmul(x[r], __ldg(&lam[F::template freq_index<r>(t)]));
    });
    F::template inv<WARP>(x, sm, t, tw1);
    if (round == 0) {
      static_for<0, F::E>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        x[q] = cmulc(x[q], tw[t + F::TT * q]);       // Q^H
      });
    }
  }
}

// Register <-> shared-memory moves (the only per-element code that is
// unrolled; all per-element arithmetic outside the transforms runs in
// runtime loops over shared memory to keep the kernels small).
template <int LOGL>
__device__ __forceinline__ void store_nat(const float2* x, float2* sm, int t) {
  using F = rf::RegFFT<float, LOGL>;
  static_for<0, F::E>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    sm[pad32(t + F::TT * q)] = x[q];
  });
}
template <int LOGL>
__device__ __forceinline__ void load_nat(float2* x, const float2* sm, int t) {
  using F = rf::RegFFT<float, LOGL>;
  static_for<0, F::E>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    x[q] = sm[pad32(t + F::TT * q)];
  });
}
template <int LOGL>
__device__ __forceinline__ void store_freq(const float2* x, float2* sm, int t) {
  using F = rf::RegFFT<float, LOGL>;
  static_for<0, F::E>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    sm[pad32(F::template freq_index<r>(t))] = x[r];
  });
}
template <int LOGL>
__device__ __forceinline__ void load_freq(float2* x, const float2* sm, int t) {
  using F = rf::RegFFT<float, LOGL>;
  static_for<0, F::E>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    x[r] = sm[pad32(F::template freq_index<r>(t))];
  });
}
__device__ __forceinline__ float real_at(const float2* sm, int k) {
  return reinterpret_cast<const float*>(sm + pad32(k >> 1))[k & 1];
}

// ---------------------------------------------------------------------------
// Every kernel handles one instance per blockIdx.y (a batch of independent
// problems with the same FFT length); blocks beyond an instance's extent exit.
template <int LOGL, int BLOCK>
__global__ void __launch_bounds__(BLOCK, RowCfg<LOGL, BLOCK>::kMinBlocks) kr_rows_r2c(const __grid_constant__ RegBatch B) {
  using F = rf::RegFFT<float, LOGL>;
  using C = RowCfg<LOGL, BLOCK>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_allow_dependents();
  const RegInst& I = B.in[blockIdx.y];
  const int N = I.N;
  if ((int)blockIdx.x * C::VB >= N) return;
  const int v = threadIdx.x / F::TT, t = threadIdx.x % F::TT;
  const int row = blockIdx.x * C::VB + v;
  const bool valid = row < N;
  float2* sm = reinterpret_cast<float2*>(smem_raw) + v * C::SMV;
  float2* s_tw1 = reinterpret_cast<float2*>(smem_raw) + C::VB * C::SMV;
  float2* s_tw = s_tw1 + F::L;
  stage_twiddles<LOGL, BLOCK>(I, s_tw1, s_tw);
  cp_async_commit();
  pdl_wait_prerequisites();
  // the increment d^n = u^n - u^{n-1} (zero before the first step): the
  // remainder is advanced incrementally
  const float* ur = I.u_d + (size_t)(valid ? row : 0) * I.ld;
  float2 x[F::E];
  static_for<0, F::E>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const int n = t + F::TT * q;
    // one 8-byte load per pair (aligned: even offset, rows of 128 bytes; at
    // 2n + 1 = N the second element is row padding, replaced by 0)
    float2 v = make_float2(0.f, 0.f);
    if (valid && 2 * n < N) v = *reinterpret_cast<const float2*>(ur + 2 * n);
    if (2 * n + 1 >= N) v.y = 0.f;
    x[q] = v;
  });
  cp_async_wait_all();
  __syncthreads();
  // a row vector belongs to TT threads of one warp: warp barriers from here
  F::template fwd<true>(x, sm, t, s_tw1);
  store_freq<LOGL>(x, sm, t);
  __syncthreads();
  // the spectrum is slot-major, S[k * N + row]: the block writes slot by slot,
  // its rows fastest (runs of VB rows), reading every vector's buffer
  const float2* base = reinterpret_cast<const float2*>(smem_raw);
  const int row0 = blockIdx.x * C::VB;
  // thread -> row vv of the block (fixed: BLOCK is a multiple of VB) and
  // slots k, k + BLOCK / VB, ...
  static_assert(BLOCK % C::VB == 0, "whole slot runs per block pass");
  const int vv = threadIdx.x % C::VB;
  if (row0 + vv >= N) return;
  const float2* smv = base + vv * C::SMV;
  float2* col = I.S + row0 + vv;
  // slots k <= N'/2 with their partners N' - k, which read the same two
  // buffer entries (slot 0 and slot N'/2 are their own partners)
  for (int k = threadIdx.x / C::VB; k <= F::L / 2; k += BLOCK / C::VB) {
    const int kp = (F::L - k) & (F::L - 1);
    const float2 Z = smv[pad32(k)], Zp = smv[pad32(kp)];
    const float2 Zc = cconj(Zp);
    const float2 Ev = cscale(cadd(Z, Zc), 0.5f);
    const float2 Ov = cscale(cmul_mi(csub(Z, Zc)), 0.5f);
    col[(size_t)k * N] = (k == 0) ? make_float2(Ev.x + Ov.x, Ev.x - Ov.x) : cadd(Ev, cmul(s_tw[k], Ov));
    if (kp != k) {
      const float2 Zc2 = cconj(Z);
      const float2 Ev2 = cscale(cadd(Zp, Zc2), 0.5f);
      const float2 Ov2 = cscale(cmul_mi(csub(Zp, Zc2)), 0.5f);
      col[(size_t)kp * N] = cadd(Ev2, cmul(s_tw[kp], Ov2));
    }
  }
}

// ---------------------------------------------------------------------------
// Items: 0 = x-frequency 0 (real part of slot 0), 1 = x-frequency N' (imag part
// of slot 0), i >= 2 = x-frequency i - 1 (slot i - 1).  Each item has two
// vectors (even / odd y-frequency halves), vectors c = 2 i + h of the block.
// A vector belongs to TT consecutive threads of one warp, so its transforms
// synchronise the warp only.  The block's columns arrive in shared memory by
// cp.async, so no registers are held while they are in flight; each lane's
// 32 symbol values are read from global memory (128-byte coalesced rows).
template <int LOGL, int BLOCK>
__global__ void __launch_bounds__(BLOCK, ConvCfg<LOGL, BLOCK>::kBlocksPerSm) kr_cols_conv(
    const __grid_constant__ RegBatch B) {
  using F = rf::RegFFT<float, LOGL>;
  using C = ConvCfg<LOGL, BLOCK>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_allow_dependents();
  const RegInst& I = B.in[blockIdx.y];
  const int N = I.N, Np = F::L;
  const int c = threadIdx.x / F::TT, t = threadIdx.x % F::TT;
  float2* s_tw1 = reinterpret_cast<float2*>(smem_raw) + C::CT * C::SMV;
  float2* s_tw = s_tw1 + F::L;
  const float2* twh = C::STAGE_TW ? s_tw : I.tw;   // tw[j] from shared or global memory
  if constexpr (C::STAGE_TW)
    for (int e = threadIdx.x; e < F::L; e += BLOCK) cp_async8(&s_tw[e], I.tw + e, true);
  // item, x-frequency and spectrum slot of vector cc of this block
  auto item_of = [&](int cc) { return (int)blockIdx.x * (C::CT / 2) + (cc >> 1); };
  auto slot_of = [&](int it) { return (it <= 1 || it > Np) ? 0 : it - 1; };
  auto kx_of = [&](int it) { return (it == 0 || it > Np) ? 0 : (it == 1 ? Np : it - 1); };
  for (int e = threadIdx.x; e < F::L; e += BLOCK) cp_async8(&s_tw1[e], I.tw1 + e, true);
  // each item's column, rows 0 .. N-1 (zero-filled to L), once, into the
  // buffer of its even-half vector: the spectrum is slot-major (S[k * N + j]),
  // so a column is contiguous; thread -> (item, row) with the rows fastest
  pdl_wait_prerequisites();
  constexpr int NI = C::CT / 2;
  for (int e = threadIdx.x; e < NI * F::L; e += BLOCK) {
    const int j = e % F::L, ci = e / F::L, it = item_of(2 * ci);
    float2* dst = reinterpret_cast<float2*>(smem_raw) + 2 * ci * C::SMV + pad32(j);
    const bool ok = it <= Np && j < N;
    cp_async8(dst, I.S + (size_t)(ok ? slot_of(it) : 0) * N + (ok ? j : 0), ok);
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();

  const int item = item_of(c), h = c & 1;
  float2* sm = reinterpret_cast<float2*>(smem_raw) + c * C::SMV;
  const float* lam = I.lreg + ((size_t)kx_of(item) * 2 + h) * Np;
  float2 x[F::E];
  // both halves read the column from the even vector's buffer; the barrier
  // keeps the even half's transform from overwriting it before the odd half
  // has read it
  load_nat<LOGL>(x, reinterpret_cast<const float2*>(smem_raw) + (c & ~1) * C::SMV, t);
  __syncthreads();
  // item and half are uniform over the vector's warp: branches, not selects
  if (item <= 1) {
    static_for<0, F::E>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      x[q] = item == 0 ? make_float2(x[q].x, 0.f) : make_float2(x[q].y, 0.f);
    });
  }
  if (h) {
    // odd half: y-frequencies 2 k2 + 1 of the length-2L transform
    static_for<0, F::E>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      x[q] = cmul(x[q], twh[t + F::TT * q]);
    });
  }
  F::template fwd<true>(x, sm, t, s_tw1);
  static_for<0, F::E>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    x[r] = cscale(x[r], __ldg(&lam[F::template freq_index<r>(t)]));
  });
  F::template inv<true>(x, sm, t, s_tw1);
  store_nat<LOGL>(x, sm, t);
  __syncthreads();
  // even + conj-twiddled odd half -> rows 0 .. N-1 of each item's column
  // (contiguous in the slot-major spectrum); the threads walk (item, row)
  // with the rows fastest.  Item 0 also holds the x-frequency N' result (item
  // 1's pair) in the imaginary part of slot 0.
  const float2* base = reinterpret_cast<const float2*>(smem_raw);
#pragma unroll 1
  for (int i = 0; i < C::CT / 2; ++i) {
    const int it = item_of(2 * i);
    if (it > Np || it == 1) continue;
    const float2* se = base + (2 * i) * C::SMV;
    float2* col = I.S + (size_t)slot_of(it) * N;
    for (int j = threadIdx.x; j < N; j += BLOCK) {
      const float2 w = twh[j];
      const float2 y = cadd(se[pad32(j)], cmulc(se[C::SMV + pad32(j)], w));
      if (it == 0) {
        const float2 yn = cadd(se[2 * C::SMV + pad32(j)], cmulc(se[3 * C::SMV + pad32(j)], w));
        col[j] = make_float2(y.x, yn.x);
      } else {
        col[j] = y;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// DENSE: the dense-inverse form stops after B^n, which it writes to W (FP32)
// and, split into BF16 pairs, to Bh / Bl (the first sweep GEMM's A operand).
template <int LOGL, int BLOCK, bool DENSE = false>
__global__ void __launch_bounds__(BLOCK, RowCfg<LOGL, BLOCK>::kMinBlocks) kr_rows_solve(const __grid_constant__ RegBatch B) {
  using F = rf::RegFFT<float, LOGL>;
  using C = RowCfg<LOGL, BLOCK>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_allow_dependents();
  const RegInst& I = B.in[blockIdx.y];
  const int N = I.N, Np = F::L;
  if ((int)blockIdx.x * C::VB >= N) return;
  const int v = threadIdx.x / F::TT, t = threadIdx.x % F::TT;
  const int row = blockIdx.x * C::VB + v;
  const bool valid = row < N;
  const int rrow = valid ? row : 0;
  float2* sm = reinterpret_cast<float2*>(smem_raw) + v * C::SMV;
  float2* s_tw1 = reinterpret_cast<float2*>(smem_raw) + C::VB * C::SMV;
  float2* s_tw = s_tw1 + F::L;
  stage_twiddles<LOGL, BLOCK>(I, s_tw1, s_tw);
  // the rows the B^n epilogue reads (remainder pair, u^n) into L2, one
  // request per 128-byte line, valid elements only, before waiting for the
  // convolution: neither kernel of this step before this one writes them
  // (they were written in the previous step), so the requests run under the
  // convolution's tail; a prefetch only warms L2, which is coherent, so it
  // cannot make a later load see older data
  if (valid) {
    const size_t rb = (size_t)row * I.ld;
    for (int c0 = 32 * t; c0 < N; c0 += 32 * F::TT) {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(I.C_hi + rb + c0));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(I.C_lo + rb + c0));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(I.u_hi + rb + c0));
    }
  }
  pdl_wait_prerequisites();
  // dense form: zero the sweep GEMM's counters for the GEMM that follows
  // (every kernel of the previous step, the GEMM that used them included,
  // has completed once the wait above returns)
  if constexpr (DENSE) {
    if (blockIdx.x == 0 && I.dep)
      for (int i = threadIdx.x; i < I.ndep; i += BLOCK) I.dep[i] = 0;
  }
  // stage the block's spectrum rows from the slot-major spectrum S[k * N + row]
  // (slot by slot, rows fastest: runs of VB rows); u^n, and phi2 on the
  // first step, are read in the B^n epilogue together with the remainder
  {
    float2* base = reinterpret_cast<float2*>(smem_raw);
    const int row0 = blockIdx.x * C::VB;
    static_assert(BLOCK % C::VB == 0, "whole slot runs per block pass");
    const int vv = threadIdx.x % C::VB;
    const bool ok = row0 + vv < N;
    const float2* col = I.S + (ok ? row0 + vv : 0);
    float2* dst = base + vv * C::SMV;
    for (int k = threadIdx.x / C::VB; k < F::L; k += BLOCK / C::VB)
      cp_async8(&dst[pad32(k)], col + (ok ? (size_t)k * N : 0), ok);
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  // a row vector belongs to TT threads of one warp: warp barriers from here
  // half spectrum X[k] -> Z[k] = E + i O (spectrum of z[n] = x[2n] + i x[2n+1]),
  // in place on partner pairs (k, Np - k)
#pragma unroll 2
  for (int q = 0; q <= F::E / 2; ++q) {
    const int k = t + F::TT * q;
    if (k > Np / 2 || (q == F::E / 2 && k != Np / 2)) continue;
    if (k == 0) {
      const float2 X0 = sm[pad32(0)];
      sm[pad32(0)] = make_float2(0.5f * (X0.x + X0.y), 0.5f * (X0.x - X0.y));
      continue;
    }
    const int kp = Np - k;
    const float2 X = sm[pad32(k)], Xq = sm[pad32(kp)];
    const float2 Ev = cscale(cadd(X, cconj(Xq)), 0.5f);
    const float2 Ov = cscale(cmulc(csub(X, cconj(Xq)), s_tw[k]), 0.5f);
    sm[pad32(k)] = cadd(Ev, cmul_pi(Ov));
    if (kp != k) {
      const float2 Eq = cscale(cadd(Xq, cconj(X)), 0.5f);
      const float2 Oq = cscale(cmulc(csub(Xq, cconj(X)), s_tw[kp]), 0.5f);
      sm[pad32(kp)] = cadd(Eq, cmul_pi(Oq));
    }
  }
  __syncwarp();
  float2 x[F::E];
  load_freq<LOGL>(x, sm, t);
  __syncwarp();
  F::template inv<true>(x, sm, t, s_tw1);
  store_nat<LOGL>(x, sm, t);
  __syncwarp();
  // B^n in place: sm[n] holds the convolution at 2n, 2n+1 (real view).  The
  // remainder pairs of four q are loaded before any of them is stored (the
  // loads overlap instead of waiting one after another).  The convolution is
  // that of the increment d^n; the wave step takes B = C + tau^2 (g(u) + f)
  // (n = 0: tau phi2 + (C + tau^2 (g + f))/2) with C <- C + conv, the
  // diffusion step B = C + conv/2 + tau (g(u~) + f) - d, u~ = u + d/2
  // (C + conv/2 = -kappa tau L_h u~; d = 0 at n = 0).
  const float tau = I.tau, tau2 = I.tau2;
  const size_t rbase = (size_t)rrow * I.ld;
  // the equation is uniform over the launch: one loop per equation, so the
  // wave step's loop carries nothing of the diffusion step's
  auto bn_loop = [&](auto diff_c) {
    constexpr bool DIFF = decltype(diff_c)::value;
    // pairs n < N'/2 only: x = 2n < N <= N' (the x sweep reads no more)
#pragma unroll 1
    for (int q0 = 0; q0 < F::E / 2; q0 += 4) {
      // the pairs x = 2n, 2n + 1 as 8-byte loads: rows start on 128-byte
      // boundaries and the row pitch is even, so a pair is aligned, and at
      // x = N - 1 (odd N) its second element is row padding, in bounds
      float2 ch[4], cl[4], uv[4], dv[4];
#pragma unroll
      for (int j2 = 0; j2 < 4; ++j2) {
        const int x = 2 * (t + F::TT * (q0 + j2));
        const bool ok = valid && x < N;
        const size_t at = ok ? rbase + x : 0;
        const float2 z = make_float2(0.f, 0.f);
        ch[j2] = ok ? *reinterpret_cast<const float2*>(I.C_hi + at) : z;
        cl[j2] = ok ? *reinterpret_cast<const float2*>(I.C_lo + at) : z;
        uv[j2] = ok ? *reinterpret_cast<const float2*>(I.u_hi + at) : z;
        if constexpr (DIFF) dv[j2] = (ok && !I.first) ? *reinterpret_cast<const float2*>(I.u_d + at) : z;
      }
#pragma unroll
      for (int j2 = 0; j2 < 4; ++j2) {
        const int n = t + F::TT * (q0 + j2);
        const float2 cv = sm[pad32(n)];
        float b[2] = {0.f, 0.f}, cn[2] = {0.f, 0.f}, cln[2] = {0.f, 0.f};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int x = 2 * n + e;
          if (valid && x < N) {
            // C <- C + conv (two-sum into the double-float pair)
            const float hi = e ? ch[j2].y : ch[j2].x, lo = e ? cl[j2].y : cl[j2].x, cx = e ? cv.y : cv.x;
            const float s = hi + cx;
            const float bb = s - hi;
            const float err = (hi - (s - bb)) + (cx - bb);
            const float l2 = lo + err;
            const float c = s + l2;
            cn[e] = c;
            cln[e] = l2 - (c - s);
            const float u = e ? uv[j2].y : uv[j2].x;
            if constexpr (!DIFF) {
              float gs = g_of_r(I, u);
              if (I.F) gs += I.fsc * I.F[rbase + x];
              const float gg = tau2 * gs;
              b[e] = I.first ? tau * I.phi2[rbase + x] + 0.5f * (c + gg) : c + gg;
            } else {
              const float d = e ? dv[j2].y : dv[j2].x;
              float gs = g_of_r(I, u + 0.5f * d);
              if (I.F) gs += I.fsc * I.F[rbase + x];
              b[e] = (c + 0.5f * cx) + tau2 * gs - d;
            }
          }
        }
        // the updated remainder pair: one 8-byte store each, or the single
        // element at x = N - 1 (the padding is never written)
        const int x = 2 * n;
        if (valid && x + 1 < N) {
          *reinterpret_cast<float2*>(I.C_hi + rbase + x) = make_float2(cn[0], cn[1]);
          *reinterpret_cast<float2*>(I.C_lo + rbase + x) = make_float2(cln[0], cln[1]);
        } else if (valid && x < N) {
          I.C_hi[rbase + x] = cn[0];
          I.C_lo[rbase + x] = cln[0];
        }
        if constexpr (DENSE) {
          // B^n of the pair straight to W (8 bytes, or the last element)
          // and its BF16 pairs (one 4-byte store each; the row pitch ldp is
          // even, and at x = N, the zero padding, the split of 0 is stored)
          if (valid && x < N) {
            float* wr = I.W + rbase;
            if (x + 1 < N) *reinterpret_cast<float2*>(wr + x) = make_float2(b[0], b[1]);
            else wr[x] = b[0];
            unsigned hi, lo;
            split_bf16x2(b[0], b[1], &hi, &lo);
            *reinterpret_cast<unsigned*>(I.Bh + (size_t)rrow * I.ldp + x) = hi;
            *reinterpret_cast<unsigned*>(I.Bl + (size_t)rrow * I.ldp + x) = lo;
          }
        } else {
          sm[pad32(n)] = make_float2(b[0], b[1]);
        }
      }
    }
  };
  if (I.eq == 1) bn_loop(std::integral_constant<bool, true>{});
  else bn_loop(std::integral_constant<bool, false>{});
  __syncwarp();
  if constexpr (DENSE) return;
  // v1 = Q (B' + i J B')
  static_for<0, F::E>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const int k = t + F::TT * q;
    x[q] = cmul(make_float2(real_at(sm, k), real_at(sm, Np - 1 - k)), s_tw[k]);
  });
  __syncwarp();
  gs_reg<LOGL, true>(x, sm, t, s_tw1, s_tw, I.lam_s, I.lam_c);
  store_nat<LOGL>(x, sm, t);
  __syncwarp();
  if (!valid) return;
  // (H^-1 B)[k] = Re vhat[k] + Im vhat[Np-1-k] + sum_q G[k,q] ybot[q],
  // ybot[q] = Re vhat[N+q] + Im vhat[r-1-q]
  const int r = I.r;
  float* wrow = I.W + (size_t)row * I.ld;
#pragma unroll 2
  for (int q = 0; q < F::E; ++q) {
    const int k = t + F::TT * q;
    if (k < N) {
      float y = sm[pad32(k)].x + sm[pad32(Np - 1 - k)].y;
      for (int qq = 0; qq < r; ++qq)
        y += __ldg(&I.G[(size_t)k * r + qq]) * (sm[pad32(N + qq)].x + sm[pad32(r - 1 - qq)].y);
      wrow[k] = y;
    }
  }
}

// ---------------------------------------------------------------------------
template <int LOGL, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 3) kr_cols_solve(const __grid_constant__ RegBatch B) {
  using F = rf::RegFFT<float, LOGL>;
  using C = ColCfg<LOGL, BLOCK>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_allow_dependents();
  const RegInst& I = B.in[blockIdx.y];
  const int N = I.N, Np = F::L;
  if ((int)blockIdx.x * C::CT >= N) return;
  const int c = threadIdx.x % C::CT, t = threadIdx.x / C::CT;
  const int i = blockIdx.x * C::CT + c;
  const bool valid = i < N;
  const int ii = valid ? i : 0;
  float2* sm = reinterpret_cast<float2*>(smem_raw) + c * C::SMV;
  // 4-byte staging arrays are interleaved by column ([k * CT + c]) so that a
  // warp (CT columns x 32/CT consecutive k) touches 32 consecutive words.
  float* st = reinterpret_cast<float*>(reinterpret_cast<float2*>(smem_raw) + C::CT * C::SMV);
  float* s_hi = st;
  float* s_lo = st + C::CT * C::STG;
  float* s_d = st + 2 * C::CT * C::STG;
  float2* s_tw1 = reinterpret_cast<float2*>(st + 3 * C::CT * C::STG);
  float2* s_tw = s_tw1 + F::L;
  stage_twiddles<LOGL, BLOCK>(I, s_tw1, s_tw);
  cp_async_commit();
  pdl_wait_prerequisites();
  // the state column (needed at the end) is staged asynchronously; the W
  // column (needed now) is loaded straight into registers, all loads in flight
  static_for<0, F::E>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const int k = t + F::TT * q;
    const bool in = valid && k < N;
    const size_t gi = (size_t)(in ? k : 0) * I.ld + ii;
    cp_async4(&s_hi[k * C::CT + c], I.u_hi + gi, in);
    cp_async4(&s_lo[k * C::CT + c], I.u_lo + gi, in);
    cp_async4(&s_d[k * C::CT + c], I.u_d + gi, in && !I.first);
  });
  cp_async_commit();
  float2 x[F::E];
  static_for<0, F::E>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const int k = t + F::TT * q, k2 = Np - 1 - k;
    const float a = (valid && k < N) ? I.W[(size_t)k * I.ld + ii] : 0.f;
    const float b = (valid && k2 < N) ? I.W[(size_t)k2 * I.ld + ii] : 0.f;
    x[q] = make_float2(a, b);
  });
  // the twiddle group (committed first) has landed once at most the state
  // group is still pending
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  __syncthreads();
  static_for<0, F::E>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    x[q] = cmul(x[q], s_tw[t + F::TT * q]);
  });
  gs_reg<LOGL>(x, sm, t, s_tw1, s_tw, I.lam_s, I.lam_c);
  store_nat<LOGL>(x, sm, t);
  cp_async_wait_all();
  __syncthreads();
  if (!valid) return;
  const int r = I.r;
  const int first = I.first;
#pragma unroll 2
  for (int q = 0; q < F::E; ++q) {
    const int j = t + F::TT * q;
    if (j < N) {
      float uh = sm[pad32(j)].x + sm[pad32(Np - 1 - j)].y;
      for (int qq = 0; qq < r; ++qq)
        uh += __ldg(&I.G[(size_t)j * r + qq]) * (sm[pad32(N + qq)].x + sm[pad32(r - 1 - qq)].y);
      // compensated leapfrog: d^{n+1} = d^n + uhat (d^1 = uhat), u^{n+1} = u^n + d^{n+1}
      // with u = u_hi + u_lo kept as a double-float pair (two-sum)
      const float d = first ? uh : s_d[j * C::CT + c] + uh;
      const float hi = s_hi[j * C::CT + c], lo = s_lo[j * C::CT + c];
      const float s = hi + d;
      const float bb = s - hi;
      const float err = (hi - (s - bb)) + (d - bb);
      const float l2 = lo + err;
      const float h2 = s + l2;
      const size_t idx = (size_t)j * I.ld + i;
      I.u_hi[idx] = h2;
      I.u_lo[idx] = l2 - (h2 - s);
      I.u_d[idx] = d;
    }
  }
}

constexpr int kRowBlock = 128;
constexpr int kColBlock = 128;
constexpr int kConvBlock = 128;
// Wide row blocks at N' = 1024: 21 rows (672 threads, at most 96 registers a
// thread, which the row kernels meet without spilling; 192 KB of shared
// memory with the twiddles staged once), one block per SM, against four
// narrow blocks of 4 rows.  The row kernels take them
// when they need fewer waves: three 1023-row instances are 147 wide blocks
// in one wave, or 768 narrow ones in 1.26 waves of 608.
constexpr int kRowBlockWide = 672;

// SM count and resident narrow / wide blocks per SM, packed (0 = unknown)
inline int pack_shape(int sms, int narrow, int wide) {
  return sms > 0 && sms < 32768 && narrow > 0 && narrow < 256 && wide > 0 && wide < 256
             ? (sms << 16) | (narrow << 8) | wide
             : 0;
}
// true when blocks of wide_rows rows take fewer waves than blocks of
// narrow_rows rows for count instances of up to max_n rows
inline bool fewer_waves(int shape, int count, int max_n, int narrow_rows, int wide_rows) {
  if (!shape) return false;
  const long sms = shape >> 16, on = (shape >> 8) & 255, ow = shape & 255;
  const long nb = (long)count * ((max_n + narrow_rows - 1) / narrow_rows);
  const long wb = (long)count * ((max_n + wide_rows - 1) / wide_rows);
  return (wb + sms * ow - 1) / (sms * ow) < (nb + sms * on - 1) / (sms * on);
}

// FFT lengths of the register path: both FP32 forms up to 2^kRegMaxLogGS, the
// dense-inverse form's FFT part (no GS sweeps) up to 2^kRegMaxLogDense.  At
// N' = 2048 the GS sweep kernels would hold 64 elements per lane at the full
// register budget, 2 blocks per SM, and measured slower than the
// shared-memory engine's; the dense form's three kernels measured faster.
constexpr int kRegMaxLogGS = 10;
constexpr int kRegMaxLogDense = 11;

template <int LOGL>
cudaError_t launch_reg_impl(const RegBatch& b, int max_n, cudaStream_t st, cudaEvent_t* ev, bool dense) {
  static_assert(LOGL <= kRegMaxLogDense, "register path FFT length");
  // the GS form's kernels (and the wide row blocks, N' = 1024 only) exist at
  // the lengths that use them
  constexpr bool kGS = LOGL <= kRegMaxLogGS;
  if (!kGS && !dense) return cudaErrorInvalidValue;
  using RC = RowCfg<LOGL, kRowBlock>;
  using CC = ColCfg<LOGL, kColBlock>;
  using VC = ConvCfg<LOGL, kConvBlock>;
  using RW = RowCfg<LOGL, kRowBlockWide>;
  constexpr int Np = 1 << LOGL;
  static LaunchCache attr_done[kLauncherDevices];
  // narrow / wide occupancy of the row kernels (r2c, GS solve, dense B^n),
  // written before attr_done is published and read after it
  static LaunchCache shape[3][kLauncherDevices];
  const int dev = device_slot();
  if (dev < 0) return cudaErrorInvalidDevice;
  if (!attr_done[dev].load(std::memory_order_acquire)) {
    cudaError_t e;
    if constexpr (LOGL == 10) {
      int sms = 0;
      if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
      // resident narrow and wide blocks per SM of one row kernel
      auto measure = [&](auto kn, auto kw, size_t bn, size_t bw, LaunchCache& out) {
        int on = 0, ow = 0;
        cudaError_t r;
        if ((r = cudaFuncSetAttribute(kn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bn)) ||
            (r = cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bw)) ||
            (r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&on, kn, kRowBlock, bn)) ||
            (r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ow, kw, kRowBlockWide, bw)))
          return r;
        out.store(pack_shape(sms, on, ow), std::memory_order_relaxed);
        return cudaSuccess;
      };
      if ((e = measure(kr_rows_r2c<LOGL, kRowBlock>, kr_rows_r2c<LOGL, kRowBlockWide>, RC::bytes_r2c, RW::bytes_r2c,
                       shape[0][dev])) ||
          (e = measure(kr_rows_solve<LOGL, kRowBlock>, kr_rows_solve<LOGL, kRowBlockWide>, RC::bytes_solve,
                       RW::bytes_solve, shape[1][dev])) ||
          (e = measure(kr_rows_solve<LOGL, kRowBlock, true>, kr_rows_solve<LOGL, kRowBlockWide, true>,
                       RC::bytes_solve, RW::bytes_solve, shape[2][dev])))
        return e;
    }
    if ((e = cudaFuncSetAttribute(kr_rows_r2c<LOGL, kRowBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)RC::bytes_r2c)) ||
        (e = cudaFuncSetAttribute(kr_rows_solve<LOGL, kRowBlock, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::bytes_solve)) ||
        (e = cudaFuncSetAttribute(kr_cols_conv<LOGL, kConvBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)VC::bytes)))
      return e;
    if constexpr (kGS) {
      if ((e = cudaFuncSetAttribute(kr_rows_solve<LOGL, kRowBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)RC::bytes_solve)) ||
          (e = cudaFuncSetAttribute(kr_cols_solve<LOGL, kColBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)CC::bytes_solve)))
        return e;
    }
    attr_done[dev].store(1, std::memory_order_release);
  }
  const dim3 rgrid((max_n + RC::VB - 1) / RC::VB, b.count);
  const dim3 cgrid((Np + 1 + VC::CT / 2 - 1) / (VC::CT / 2), b.count);
  const dim3 sgrid((max_n + CC::CT - 1) / CC::CT, b.count);
  // wide row blocks where they take fewer waves (N' = 1024 only)
  bool wide[3] = {false, false, false};
  if constexpr (LOGL == 10)
    for (int k = 0; k < 3; ++k)
      wide[k] = fewer_waves(shape[k][dev].load(std::memory_order_relaxed), b.count, max_n, RC::VB, RW::VB);
  const dim3 wgrid((max_n + RW::VB - 1) / RW::VB, b.count);
  // every kernel of the step is a programmatic dependent of the one before it
  // in the stream (see pdl_wait_prerequisites)
  cudaLaunchAttribute pdl[1];
  pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl[0].val.programmaticStreamSerializationAllowed = 1;
  auto launch = [&](auto kernel, dim3 grid, int block, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = pdl;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, b);
  };
  cudaError_t e;
  if (ev) cudaEventRecord(ev[0], st);
  if constexpr (LOGL == 10) {
    if (wide[0]) e = launch(kr_rows_r2c<LOGL, kRowBlockWide>, wgrid, kRowBlockWide, RW::bytes_r2c);
    else e = launch(kr_rows_r2c<LOGL, kRowBlock>, rgrid, kRowBlock, RC::bytes_r2c);
  } else {
    e = launch(kr_rows_r2c<LOGL, kRowBlock>, rgrid, kRowBlock, RC::bytes_r2c);
  }
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[1], st);
  if ((e = launch(kr_cols_conv<LOGL, kConvBlock>, cgrid, kConvBlock, VC::bytes))) return e;
  if (ev) cudaEventRecord(ev[2], st);
  if (dense) {
    if constexpr (LOGL == 10) {
      if (wide[2]) return launch(kr_rows_solve<LOGL, kRowBlockWide, true>, wgrid, kRowBlockWide, RW::bytes_solve);
    }
    return launch(kr_rows_solve<LOGL, kRowBlock, true>, rgrid, kRowBlock, RC::bytes_solve);
  }
  if constexpr (kGS) {
    if constexpr (LOGL == 10) {
      if (wide[1]) e = launch(kr_rows_solve<LOGL, kRowBlockWide>, wgrid, kRowBlockWide, RW::bytes_solve);
      else e = launch(kr_rows_solve<LOGL, kRowBlock>, rgrid, kRowBlock, RC::bytes_solve);
    } else {
      e = launch(kr_rows_solve<LOGL, kRowBlock>, rgrid, kRowBlock, RC::bytes_solve);
    }
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[3], st);
    if ((e = launch(kr_cols_solve<LOGL, kColBlock>, sgrid, kColBlock, CC::bytes_solve))) return e;
    if (ev) cudaEventRecord(ev[4], st);
  }
  return cudaSuccess;
}

}  // namespace regk
}  // namespace sadi
