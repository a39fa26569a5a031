// gemm_tc.cu -- split-BF16 GEMM on the 5th-generation tensor cores (tcgen05)
// for the dense-inverse form of the two ADI sweeps.
//
// Computes ACC = A B^T (FP32 accumulate) where both FP32 operands are given as
// BF16 pairs X = X_hi + X_lo (X_hi = BF16 round-to-nearest of X, X_lo = BF16
// of the remainder):
//     ACC = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T       (A_lo B_lo^T dropped)
// All operands are K-major (row-major, K contiguous), zero-padded to whole
// tiles.  Per-element representation error of a pair is <= 2^-16 relative, so
// ACC carries about 2^-16 relative error on top of FP32 accumulation.
//
// Persistent: one CTA per SM (at most one per tile) walks the output tiles
// of all problems of the launch, 128 x 256 when there are enough of them to
// give every SM two, else 128 x 128 (BN below), 10 warps:
//   * thread 0 streams 64-wide K blocks of A_hi, A_lo (128 rows) and B_hi,
//     B_lo (BN rows, in 128-row boxes) with TMA (cp.async.bulk.tensor,
//     128-byte swizzle) into a ring of 2 (BN = 256) or 3 (BN = 128) stages
//     guarded by mbarriers, continuing across tiles;
//   * thread 32 issues tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulator
//     of 128 lanes x BN columns in tensor memory) into one of two
//     accumulators (2 BN TMEM columns), returns each stage to the producer
//     with tcgen05.commit and signals the finished accumulator;
//   * 8 epilogue warps drain the other accumulator meanwhile (tcgen05.ld
//     32x32b; a warp takes the lane quarter 32 (w % 4) .. +31 and one column
//     half), transpose 32 x 32 blocks through shared memory and run the
//     epilogue of the launch (plain store, or the two fused sweep epilogues of
//     the dense S-ADI step) with coalesced global accesses: 4-byte accesses
//     of 128-byte row segments, or, when every row of the launch's arrays
//     starts on a 16-byte boundary, 16-byte vectors (4 rows x 128 B per warp
//     access; a separate instantiation of the kernel).
// Problems of one launch may depend on earlier ones by 128-column panels (the
// two sweeps of the dense step: the y sweep reads the W that the x sweep
// stores): the last epilogue warp of a tile raises the panel counters of its
// columns after a GPU-scope fence, and the producer of a dependent tile waits
// (acquire) for its panels before its first copy.  All tiles of the earlier
// problems precede those of the later ones in every CTA's walk, and such a
// launch is cooperative, so every counter is raised by a resident CTA that
// never waits itself.
// A launch may be a programmatic dependent of the kernel before it
// (TcBatch::pdl): its CTAs set up barriers and tensor memory under that
// kernel's tail and wait for it (griddepcontrol.wait) before any other
// global access; the counters are then zeroed by that kernel.
// Every mbarrier and counter wait is bounded (1 s of %globaltimer, or the
// launch's TcBatch::wait_ns); on expiry the CTA sets *err, the other roles stop at their next wait, the
// producer waits (bounded) for the copies it issued, all MMAs are waited for,
// and the tensor memory is freed before the CTA returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

#include "../../include/sadi.h"
#include "bf16split.cuh"
#include "sadi_internal.h"

namespace sadi {
namespace {

constexpr int BM = kTcTileM, BK = kTcTileK;
constexpr int BOX = kTcBox;             // rows of every TMA box, A and B alike
constexpr int A_TILE = BM * BK * 2;     // 16 KB
constexpr int BOX_BYTES = BOX * BK * 2; // 16 KB

// What depends on the tile width BN (256 or 128 output columns): the B block of
// one stage, the stage bytes, the depth of the stage ring and the TMEM columns
// of one accumulator.  Both widths fill the same shared memory (2 x 96 KB or
// 3 x 64 KB of stages).
template <int BN>
struct TileCfg {
  static_assert(BN == 256 || BN == 128, "tile width");
  static constexpr int B_TILE = BN * BK * 2;
  static constexpr int STAGE_BYTES = 2 * A_TILE + 2 * B_TILE;
  static constexpr int STAGES = BN == 256 ? 2 : 3;
  static constexpr int TMEM_COLS = BN;
};
constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;   // default limit of every bounded wait

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait until the phase with the given parity has completed; false after limit ns.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_try(bar, parity))
    if (gtimer() - t0 > limit) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Pull one box of a tensor into L2 (no shared memory, no completion to wait
// for): the producer runs these some K blocks ahead of its loads, so that the
// loads of the ring find their operands in L2.
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 B, 8-row core groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);   // start address / 16
  d |= (uint64_t)1 << 16;                    // leading-dimension offset (unused when swizzled, K-major)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride-dimension offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                    // descriptor version of tcgen05
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major, N / 8 at bit 17, M / 16 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Epilogue of one 32 x 32 accumulator block: rows rowbase .. rowbase+31 (one
// per lane in r[], as tcgen05.ld delivers them), columns col0 .. col0+31.
// The block is transposed through the warp's padded shared tile so that every
// global access of the row-major arrays is a coalesced 128-byte row segment;
// loads of 8 rows are issued before any store (memory-level parallelism).
constexpr int EPI_LD = 33;
__device__ __forceinline__ void epilogue_block(const TcEpi& e, int rowbase, int col0, const uint32_t* r, float* tile,
                                               int lane) {
#pragma unroll
  for (int j = 0; j < 32; ++j) tile[lane * EPI_LD + j] = __uint_as_float(r[j]);
  __syncwarp();
  const int col = col0 + lane;
  const bool cok = col < e.n_valid;
  if (e.mode == kTcStore) {
#pragma unroll 4
    for (int rr = 0; rr < 32; ++rr) {
      const int row = rowbase + rr;
      if (row < e.m_valid && cok) e.C[(size_t)row * e.ldc + col] = tile[rr * EPI_LD + lane];
    }
  } else if (e.mode == kTcSweepX) {
    // W = B + B E (in place over B); all 32 rows of B loaded at once
    float wv[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int row = rowbase + q;
      wv[q] = (row < e.m_valid && cok) ? e.C[(size_t)row * e.ldc + col] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int row = rowbase + q;
      const float w = wv[q] + tile[q * EPI_LD + lane];
      tile[q * EPI_LD + lane] = w;
      if (row < e.m_valid && cok) e.C[(size_t)row * e.ldc + col] = w;
    }
    __syncwarp();
    // the transposed BF16 split of W (the y-sweep GEMM's B operand): lanes
    // 0-15 take the row pairs of column j, lanes 16-31 those of column j + 1,
    // one 4-byte store of two adjacent rows per lane.  Rows beyond m_valid
    // (padding up to the GEMM tile) hold W = 0 there (their B rows and
    // accumulator rows are zero), so the pairs are stored whole.
    const int p = lane & 15, jj = lane >> 4;
    const int row = rowbase + 2 * p;
#pragma unroll 4
    for (int j = 0; j < 32; j += 2) {
      const int cj = j + jj;
      if (col0 + cj < e.n_valid) {
        unsigned hi, lo;
        split_bf16x2(tile[(2 * p) * EPI_LD + cj], tile[(2 * p + 1) * EPI_LD + cj], &hi, &lo);
        const size_t t = (size_t)(col0 + cj) * e.ldt + row;
        *reinterpret_cast<unsigned*>(e.t_hi + t) = hi;
        *reinterpret_cast<unsigned*>(e.t_lo + t) = lo;
      }
    }
  } else {
    // uhat = W + E W; compensated leapfrog d^{n+1} = d^n + uhat (d^1 = uhat),
    // u^{n+1} = u^n + d^{n+1} with u = u_hi + u_lo (two-sum), in place.
    // Groups of 8 rows, the loads of the next group issued before the
    // current one is computed and stored (different rows: no overlap).
    float wv[2][8], dv[2][8], hv[2][8], lv[2][8];
#pragma unroll
    for (int gi = 0; gi <= 4; ++gi) {
      if (gi < 4) {
        const int nb = gi & 1;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int row = rowbase + 8 * gi + q;
          const bool ok = row < e.m_valid && cok;
          const size_t idx = (size_t)row * e.ldu + col;
          wv[nb][q] = ok ? e.C[(size_t)row * e.ldc + col] : 0.f;
          dv[nb][q] = (ok && !e.first) ? e.u_d[idx] : 0.f;
          hv[nb][q] = ok ? e.u_hi[idx] : 0.f;
          lv[nb][q] = ok ? e.u_lo[idx] : 0.f;
        }
      }
      if (gi > 0) {
        const int g = gi - 1, cb = g & 1;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int row = rowbase + 8 * g + q;
          if (row < e.m_valid && cok) {
            const float uh = wv[cb][q] + tile[(8 * g + q) * EPI_LD + lane];
            const float d = dv[cb][q] + uh;
            const float hi = hv[cb][q], lo = lv[cb][q];
            const float s = hi + d;
            const float bb = s - hi;
            const float err = (hi - (s - bb)) + (d - bb);
            const float l2 = lo + err;
            const float h2 = s + l2;
            const size_t idx = (size_t)row * e.ldu + col;
            e.u_hi[idx] = h2;
            e.u_lo[idx] = l2 - (h2 - s);
            e.u_d[idx] = d;
          }
        }
      }
    }
  }
  __syncwarp();
}

// The same epilogue with 16-byte accesses, for arrays whose rows start on
// 16-byte boundaries (TcEpi::vec).  The warp's tile holds the 32 x 32 block
// unpadded, in 4-float granules XOR-swizzled per row: element (r, c) sits at
// r * 32 + 4 * ((c / 4) ^ vsw(r)) + c % 4.  The swizzle makes the three
// access patterns free of bank conflicts: a lane's row of granules from
// tcgen05.ld (8 lanes of a phase: 8 rows, one granule each), the row-major
// vectors of the global arrays (8 lanes: one row, 8 granules) and the
// column reads of the transposed split (32 lanes: 8 columns x 4 row octets,
// vsw mixes the octet into the granule).
__device__ __forceinline__ int vsw(int r) { return (r ^ ((r >> 3) << 1)) & 7; }
__device__ __forceinline__ int vpos(int r, int g) { return r * 32 + ((g ^ vsw(r)) << 2); }

// a row segment of nv valid floats (0..4) starting at p: one 16-byte access
// when all four are valid
__device__ __forceinline__ float4 ld4(const float* p, int nv) {
  if (nv >= 4) return *reinterpret_cast<const float4*>(p);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (nv > 0) v.x = p[0];
  if (nv > 1) v.y = p[1];
  if (nv > 2) v.z = p[2];
  return v;
}
__device__ __forceinline__ void st4(float* p, float4 v, int nv) {
  if (nv >= 4) {
    *reinterpret_cast<float4*>(p) = v;
    return;
  }
  if (nv > 0) p[0] = v.x;
  if (nv > 1) p[1] = v.y;
  if (nv > 2) p[2] = v.z;
}

// one element of the compensated leapfrog: d^{n+1} = d^n + uhat and
// u^{n+1} = (hi + lo) + d^{n+1} by a two-sum, renormalised
__device__ __forceinline__ void leapfrog2(float uh, float dv, float hi, float lo, float* h_out, float* l_out,
                                          float* d_out) {
  const float d = dv + uh;
  const float s = hi + d;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (d - bb);
  const float l2 = lo + err;
  const float h2 = s + l2;
  *h_out = h2;
  *l_out = l2 - (h2 - s);
  *d_out = d;
}

__device__ __forceinline__ void epilogue_block_vec(const TcEpi& e, int rowbase, int col0, const uint32_t* r,
                                                   float* tile, int lane) {
#pragma unroll
  for (int g = 0; g < 8; ++g)
    *reinterpret_cast<float4*>(tile + vpos(lane, g)) =
        make_float4(__uint_as_float(r[4 * g]), __uint_as_float(r[4 * g + 1]), __uint_as_float(r[4 * g + 2]),
                    __uint_as_float(r[4 * g + 3]));
  __syncwarp();
  // lane -> row rr of each group of 4 rows (rows 4 i + rr, i = 0..7),
  // granule gg (columns col0 + 4 gg ..): a warp access covers 4 rows x 128 B
  const int rr = lane >> 3, gg = lane & 7;
  const int c4 = col0 + 4 * gg;
  const int ncol = min(max(e.n_valid - c4, 0), 4);
  auto nv_of = [&](int i) { return rowbase + 4 * i + rr < e.m_valid ? ncol : 0; };
  auto tile4 = [&](int i) -> float4* { return reinterpret_cast<float4*>(tile + vpos(4 * i + rr, gg)); };
  if (e.mode == kTcStore) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int nv = nv_of(i);
      if (nv) st4(e.C + (size_t)(rowbase + 4 * i + rr) * e.ldc + c4, *tile4(i), nv);
    }
  } else if (e.mode == kTcSweepX) {
    // W = B + B E (in place over B), then the transposed BF16 split of W
    float4 bv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int nv = nv_of(i);
      bv[i] = ld4(e.C + (size_t)(nv ? rowbase + 4 * i + rr : 0) * e.ldc + (nv ? c4 : 0), nv);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int nv = nv_of(i);
      float4* tp = tile4(i);
      const float4 a = *tp;
      const float4 w = make_float4(bv[i].x + a.x, bv[i].y + a.y, bv[i].z + a.z, bv[i].w + a.w);
      *tp = w;
      if (nv) st4(e.C + (size_t)(rowbase + 4 * i + rr) * e.ldc + c4, w, nv);
    }
    __syncwarp();
    // lane -> row octet oc (rows 8 oc .. 8 oc + 7), column cl of each group
    // of 8 columns: the octet as one 16-byte store each of hi and lo.  Rows
    // beyond m_valid (padding up to the GEMM tile) hold W = 0 there (their B
    // rows were loaded as 0 and their accumulator rows are zero), so the
    // octets are stored whole.
    const int oc = lane >> 3, cl = lane & 7;
#pragma unroll
    for (int jb = 0; jb < 4; ++jb) {
      const int c = 8 * jb + cl;
      if (col0 + c < e.n_valid) {
        unsigned hi[4], lo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int ra = 8 * oc + 2 * q;
          split_bf16x2(tile[vpos(ra, c >> 2) + (c & 3)], tile[vpos(ra + 1, c >> 2) + (c & 3)], &hi[q], &lo[q]);
        }
        const size_t t = (size_t)(col0 + c) * e.ldt + rowbase + 8 * oc;
        *reinterpret_cast<uint4*>(e.t_hi + t) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(e.t_lo + t) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
  } else {
    // uhat = W + E W; compensated leapfrog as in epilogue_block.  Four
    // groups of two row quads; the loads of the next group are issued
    // before the current one is computed and stored (different rows).
    float4 wv[2][2], dv[2][2], hv[2][2], lv[2][2];
#pragma unroll
    for (int gi = 0; gi <= 4; ++gi) {
      if (gi < 4) {
        const int nb = gi & 1;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int i = 2 * gi + q, nv = nv_of(i);
          const size_t rowc = (size_t)(nv ? rowbase + 4 * i + rr : 0), cc = nv ? c4 : 0;
          wv[nb][q] = ld4(e.C + rowc * e.ldc + cc, nv);
          dv[nb][q] = ld4(e.u_d + rowc * e.ldu + cc, e.first ? 0 : nv);
          hv[nb][q] = ld4(e.u_hi + rowc * e.ldu + cc, nv);
          lv[nb][q] = ld4(e.u_lo + rowc * e.ldu + cc, nv);
        }
      }
      if (gi > 0) {
        const int g = gi - 1, cb = g & 1;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int i = 2 * g + q, nv = nv_of(i);
          if (!nv) continue;
          const float4 a = *tile4(i);
          const float4 w = wv[cb][q], dd = dv[cb][q], hh = hv[cb][q], ll = lv[cb][q];
          float4 h, l, d;
          leapfrog2(w.x + a.x, dd.x, hh.x, ll.x, &h.x, &l.x, &d.x);
          leapfrog2(w.y + a.y, dd.y, hh.y, ll.y, &h.y, &l.y, &d.y);
          leapfrog2(w.z + a.z, dd.z, hh.z, ll.z, &h.z, &l.z, &d.z);
          leapfrog2(w.w + a.w, dd.w, hh.w, ll.w, &h.w, &l.w, &d.w);
          const size_t idx = (size_t)(rowbase + 4 * i + rr) * e.ldu + c4;
          st4(e.u_hi + idx, h, nv);
          st4(e.u_lo + idx, l, nv);
          st4(e.u_d + idx, d, nv);
        }
      }
    }
  }
  __syncwarp();
}

// Pull the global inputs of a warp's epilogue share into L2 while the tile's
// MMAs still run: the lane's row, columns c0 .. c0 + W - 1 (clipped to the
// valid columns) of each array the epilogue reads.  Only addresses of valid
// elements are named; one every 128 bytes plus the last covers every line.
__device__ __forceinline__ void prefetch_l2(const float* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
template <int W>
__device__ __forceinline__ void prefetch_row(const float* a, int ld, int row, int c0, int c1) {
  const float* p = a + (size_t)row * ld;
#pragma unroll
  for (int c = 0; c < W; c += 32)
    if (c0 + c < c1) prefetch_l2(p + c0 + c);
  prefetch_l2(p + c1 - 1);
}
template <int W>
__device__ __forceinline__ void prefetch_epilogue(const TcEpi& e, int row, int c0) {
  const int c1 = min(c0 + W, e.n_valid);
  if (row >= e.m_valid || c0 >= c1 || e.mode == kTcStore) return;
  prefetch_row<W>(e.C, e.ldc, row, c0, c1);
  if (e.mode == kTcSweepY) {
    prefetch_row<W>(e.u_hi, e.ldu, row, c0, c1);
    prefetch_row<W>(e.u_lo, e.ldu, row, c0, c1);
    if (!e.first) prefetch_row<W>(e.u_d, e.ldu, row, c0, c1);
  }
}

// Wait for a phase like mbar_wait, but give up at once when another role of
// the CTA has aborted, and abort the CTA when the time limit runs out.
__device__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort_flag, uint64_t limit) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (gtimer() - t0 > limit) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

// Bounded wait until *cnt >= need (acquire at GPU scope), for the order
// between problems of one launch; sets the abort flag when the time runs out.
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ bool wait_count(const int* cnt, int need, volatile int* abort_flag, uint64_t limit) {
  if (ld_acquire(cnt) >= need) return true;
  const uint64_t t0 = gtimer();
  while (ld_acquire(cnt) < need) {
    if (*abort_flag) return false;
    if (gtimer() - t0 > limit) {
      *abort_flag = 1;
      return false;
    }
    __nanosleep(128);
  }
  return true;
}
// Wait for every 128-column panel of the columns n0 .. n0 + BN - 1.
template <int BN>
__device__ bool wait_panels(const TcInst& in, int n0, volatile int* abort_flag, uint64_t limit) {
  for (int p = n0 / BOX; p < (n0 + BN) / BOX; ++p)
    if (!wait_count(in.dep_wait + p, in.dep_need, abort_flag, limit)) return false;
  return true;
}

// Tile t of the launch -> problem z and tile origin (m0, n0).  Tiles are
// numbered problem by problem; inside a problem in groups of kGroupM tile
// rows, column-major within a group, so that the tiles in flight at one time
// share A and B panels in L2.
constexpr int kGroupM = 32;
template <int BN>
__device__ __forceinline__ void tile_coords(const TcBatch& bt, int t, int* z, int* m0, int* n0) {
  constexpr int per = BN / BOX;   // B boxes per tile width
  int k = 0;
  for (; k < bt.count - 1; ++k) {
    const int nt = bt.in[k].tiles_m * (bt.in[k].boxes_n / per);
    if (t < nt) break;
    t -= nt;
  }
  const int tm = bt.in[k].tiles_m, tn = bt.in[k].boxes_n / per;
  const int per_group = kGroupM * tn;
  const int first_m = (t / per_group) * kGroupM;
  const int gsz = min(tm - first_m, kGroupM);
  const int local = t % per_group;
  *z = k;
  *m0 = (first_m + local % gsz) * BM;
  *n0 = (local / gsz) * BN;
}

// Persistent kernel: one CTA per SM walks the tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ...  Warp 0 (one thread) streams operand blocks by
// TMA through the stage ring, warp 1 (one thread) issues the MMAs into one
// of two TMEM accumulators (columns 0 .. BN-1 and BN .. 2BN-1) and signals tmem_full;
// warps 2-9 run the epilogue of the other accumulator meanwhile (two warps
// per TMEM lane quarter, one per column half) and free it through
// tmem_empty.  The ring and the accumulator pair carry over from tile to
// tile.
constexpr int EPI_WARPS = 8;
constexpr int TQ = 4;   // slots of the tile-index ring (the producer runs at most three tiles ahead)
constexpr int GEMM_THREADS = 64 + 32 * EPI_WARPS;
constexpr size_t EPI_BYTES = (size_t)EPI_WARPS * 32 * EPI_LD * sizeof(float);
template <int BN>
constexpr size_t psmem_bytes() {
  return (size_t)TileCfg<BN>::STAGES * TileCfg<BN>::STAGE_BYTES + EPI_BYTES + 1024 + 256;
}
static_assert(psmem_bytes<256>() <= 232448 && psmem_bytes<128>() <= 232448, "shared memory per CTA");

// VEC: every problem of the launch has TcEpi::vec set (16-byte epilogue
// accesses); the two epilogues are separate instantiations, so that neither
// carries the other's registers.
template <int BN, bool VEC>
__global__ void __launch_bounds__(GEMM_THREADS, 1) k_tc_gemm(const __grid_constant__ TcBatch bt, int total, int* err) {
  constexpr int STAGES = TileCfg<BN>::STAGES, STAGE_BYTES = TileCfg<BN>::STAGE_BYTES;
  constexpr int B_TILE = TileCfg<BN>::B_TILE, TMEM_COLS = TileCfg<BN>::TMEM_COLS;
  // K blocks prefetched into L2 beyond the ring, about 192 KB per SM, for the
  // wide tiles (large problems, operands far beyond L2); the narrow tiles of
  // small problems run without (measured slower with it at N = 1023)
  constexpr int PF_LEAD = BN == 256 ? 2 : 0;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* epi = reinterpret_cast<float*>(base + STAGES * STAGE_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES + EPI_BYTES);
  // bars: full[STAGES], empty[STAGES], tmem_full[2], tmem_empty[2], mma_done,
  // tile_full[TQ], tile_empty[TQ]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5 + 2 * TQ);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* epi_arrive = reinterpret_cast<int*>(tmem_slot + 2);   // per accumulator
  volatile int* tile_ring = reinterpret_cast<volatile int*>(tmem_slot + 4);   // TQ tile indices
  const uint32_t full0 = su32(bars), empty0 = su32(bars + STAGES);
  const uint32_t tfull0 = su32(bars + 2 * STAGES), tempty0 = su32(bars + 2 * STAGES + 2);
  const uint32_t mdone = su32(bars + 2 * STAGES + 4);
  const uint32_t qfull0 = su32(bars + 2 * STAGES + 5), qempty0 = su32(bars + 2 * STAGES + 5 + TQ);
  // Dynamic tile order (narrow tiles with a tile counter): the producer takes
  // the next tile from the launch's counter and passes its index to the MMA
  // thread and the epilogue warps through tile_ring (slot tl % TQ for the
  // CTA's tl-th tile, -1 when there are no more), guarded by tile_full (the
  // producer's arrival) and tile_empty (the MMA thread and every epilogue warp
  // have read it).  Otherwise the static order blockIdx.x + tl * gridDim.x.
  int* const tile_next = BN == 128 ? bt.tile_next : nullptr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t limit = bt.wait_ns ? bt.wait_ns : WAIT_LIMIT_NS;
  // the next step's first kernel (a programmatic dependent) may be scheduled
  // onto SMs as these CTAs exit; it waits for this grid before reading
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, EPI_WARPS);
    }
    mbar_init(mdone, 1);
    for (int q = 0; q < TQ; ++q) {
      mbar_init(qfull0 + 8 * q, 1);
      mbar_init(qempty0 + 8 * q, 1 + EPI_WARPS);
    }
    *abort_flag = 0;
    epi_arrive[0] = epi_arrive[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(2 * TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // launched as a programmatic dependent, the set-up above ran under the
  // kernel before this one; wait for it (its outputs are this launch's
  // operands, and it zeroed the counters) before any global access.
  // Launched without that attribute this is a no-op.
  asm volatile("griddepcontrol.wait;" ::: "memory");

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer ----
      // L2 prefetch cursor (tile pt, K block pkb; sequence number pseq): it
      // runs PF_LEAD K blocks beyond the ring, which the loads fill
      int pt = blockIdx.x, pkb = 0, pseq = 0;
      auto prefetch_upto = [&](int seq_end) {
        while (pseq < seq_end && pt < total) {
          int pz, pm0, pn0;
          tile_coords<BN>(bt, pt, &pz, &pm0, &pn0);
          const TcInst& pin = bt.in[pz];
          if (pseq >= STAGES) {   // the first ring fill is loaded at once
            tma_prefetch_2d(&pin.a_hi, pkb * BK, pm0);
            tma_prefetch_2d(&pin.a_lo, pkb * BK, pm0);
#pragma unroll
            for (int j = 0; j < BN / BOX; ++j) {
              tma_prefetch_2d(&pin.b_hi, pkb * BK, pn0 + j * BOX);
              tma_prefetch_2d(&pin.b_lo, pkb * BK, pn0 + j * BOX);
            }
          }
          ++pseq;
          if (++pkb == pin.K / BK) {
            pkb = 0;
            pt += gridDim.x;
          }
        }
      };
      int it = 0;
      for (int tl = 0; !*abort_flag; ++tl) {
        // the next tile: publish its index (or -1) in the ring for the others
        const int q = tl % TQ;
        if (tl >= TQ && !wait_or_abort(qempty0 + 8 * q, (uint32_t)(tl / TQ - 1) & 1u, abort_flag, limit)) break;
        int t = tile_next ? atomicAdd(tile_next, 1) : blockIdx.x + tl * gridDim.x;
        if (t >= total) t = -1;
        tile_ring[q] = t;
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(qfull0 + 8 * q) : "memory");
        if (t < 0) break;
        int z, m0, n0;
        tile_coords<BN>(bt, t, &z, &m0, &n0);
        const TcInst& in = bt.in[z];
        const int nk = in.K / BK;
        if (in.dep_wait) {
          // the B rows are written by an earlier problem of this launch with
          // generic stores: acquire them, then order them before the copies
          if (!wait_panels<BN>(in, n0, abort_flag, limit)) break;
          asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t use = (uint32_t)(it / STAGES);
          if constexpr (PF_LEAD > 0) prefetch_upto(it + STAGES + PF_LEAD);
          if (it >= STAGES && !wait_or_abort(empty0 + 8 * s, (use - 1) & 1u, abort_flag, limit)) break;
          uint8_t* st = base + s * STAGE_BYTES;
          mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
          tma_load_2d(su32(st), &in.a_hi, kb * BK, m0, full0 + 8 * s);
          tma_load_2d(su32(st + A_TILE), &in.a_lo, kb * BK, m0, full0 + 8 * s);
#pragma unroll
          for (int j = 0; j < BN / BOX; ++j) {
            // 128-row boxes stacked in 16 KB steps continue the 8-row, 1024 B
            // pattern of the swizzled layout
            tma_load_2d(su32(st + 2 * A_TILE + j * BOX_BYTES), &in.b_hi, kb * BK, n0 + j * BOX, full0 + 8 * s);
            tma_load_2d(su32(st + 2 * A_TILE + B_TILE + j * BOX_BYTES), &in.b_lo, kb * BK, n0 + j * BOX,
                        full0 + 8 * s);
          }
        }
      }
      if (*abort_flag) {
        // the copies issued last must land before the CTA may exit
        for (int j = (it > STAGES ? it - STAGES : 0); j < it; ++j)
          (void)mbar_wait(full0 + 8 * (j % STAGES), (uint32_t)(j / STAGES) & 1u, limit);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      int it = 0;
      for (int tl = 0; !*abort_flag; ++tl) {
        const int q = tl % TQ;
        if (!wait_or_abort(qfull0 + 8 * q, (uint32_t)(tl / TQ) & 1u, abort_flag, limit)) break;
        const int t = tile_ring[q];
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(qempty0 + 8 * q) : "memory");
        if (t < 0) break;
        int z, m0, n0;
        tile_coords<BN>(bt, t, &z, &m0, &n0);
        const int nk = bt.in[z].K / BK;
        const int b = tl & 1;
        const uint32_t ub = (uint32_t)(tl >> 1);
        if (tl >= 2 && !wait_or_abort(tempty0 + 8 * b, (ub - 1) & 1u, abort_flag, limit)) break;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * TMEM_COLS);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % STAGES;
          if (!wait_or_abort(full0 + 8 * s, (uint32_t)(it / STAGES) & 1u, abort_flag, limit)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = su32(base + s * STAGE_BYTES);
          const uint64_t a_hi = sw128_desc(st), a_lo = sw128_desc(st + A_TILE);
          const uint64_t b_hi = sw128_desc(st + 2 * A_TILE), b_lo = sw128_desc(st + 2 * A_TILE + B_TILE);
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            const uint64_t a = (p < 2) ? a_hi : a_lo;
            const uint64_t bb = (p == 1) ? b_lo : b_hi;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)
              mma_bf16(acc, a + (uint64_t)(2 * k), bb + (uint64_t)(2 * k), idesc, (kb | p | k) != 0 ? 1u : 0u);
          }
          mma_commit(empty0 + 8 * s);
        }
        mma_commit(tfull0 + 8 * b);
        if (!ok) break;
      }
      // every MMA issued must have finished before the tensor memory is freed
      mma_commit(mdone);
      (void)mbar_wait(mdone, 0, limit);
    }
  } else {
    // ---- epilogue warps: TMEM lane quarter = warp % 4, column half ----
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    float* tile = epi + (warp - 2) * 32 * EPI_LD;
    for (int tl = 0;; ++tl) {
      const int q = tl % TQ;
      if (!wait_or_abort(qfull0 + 8 * q, (uint32_t)(tl / TQ) & 1u, abort_flag, limit)) break;
      const int t = tile_ring[q];
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(qempty0 + 8 * q) : "memory");
      if (t < 0) break;
      int z, m0, n0;
      tile_coords<BN>(bt, t, &z, &m0, &n0);
      const int b = tl & 1;
      const uint32_t ub = (uint32_t)(tl >> 1);
      const TcInst& in = bt.in[z];
      prefetch_epilogue<BN / 2>(in.e, m0 + quarter * 32 + lane, n0 + half * (BN / 2));
      if (!wait_or_abort(tfull0 + 8 * b, ub & 1u, abort_flag, limit) || *abort_flag) break;
      tc_fence_after();
      if (in.dep_wait) {
        // the epilogue reads W of the same panels (already complete: the
        // producer waited for them before this tile's loads)
        bool ok = true;
        if (lane == 0) ok = wait_panels<BN>(in, n0, abort_flag, limit);
        if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
      }
      const uint32_t acc = tmem + (uint32_t)(b * TMEM_COLS) + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int c = 0; c < BN / 64; ++c) {
        const int cc = half * (BN / 64) + c;
        uint32_t r[32];
        tmem_ld32(acc + (uint32_t)(cc * 32), r);
        if constexpr (VEC)
          epilogue_block_vec(in.e, m0 + quarter * 32, n0 + cc * 32, r, tile, lane);
        else
          epilogue_block(in.e, m0 + quarter * 32, n0 + cc * 32, r, tile, lane);
      }
      if (in.dep_signal) {
        // publish the tile: every warp's stores, then the last of the
        // EPI_WARPS warps (arrival count modulo EPI_WARPS per accumulator;
        // the accumulator is freed only after this, so uses do not overlap)
        // releases the panel counters
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __threadfence();
        __syncwarp();
        if (lane == 0) {
          const int old = atomicAdd(&epi_arrive[b], 1);
          if (old % EPI_WARPS == EPI_WARPS - 1) {
            __threadfence();
            for (int p = n0 / BOX; p < (n0 + BN) / BOX; ++p) atomicAdd(in.dep_signal + p, 1);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8 * b) : "memory");
    }
  }
  __syncwarp();
  if (*abort_flag && threadIdx.x == 64) {
    int z, m0, n0;
    tile_coords<BN>(bt, blockIdx.x, &z, &m0, &n0);
    atomicExch(bt.in[z].e.err ? bt.in[z].e.err : err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TMEM_COLS) : "memory");
  }
}

// FP32 (rows x cols, row-major, ld src_ld) -> BF16 hi/lo pair in a zero-padded
// prow x pcol buffer.
__global__ void k_split_pad(const float* __restrict__ src, int rows, int cols, int src_ld, unsigned short* hi,
                            unsigned short* lo, int prow, int pcol) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)prow * pcol) return;
  const int r = (int)(idx / pcol), c = (int)(idx % pcol);
  const float v = (r < rows && c < cols) ? src[(size_t)r * src_ld + c] : 0.f;
  split_bf16(v, hi + idx, lo + idx);
}

CUresult (*g_encode)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                     const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                     CUtensorMapL2promotion, CUtensorMapFloatOOBfill) = nullptr;

// Looked up once per process; the static's initialisation is thread-safe.
cudaError_t get_encoder() {
  static const cudaError_t status = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<decltype(g_encode)>(fn);
    return cudaSuccess;
  }();
  return status;
}

}  // namespace

cudaError_t tc_encode(CUtensorMap* map, const void* base, int rows, int kdim, int box_rows) {
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  // TMA needs a 16-byte aligned base and a row pitch that is a multiple of 16 B
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (kdim % 8) || kdim % BK || rows % box_rows)
    return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)kdim, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kdim * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_set_operands(TcInst* in, const void* a_hi, const void* a_lo, const void* b_hi, const void* b_lo,
                            int M, int N, int K) {
  cudaError_t e;
  if ((e = tc_encode(&in->a_hi, a_hi, M, K, BM))) return e;
  if ((e = tc_encode(&in->a_lo, a_lo, M, K, BM))) return e;
  if ((e = tc_encode(&in->b_hi, b_hi, N, K, BOX))) return e;
  if ((e = tc_encode(&in->b_lo, b_lo, N, K, BOX))) return e;
  if (M % BM || N % BOX || K % BK || K <= 0) return cudaErrorInvalidValue;
  in->K = K;
  in->tiles_m = M / BM;
  in->boxes_n = N / BOX;
  return cudaSuccess;
}

cudaError_t launch_tc_gemm(const TcBatch& b, int* err, cudaStream_t st) {
  if (b.count < 1 || b.count > kTcMaxBatch) return cudaErrorInvalidValue;
  int boxes = 0;
  bool even = true, vec = true;
  for (int k = 0; k < b.count; ++k) {
    const TcInst& in = b.in[k];
    if (in.K <= 0 || in.K % BK || in.tiles_m < 1 || in.boxes_n < 1) return cudaErrorInvalidValue;
    boxes += in.tiles_m * in.boxes_n;
    even = even && in.boxes_n % 2 == 0;
    vec = vec && in.e.vec;
  }
  static LaunchCache sms_of[kLauncherDevices];
  const int dev = device_slot();
  if (dev < 0) return cudaErrorInvalidDevice;
  int sms = sms_of[dev].load(std::memory_order_acquire);
  if (!sms) {
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tc_gemm<256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)psmem_bytes<256>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tc_gemm<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)psmem_bytes<256>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tc_gemm<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)psmem_bytes<128>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tc_gemm<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)psmem_bytes<128>());
    if (e != cudaSuccess) return e;
    sms_of[dev].store(sms, std::memory_order_release);
  }
  // 128 x 256 tiles (fewer operand bytes per flop) once they give every SM
  // two or more; below that the 128 x 128 tiles balance better (measured:
  // three N = 1023 problems per launch run faster as 192 narrow tiles than
  // as 96 wide ones), and a CTA with several runs the epilogue of one under
  // the MMAs of the next
  // tiles of a waiting problem spin on counters that other CTAs raise, so
  // all CTAs must be resident together: a cooperative launch (grid <= SMs,
  // one CTA per SM by its shared memory)
  bool coop = false;
  for (int k = 0; k < b.count; ++k) coop = coop || b.in[k].dep_wait;
  cudaLaunchAttribute attr[2];
  int nattr = 0;
  if (coop) {
    attr[nattr].id = cudaLaunchAttributeCooperative;
    attr[nattr].val.cooperative = 1;
    ++nattr;
  }
  if (b.pdl) {
    attr[nattr].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[nattr].val.programmaticStreamSerializationAllowed = 1;
    ++nattr;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(GEMM_THREADS);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = nattr;
  if (even && boxes / 2 >= 2 * sms) {
    const int total = boxes / 2;
    cfg.gridDim = dim3(sms);
    cfg.dynamicSmemBytes = psmem_bytes<256>();
    return vec ? cudaLaunchKernelEx(&cfg, k_tc_gemm<256, true>, b, total, err)
               : cudaLaunchKernelEx(&cfg, k_tc_gemm<256, false>, b, total, err);
  }
  const int total = boxes;
  cfg.gridDim = dim3(total < sms ? total : sms);
  cfg.dynamicSmemBytes = psmem_bytes<128>();
  return vec ? cudaLaunchKernelEx(&cfg, k_tc_gemm<128, true>, b, total, err)
             : cudaLaunchKernelEx(&cfg, k_tc_gemm<128, false>, b, total, err);
}

cudaError_t launch_split_pad(const float* src, int rows, int cols, int src_ld, void* hi, void* lo, int prow, int pcol,
                             cudaStream_t st) {
  const size_t n = (size_t)prow * pcol;
  if (n == 0) return cudaSuccess;
  k_split_pad<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, rows, cols, src_ld, static_cast<unsigned short*>(hi),
                                                            static_cast<unsigned short*>(lo), prow, pcol);
  return cudaGetLastError();
}

}  // namespace sadi

// ---- diagnostic entry point ---------------------------------------------------

using namespace sadi;

namespace {
int round_up(int v, int m) { return (v + m - 1) / m * m; }
}  // namespace

extern "C" sadi_status sadi_gemm_split_bf16(const float* A, const float* B, float* C, int M, int N, int K,
                                            void* stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || M > 65536 || N > 65536 || K > 65536) return SADI_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int Mp = round_up(M, BM), Np = round_up(N, kTcTileN), Kp = round_up(K, BK);
  unsigned short* buf = nullptr;
  int* err = nullptr;
  const size_t na = (size_t)Mp * Kp, nb = (size_t)Np * Kp;
  if (cudaMalloc(&buf, (2 * na + 2 * nb) * sizeof(unsigned short)) != cudaSuccess) return SADI_ENOMEM;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaFree(buf);
    return SADI_ENOMEM;
  }
  unsigned short *ah = buf, *al = buf + na, *bh = buf + 2 * na, *bl = buf + 2 * na + nb;
  static thread_local TcBatch bt;   // about 1.2 KB of tensor maps; built on the host only
  std::memset(&bt, 0, sizeof(bt));
  bt.count = 1;
  TcEpi& e = bt.in[0].e;
  e.mode = kTcStore;
  e.m_valid = M;
  e.n_valid = N;
  e.C = C;
  e.ldc = N;
  e.vec = tc_vec_ok(e) ? 1 : 0;
  sadi_status rs = SADI_OK;
  int herr = 0;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
      launch_split_pad(A, M, K, K, ah, al, Mp, Kp, st) != cudaSuccess ||
      launch_split_pad(B, N, K, K, bh, bl, Np, Kp, st) != cudaSuccess ||
      tc_set_operands(&bt.in[0], ah, al, bh, bl, Mp, Np, Kp) != cudaSuccess ||
      launch_tc_gemm(bt, err, st) != cudaSuccess ||
      cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    rs = SADI_ECUDA;
  } else if (herr) {
    rs = SADI_ETIMEOUT;
  }
  cudaFree(buf);
  cudaFree(err);
  return rs;
}
