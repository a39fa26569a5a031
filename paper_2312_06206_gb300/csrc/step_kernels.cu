// step_kernels.cu -- the per-time-step hot path of the S-ADI scheme
// (arXiv 2312.06206, Sec. 3, eq. "ADI scheme equivalent"):
//
//   B^n  = -tau^2 kappa L_h u^n + tau^2 g(u^n)            (n >= 1)
//        = tau phi2 + 1/2 (-tau^2 kappa L_h u^0 + tau^2 g(u^0))   (n = 0)
//   W    = B H^-1      (x sweep: H w = b on every grid row)
//   uhat = H^-1 W      (y sweep: on every grid column)
//   u^{n+1} = 2u^n - u^{n-1} + uhat   (n >= 1),   u^1 = u^0 + uhat   (n = 0)
//
// L_h u^n is the block-Toeplitz-Toeplitz-block product of Sec. 3, applied by
// the 2Np x 2Np block-circulant embedding and 2D FFTs.  Each H^-1 v is the
// Gohberg-Semencul formula (Proposition 1) evaluated by Algorithm 1 on the
// bordered Toeplitz matrix H' (size Np = power of two) followed by a rank-r
// correction (r = Np - N) that recovers H^-1 exactly.
//
// Kernels per step, all FFTs of the single length Np in shared memory:
//   k_rows_r2c   rows of u^n -> half spectrum along x (real FFT of length 2Np)
//   k_cols_conv  per x frequency: FFT along y, x symbol, inverse FFT along y
//                (FP32 at Np = 8192: the three passes of conv3.cu instead)
//   k_rows_solve inverse real FFT along x + B^n epilogue + x sweep (Algorithm 1)
//   k_cols_solve y sweep (Algorithm 1) + leapfrog epilogue (FP64); the FP32
//                forms run it on the transpose: k_transpose_f32, k_rows_gs,
//                k_transpose_leapfrog
#include <cuda_runtime.h>

#include "fft.cuh"
#include "bf16split.cuh"
#include "sadi_internal.h"

namespace sadi {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxPairs = 16;

// the general nonlinearity out of line: the row kernels' epilogues inline
// g many times over, and only launches with g kind 3 take this call
template <typename T>
__device__ __noinline__ T g_general(T u, T c1, T c3, T cs) {
  return (c1 + c3 * u * u) * u + cs * sin(u);
}
template <typename T>
__device__ __forceinline__ T g_of(const RhsParams& rp, T u) {
  if (rp.g == 1) return -u * u * u;
  if (rp.g == 2) return -sin(u);
  if (rp.g == 3) return g_general<T>(u, T(rp.gc1), T(rp.gc3), T(rp.gcs));
  return T(0);
}

// u^{n+1} = u^n + d^{n+1}, d^{n+1} = d^n + uhat, with u a double-float pair
// (hi = uc, lo); two-sum and fast-two-sum keep the rounding of the sum in lo.
template <typename T>
__device__ __forceinline__ void leapfrog_comp(T hi, T uh, int first, size_t idx, T* dbuf, T* hibuf, T* lobuf) {
  const T d = first ? uh : dbuf[idx] + uh;
  const T lo = lobuf[idx];
  const T s = hi + d;
  const T bb = s - hi;
  const T err = (hi - (s - bb)) + (d - bb);
  const T l2 = lo + err;
  const T h2 = s + l2;
  const T lo2 = l2 - (h2 - s);
  hibuf[idx] = h2;
  lobuf[idx] = lo2;
  dbuf[idx] = d;
}

template <typename T>
__device__ __forceinline__ T real_view(const cx<T>* v, int k) {
  const T* f = reinterpret_cast<const T*>(v + sidx<T>(k >> 1));
  return f[k & 1];
}

// Incremental remainder of the FP32 forms: C = -kappa tau^2 L_h u^n is kept
// as a double-float pair (Ch + Cl) and advanced by the convolution of the
// increment d^n = u^n - u^{n-1} (two-sum); returns the new Ch.
template <typename T>
__device__ __forceinline__ T acc_remainder(float* Ch, float* Cl, size_t idx, T conv) {
  const float hi = Ch[idx], lo = Cl[idx];
  const float x = (float)conv;
  const float s = hi + x;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (x - bb);
  const float l2 = lo + err;
  const float h2 = s + l2;
  Ch[idx] = h2;
  Cl[idx] = l2 - (h2 - s);
  return T(h2);
}

// ---------------------------------------------------------------------------
// Gohberg-Semencul core, Algorithm 1 on the bordered matrix H':
// input  buf[v] = Q v1 with v1 = (v' + i J v') (natural order),
// output buf[v] = vhat (natural order); H'^-1 v' = Re vhat + J Im vhat.
// lam_s, lam_c carry 1/Np and 1/(2 p1 Np); Q = diag(exp(-i pi k / Np)).
// ---------------------------------------------------------------------------
template <typename T>
__device__ void gs_core(cx<T>* buf, int nvec, int vs, const Geom& g, const cx<T>* __restrict__ stw,
                        const cx<T>* __restrict__ tw, const cx<T>* __restrict__ lam_s,
                        const cx<T>* __restrict__ lam_c) {
  const int Np = g.Np, logNp = g.logNp;
  const int ns = plan_stages(logNp);
  if (ns >= 2) {
    dif_stages<T>(buf, logNp, nvec, vs, stw, 0, ns - 1);
    fused8<T>(buf, logNp, nvec, vs, lam_s, 0);           // x lambda_s between DIF and DIT
    dit_stages<T>(buf, logNp, nvec, vs, stw, 1, ns - 1);
    fusedL<T>(buf, logNp, nvec, vs, stw, tw);             // Q^H between DIT and DIF
    dif_stages<T>(buf, logNp, nvec, vs, stw, 1, ns - 1);
    fused8<T>(buf, logNp, nvec, vs, lam_c, 0);            // x lambda_c between DIF and DIT
    dit_stages<T>(buf, logNp, nvec, vs, stw, 0, ns - 1);
    return;
  }
  fft_dif<T>(buf, logNp, nvec, vs, stw);
  for (int t = threadIdx.x; t < (nvec << logNp); t += blockDim.x) {
    const int v = t >> logNp, p = t & (Np - 1);
    cx<T>* e = buf + v * vs + sidx<T>(p);
    *e = cmul(*e, __ldg(&lam_s[p]));
  }
  __syncthreads();
  fft_dit<T>(buf, logNp, nvec, vs, stw);
  for (int t = threadIdx.x; t < (nvec << logNp); t += blockDim.x) {
    const int v = t >> logNp, k = t & (Np - 1);
    cx<T>* e = buf + v * vs + sidx<T>(k);
    *e = cmulc(*e, __ldg(&tw[k]));       // Q^H
  }
  __syncthreads();
  fft_dif<T>(buf, logNp, nvec, vs, stw);
  for (int t = threadIdx.x; t < (nvec << logNp); t += blockDim.x) {
    const int v = t >> logNp, p = t & (Np - 1);
    cx<T>* e = buf + v * vs + sidx<T>(p);
    *e = cmul(*e, __ldg(&lam_c[p]));
  }
  __syncthreads();
  fft_dit<T>(buf, logNp, nvec, vs, stw);
}

// (H^-1 v)[k] for k < N from vhat: Re vhat[k] + Im vhat[Np-1-k] plus the
// border correction sum_q G[k, q] ybot[q], ybot[q] = (H'^-1 v')[N + q].
template <typename T>
__device__ __forceinline__ T gs_out(const cx<T>* vh, int k, const Geom& g, const T* __restrict__ G) {
  T y = vh[sidx<T>(k)].x + vh[sidx<T>(g.Np - 1 - k)].y;
  for (int q = 0; q < g.r; ++q) {
    const int kb = g.N + q;
    const T yb = vh[sidx<T>(kb)].x + vh[sidx<T>(g.Np - 1 - kb)].y;
    y += __ldg(&G[(size_t)k * g.r + q]) * yb;
  }
  return y;
}

// ---------------------------------------------------------------------------
// k_rows_r2c: rows j of u -> S[j][slot], the DFT of the row zero-padded to
// length P = 2Np, via a complex FFT of length Np of z[n] = x[2n] + i x[2n+1].
// Slot s >= 1 holds X[brev(s)]; slot 0 holds X[0] + i X[Np] (both real).
// ---------------------------------------------------------------------------
// With u2 (the diffusion step, FP64) the transformed rows are those of
// u + beta (u - u2): the extrapolation u~ = u^n + (u^n - u^{n-1})/2; EXTRAP
// selects that form at compile time (the other launches carry none of it).
template <typename T, bool EXTRAP = false>
__global__ void __launch_bounds__(kThreads)
k_rows_r2c(const T* __restrict__ u, cx<T>* __restrict__ S, Geom g, const cx<T>* __restrict__ stw,
           const cx<T>* __restrict__ tw, int NR, const T* __restrict__ u2 = nullptr, T beta = T(0)) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const int N = g.N, Np = g.Np, logNp = g.logNp;
  const int vs = vstride<T>(Np);
  const int row0 = blockIdx.x * NR;
  const int nrows = min(NR, N - row0);
  for (int t = threadIdx.x; t < (NR << logNp); t += blockDim.x) {
    const int v = t >> logNp, n = t & (Np - 1);
    T a = T(0), b = T(0);
    if (v < nrows) {
      const T* row = u + (size_t)(row0 + v) * N;
      if (2 * n < N) a = row[2 * n];
      if (2 * n + 1 < N) b = row[2 * n + 1];
      if constexpr (EXTRAP) {
        const T* row2 = u2 + (size_t)(row0 + v) * N;
        if (2 * n < N) a += beta * (a - row2[2 * n]);
        if (2 * n + 1 < N) b += beta * (b - row2[2 * n + 1]);
      }
    }
    buf[v * vs + sidx<T>(n)] = mkc(a, b);
  }
  __syncthreads();
  fft_dif<T>(buf, logNp, NR, vs, stw);
  const T half = T(0.5);
  for (int t = threadIdx.x; t < (nrows << logNp); t += blockDim.x) {
    const int v = t >> logNp, s = t & (Np - 1);
    const int k = brev(s, logNp);
    const int sp = brev((Np - k) & (Np - 1), logNp);
    const cx<T> Z = buf[v * vs + sidx<T>(s)];
    const cx<T> Zc = cconj(buf[v * vs + sidx<T>(sp)]);
    const cx<T> E = cscale(cadd(Z, Zc), half);
    const cx<T> O = cscale(cmul_mi(csub(Z, Zc)), half);   // (Z - Zc) / (2i)
    cx<T> X;
    if (s == 0) X = mkc(E.x + O.x, E.x - O.x);
    else X = cadd(E, cmul(__ldg(&tw[k]), O));
    S[(size_t)(row0 + v) * Np + s] = X;
  }
}

// ---------------------------------------------------------------------------
// k_cols_conv: for each slot (x frequency k1) the column over j is convolved
// along y with the symbol: FFT of length P (N nonzero inputs) split into its
// even and odd frequency halves (two FFTs of length Np), multiply by the
// symbol, inverse, keep rows j < N.  Slot 0 holds two real columns (k1 = 0
// and k1 = Np) packed as re + i im: they are separated with the partner
// bin Y[-k] (Ev = (Y[k] + conj Y[-k]) / 2, Od = (Y[k] - conj Y[-k]) / 2) and
// each multiplied by its own symbol, L0 Ev + LN Od.  In place on S.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_cols_conv(cx<T>* __restrict__ S, Geom g, const cx<T>* __restrict__ stw, const cx<T>* __restrict__ tw,
            const T* __restrict__ lpb, int CT) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const int N = g.N, Np = g.Np, logNp = g.logNp;
  const int vs = vstride<T>(Np);
  const int s0 = blockIdx.x * CT;
  for (int t = threadIdx.x; t < CT * Np; t += blockDim.x) {
    const int c = t % CT, j = t / CT;
    cx<T> val = mkc(T(0), T(0));
    if (j < N) val = S[(size_t)j * Np + s0 + c];
    buf[(2 * c) * vs + sidx<T>(j)] = val;
    buf[(2 * c + 1) * vs + sidx<T>(j)] = cmul(val, __ldg(&tw[j]));
  }
  __syncthreads();
  const int ns = plan_stages(logNp);
  if (s0 != 0 && ns >= 2) {
    // symbol multiply fused between the forward and the inverse transform
    dif_stages<T>(buf, logNp, 2 * CT, vs, stw, 0, ns - 1);
    fused8<T>(buf, logNp, 2 * CT, vs, lpb + (size_t)s0 * 2 * Np, Np);
    dit_stages<T>(buf, logNp, 2 * CT, vs, stw, 0, ns - 1);
  } else {
    fft_dif<T>(buf, logNp, 2 * CT, vs, stw);
    for (int t = threadIdx.x; t < ((2 * CT) << logNp); t += blockDim.x) {
      const int vec = t >> logNp, p = t & (Np - 1);
      const int slot = s0 + (vec >> 1), h = vec & 1;
      if (slot == 0) continue;
      cx<T>* e = buf + vec * vs + sidx<T>(p);
      *e = cscale(*e, __ldg(&lpb[((size_t)slot * 2 + h) * Np + p]));
    }
    if (s0 == 0) {
      // slot 0: pairs (p, partner) in each half, handled by one thread each.
      const T half = T(0.5);
      for (int t = threadIdx.x; t < 2 * Np; t += blockDim.x) {
        const int h = t >> logNp, p = t & (Np - 1);
        const int pp = (h == 0) ? brev((Np - brev(p, logNp)) & (Np - 1), logNp) : (Np - 1 - p);
        if (pp < p) continue;
        cx<T>* e = buf + h * vs;
        const cx<T> Y = e[sidx<T>(p)], Yp = e[sidx<T>(pp)];
        // unpack the two real columns first: Ev = spectrum of the k1 = 0
        // column, Od = i x spectrum of the k1 = Np column; each then takes its
        // own symbol (no cancellation between the large k1 = Np symbol and
        // the small low-frequency k1 = 0 symbol)
        const cx<T> Ev = cscale(cadd(Y, cconj(Yp)), half);
        const cx<T> Od = cscale(csub(Y, cconj(Yp)), half);
        const T L0 = __ldg(&lpb[(size_t)h * Np + p]);
        const T LN = __ldg(&lpb[((size_t)Np * 2 + h) * Np + p]);
        e[sidx<T>(p)] = cadd(cscale(Ev, L0), cscale(Od, LN));
        if (pp != p) {
          const T L0p = __ldg(&lpb[(size_t)h * Np + pp]);
          const T LNp = __ldg(&lpb[((size_t)Np * 2 + h) * Np + pp]);
          e[sidx<T>(pp)] = csub(cscale(cconj(Ev), L0p), cscale(cconj(Od), LNp));
        }
      }
    }
    __syncthreads();
    fft_dit<T>(buf, logNp, 2 * CT, vs, stw);
  }
  for (int t = threadIdx.x; t < CT * N; t += blockDim.x) {
    const int c = t % CT, j = t / CT;
    const cx<T> ye = buf[(2 * c) * vs + sidx<T>(j)];
    const cx<T> yo = buf[(2 * c + 1) * vs + sidx<T>(j)];
    S[(size_t)j * Np + s0 + c] = cadd(ye, cmulc(yo, __ldg(&tw[j])));
  }
}

// Rows row0 .. row0+nrows-1 of the convolved half spectrum S -> buf (real
// view: the inverse real FFT of length 2Np, i.e. the convolution values at
// x indices 0 .. 2Np-1): half spectrum X[k] (slots) -> Z[k] = E + iO, the
// spectrum of z[n] = x[2n] + i x[2n+1], then an inverse complex FFT.
template <typename T>
__device__ __forceinline__ void rows_inverse(cx<T>* buf, const cx<T>* __restrict__ S, const Geom& g, int NR, int row0,
                                             int nrows, int vs, const cx<T>* __restrict__ stw,
                                             const cx<T>* __restrict__ tw) {
  const int Np = g.Np, logNp = g.logNp;
  for (int t = threadIdx.x; t < (NR << logNp); t += blockDim.x) {
    const int v = t >> logNp, s = t & (Np - 1);
    cx<T> val = mkc(T(0), T(0));
    if (v < nrows) val = S[(size_t)(row0 + v) * Np + s];
    buf[v * vs + sidx<T>(s)] = val;
  }
  __syncthreads();
  // each thread owns a partner pair of slots
  const T half = T(0.5);
  for (int t = threadIdx.x; t < (NR << logNp); t += blockDim.x) {
    const int v = t >> logNp, s = t & (Np - 1);
    const int k = brev(s, logNp);
    const int kp = (Np - k) & (Np - 1);
    const int sp = brev(kp, logNp);
    if (sp < s) continue;
    cx<T>* e = buf + v * vs;
    const cx<T> X = e[sidx<T>(s)];
    if (s == 0) {
      e[sidx<T>(0)] = mkc((X.x + X.y) * half, (X.x - X.y) * half);
      continue;
    }
    const cx<T> Xp = e[sidx<T>(sp)];
    {
      const cx<T> E = cscale(cadd(X, cconj(Xp)), half);
      const cx<T> O = cscale(cmulc(csub(X, cconj(Xp)), __ldg(&tw[k])), half);
      e[sidx<T>(s)] = cadd(E, cmul_pi(O));
    }
    if (sp != s) {
      const cx<T> E = cscale(cadd(Xp, cconj(X)), half);
      const cx<T> O = cscale(cmulc(csub(Xp, cconj(X)), __ldg(&tw[kp])), half);
      e[sidx<T>(sp)] = cadd(E, cmul_pi(O));
    }
  }
  __syncthreads();
  fft_dit<T>(buf, logNp, NR, vs, stw);
}

// ---------------------------------------------------------------------------
// k_rows_remainder: the convolution rows only, C = -kappa tau^2 L_h u (the
// scale is in the symbol), written as a double-float pair of floats (the
// starting value of the incremental remainder of the FP32 forms).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_rows_remainder(const cx<T>* __restrict__ S, Geom g, const cx<T>* __restrict__ stw, const cx<T>* __restrict__ tw,
                 int NR, float* __restrict__ Ch, float* __restrict__ Cl) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const int N = g.N;
  const int vs = vstride<T>(g.Np);
  const int row0 = blockIdx.x * NR;
  const int nrows = min(NR, N - row0);
  rows_inverse<T>(buf, S, g, NR, row0, nrows, vs, stw, tw);
  for (int t = threadIdx.x; t < nrows * N; t += blockDim.x) {
    const int v = t / N, k = t % N;
    const T c = real_view<T>(buf + v * vs, k);
    const float hi = (float)c;
    const size_t idx = (size_t)(row0 + v) * g.ld + k;
    Ch[idx] = hi;
    Cl[idx] = (float)(c - (T)hi);
  }
}

// ---------------------------------------------------------------------------
// B^n at grid index idx (row element k, convolution read from the row vector
// e).  Wave (Sec. 3): conv + tau^2 (g(u^n) + f^n), or at n = 0
// tau phi2 + (conv + tau^2 (g + f))/2, conv = -kappa tau^2 L_h u^n.
// Diffusion: tau (g(u~) + f) - d + conv, with conv = -kappa tau L_h u~ (the
// plain form transforms u~ itself), or in the compensated form (Ch: the
// increment d is what was transformed, and C accumulates -kappa tau L_h u^n)
// C + conv/2 = -kappa tau L_h (u^n + d/2).  uaux is u^{n-1} in the plain form
// and d in the compensated one.
// DIFF: the equation of the launch (a template parameter of the row kernel,
// so that the wave step's epilogue carries none of the diffusion step's code).
template <typename T, bool DIFF>
__device__ __forceinline__ T rhs_at(const RhsParams& rp, const cx<T>* e, int k, size_t idx, const T* u,
                                    const T* uaux, const T* phi2, float* Ch, float* Cl) {
  if constexpr (!DIFF) {
    T conv = real_view<T>(e, k);
    if (Ch) conv = acc_remainder<T>(Ch, Cl, idx, conv);
    const T uu = u[idx];
    T gsrc = g_of<T>(rp, uu);
    if (rp.F) gsrc += T(rp.fsc) * static_cast<const T*>(rp.F)[idx];
    const T gg = T(rp.tau2) * gsrc;
    return rp.first ? T(rp.tau) * phi2[idx] + T(0.5) * (conv + gg) : conv + gg;
  }
  const T cd = real_view<T>(e, k);
  const T conv = Ch ? acc_remainder<T>(Ch, Cl, idx, cd) : cd;
  const T uu = u[idx];
  T fsrc = rp.F ? T(rp.fsc) * static_cast<const T*>(rp.F)[idx] : T(0);
  const T d = rp.first ? T(0) : (Ch ? uaux[idx] : uu - uaux[idx]);
  const T ut = uu + T(0.5) * d;
  const T b = conv + T(rp.tau2) * (g_of<T>(rp, ut) + fsrc) - d;
  return Ch ? b + T(0.5) * cd : b;
}

// ---------------------------------------------------------------------------
// k_rows_solve: per row j: inverse real FFT of the convolved half spectrum
// (gives -kappa tau^2 L_h u^n, the scale being folded into the symbol),
// B^n epilogue with g(u^n) (and phi2 when n = 0), then the x sweep W_j = H^-1 B_j.
// ---------------------------------------------------------------------------
// DENSE: the dense-inverse form stops after B^n, which it writes to W and,
// split into BF16 pairs, to Bh / Bl (ld ldp).
template <typename T, bool DENSE = false, int NT = kThreads, bool DIFF = false>
__global__ void __launch_bounds__(NT)
k_rows_solve(const cx<T>* __restrict__ S, const T* __restrict__ u, const T* __restrict__ uaux,
             const T* __restrict__ phi2, T* __restrict__ W,
             Geom g, RhsParams rp, const cx<T>* __restrict__ stw, const cx<T>* __restrict__ tw,
             const cx<T>* __restrict__ lam_s, const cx<T>* __restrict__ lam_c, const T* __restrict__ G, int NR,
             float* Ch, float* Cl, unsigned short* Bh = nullptr, unsigned short* Bl = nullptr, int ldp = 0) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const int N = g.N, Np = g.Np;
  const int vs = vstride<T>(Np);
  const int row0 = blockIdx.x * NR;
  const int nrows = min(NR, N - row0);
  rows_inverse<T>(buf, S, g, NR, row0, nrows, vs, stw, tw);
  // B^n and v1 = Q (v' + i J v'), staged through registers (in place).
  const int halfNp = Np >> 1;
  const int npairs = NR * halfNp;
  constexpr int MP = kMaxPairs * kThreads / NT;   // same pair capacity at any block size
  if constexpr (DENSE) {
    // B^n straight to W and its BF16 pair (no register staging: the rows are
    // not transformed further)
#pragma unroll 4
    for (int it = 0; it < MP; ++it) {
      const int t = threadIdx.x + it * blockDim.x;
      if (t < npairs) {
        const int v = t / halfNp, k = t % halfNp, k2 = Np - 1 - k;
        if (v < nrows) {
          const size_t row = (size_t)(row0 + v);
          const cx<T>* e = buf + v * vs;
          if (k < N) {
            const T b = rhs_at<T, DIFF>(rp, e, k, row * N + k, u, uaux, phi2, Ch, Cl);
            W[row * N + k] = b;
            split_bf16(b, Bh + row * ldp + k, Bl + row * ldp + k);
          }
          if (k2 < N) {
            const T b = rhs_at<T, DIFF>(rp, e, k2, row * N + k2, u, uaux, phi2, Ch, Cl);
            W[row * N + k2] = b;
            split_bf16(b, Bh + row * ldp + k2, Bl + row * ldp + k2);
          }
        }
      }
    }
  } else {
    T ra[MP], rb[MP];
#pragma unroll
    for (int it = 0; it < MP; ++it) {
      const int t = threadIdx.x + it * blockDim.x;
      ra[it] = T(0);
      rb[it] = T(0);
      if (t < npairs) {
        const int v = t / halfNp, k = t % halfNp, k2 = Np - 1 - k;
        if (v < nrows) {
          const int row = row0 + v;
          const cx<T>* e = buf + v * vs;
          if (k < N) ra[it] = rhs_at<T, DIFF>(rp, e, k, (size_t)row * N + k, u, uaux, phi2, Ch, Cl);
          if (k2 < N) rb[it] = rhs_at<T, DIFF>(rp, e, k2, (size_t)row * N + k2, u, uaux, phi2, Ch, Cl);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < MP; ++it) {
      const int t = threadIdx.x + it * blockDim.x;
      if (t < npairs) {
        const int v = t / halfNp, k = t % halfNp, k2 = Np - 1 - k;
        cx<T>* e = buf + v * vs;
        e[sidx<T>(k)] = cmul(mkc(ra[it], rb[it]), __ldg(&tw[k]));
        e[sidx<T>(k2)] = cmul(mkc(rb[it], ra[it]), __ldg(&tw[k2]));
      }
    }
    __syncthreads();
    gs_core<T>(buf, NR, vs, g, stw, tw, lam_s, lam_c);
    for (int t = threadIdx.x; t < nrows * N; t += blockDim.x) {
      const int v = t / N, k = t % N;
      W[(size_t)(row0 + v) * N + k] = gs_out<T>(buf + v * vs, k, g, G);
    }
  }
}

// ---------------------------------------------------------------------------
// k_cols_solve: per column i: y sweep uhat = H^-1 W_{:,i}, then the leapfrog
// u^{n+1} = 2u^n - u^{n-1} + uhat (n >= 1) or u^1 = u^0 + uhat (n = 0).
// u_next may alias u_prev (each element is read before it is written, by the
// same thread).  Compensated form (u_lo != nullptr, FP32): the state is the
// double-float pair u = u_cur + u_lo and the increment d = u^n - u^{n-1} held
// in u_prev; d^{n+1} = d^n + uhat (d^1 = uhat) and u^{n+1} = u^n + d^{n+1} by
// an error-free two-sum, written in place (u_next == u_cur).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_cols_solve(const T* __restrict__ W, const T* u_cur, T* u_prev, T* u_next, T* u_lo, Geom g, int first,
             const cx<T>* __restrict__ stw, const cx<T>* __restrict__ tw, const cx<T>* __restrict__ lam_s,
             const cx<T>* __restrict__ lam_c, const T* __restrict__ G, int CT) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const int N = g.N, Np = g.Np;
  const int vs = vstride<T>(Np);
  const int i0 = blockIdx.x * CT;
  for (int t = threadIdx.x; t < CT * Np; t += blockDim.x) {
    const int c = t % CT, k = t / CT;
    const int i = i0 + c, k2 = Np - 1 - k;
    T a = T(0), b = T(0);
    if (i < N) {
      if (k < N) a = W[(size_t)k * N + i];
      if (k2 < N) b = W[(size_t)k2 * N + i];
    }
    buf[c * vs + sidx<T>(k)] = cmul(mkc(a, b), __ldg(&tw[k]));
  }
  __syncthreads();
  gs_core<T>(buf, CT, vs, g, stw, tw, lam_s, lam_c);
  for (int t = threadIdx.x; t < CT * N; t += blockDim.x) {
    const int c = t % CT, j = t / CT;
    const int i = i0 + c;
    if (i >= N) continue;
    const T uh = gs_out<T>(buf + c * vs, j, g, G);
    const size_t idx = (size_t)j * N + i;
    const T uc = u_cur[idx];
    if (u_lo) {
      leapfrog_comp<T>(uc, uh, first, idx, u_prev, u_next, u_lo);
    } else {
      u_next[idx] = first ? uc + uh : (T(2) * uc - u_prev[idx]) + uh;
    }
  }
}

// ---------------------------------------------------------------------------
// The y sweep of the FP32 forms on the shared-memory engine, as the x sweep of
// the transpose (both sweeps apply the same H^-1, Sec. 3): W -> W^T by 32 x 32
// tiles, k_rows_gs on rows of W^T (whole rows, coalesced, where k_cols_solve
// gathers 4-byte column elements), and the transpose back fused with the
// leapfrog.  W^T and uhat^T live in the spectrum scratch, free at this point.
// ---------------------------------------------------------------------------
constexpr int kTT = 32;   // transpose tile

__global__ void __launch_bounds__(kTT * 8) k_transpose_f32(const float* __restrict__ A, float* __restrict__ AT, int N) {
  pdl_entry();
  __shared__ float tile[kTT][kTT + 1];
  const int x0 = blockIdx.x * kTT, y0 = blockIdx.y * kTT;
  for (int r = threadIdx.y; r < kTT; r += 8) {
    const int y = y0 + r, x = x0 + threadIdx.x;
    tile[r][threadIdx.x] = (y < N && x < N) ? A[(size_t)y * N + x] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < kTT; r += 8) {
    const int y = x0 + r, x = y0 + threadIdx.x;   // AT[y][x] = A[x][y]
    if (y < N && x < N) AT[(size_t)y * N + x] = tile[threadIdx.x][r];
  }
}

// rows i of W^T (columns of W): uhat_i^T = H^-1 W^T_i, as in k_cols_solve
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_rows_gs(const T* __restrict__ WT, T* __restrict__ UT, Geom g, const cx<T>* __restrict__ stw,
          const cx<T>* __restrict__ tw, const cx<T>* __restrict__ lam_s, const cx<T>* __restrict__ lam_c,
          const T* __restrict__ G, int NR) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const int N = g.N, Np = g.Np;
  const int vs = vstride<T>(Np);
  const int row0 = blockIdx.x * NR;
  const int nrows = min(NR, N - row0);
  for (int t = threadIdx.x; t < NR * Np; t += blockDim.x) {
    const int v = t / Np, k = t % Np, k2 = Np - 1 - k;
    T a = T(0), b = T(0);
    if (v < nrows) {
      const T* row = WT + (size_t)(row0 + v) * N;
      if (k < N) a = row[k];
      if (k2 < N) b = row[k2];
    }
    buf[v * vs + sidx<T>(k)] = cmul(mkc(a, b), __ldg(&tw[k]));
  }
  __syncthreads();
  gs_core<T>(buf, NR, vs, g, stw, tw, lam_s, lam_c);
  for (int t = threadIdx.x; t < nrows * N; t += blockDim.x) {
    const int v = t / N, j = t % N;
    UT[(size_t)(row0 + v) * N + j] = gs_out<T>(buf + v * vs, j, g, G);
  }
}

// u^{n+1} from uhat^T by 32 x 32 tiles: the compensated leapfrog of
// k_cols_solve, element (j, i) with uhat = UT[i][j]
__global__ void __launch_bounds__(kTT * 8) k_transpose_leapfrog(const float* __restrict__ UT, float* u_cur,
                                                                 float* d, float* u_lo, int N, int first) {
  pdl_entry();
  __shared__ float tile[kTT][kTT + 1];
  const int i0 = blockIdx.x * kTT, j0 = blockIdx.y * kTT;
  for (int r = threadIdx.y; r < kTT; r += 8) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < N && j < N) ? UT[(size_t)i * N + j] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < kTT; r += 8) {
    const int j = j0 + r, i = i0 + threadIdx.x;
    if (j < N && i < N) {
      const size_t idx = (size_t)j * N + i;
      leapfrog_comp<float>(u_cur[idx], tile[threadIdx.x][r], first, idx, d, u_cur, u_lo);
    }
  }
}

}  // namespace

template <typename T>
cudaError_t step_setup_attributes() {
  const int mx = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_rows_r2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
  if ((e = cudaFuncSetAttribute(k_rows_r2c<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
  if ((e = cudaFuncSetAttribute(k_cols_conv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
  if ((e = cudaFuncSetAttribute(k_rows_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
  if ((e = cudaFuncSetAttribute(k_rows_solve<T, false, kThreads, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                mx)))
    return e;
  if ((e = cudaFuncSetAttribute(k_cols_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
  if ((e = cudaFuncSetAttribute(k_rows_remainder<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
  if ((e = cudaFuncSetAttribute(k_rows_gs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
  if constexpr (sizeof(T) == 4) {
    if ((e = cudaFuncSetAttribute(k_rows_solve<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_rows_solve<T, true, 2 * kThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  mx)))
      return e;
    if ((e = cudaFuncSetAttribute(k_rows_solve<T, true, kThreads, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  mx)))
      return e;
    if ((e = cudaFuncSetAttribute(k_rows_solve<T, true, 2 * kThreads, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, mx)))
      return e;
  }
  return cudaSuccess;
}

template <typename T>
Tiles default_tiles(int Np, int N) {
  // rows per block of the row kernels and slots/columns per block of the
  // column kernels: about two resident blocks of 256 threads per SM at N' = 1024
  const int es = (int)sizeof(T) / 4;   // 1 (float) or 2 (double)
  Tiles t;
  t.rows = 2048 / es / Np;
  t.conv_cols = 1024 / es / Np;
  t.solve_cols = 2048 / es / Np;
  if (t.rows < 1) t.rows = 1;
  if (t.conv_cols < 1) t.conv_cols = 1;
  if (t.solve_cols < 1) t.solve_cols = 1;
  if (t.conv_cols > 8) t.conv_cols = 8;
  if (t.solve_cols > 16) t.solve_cols = 16;
  if (N > 0) {
    const int cap = (N + kSmallTileBlocks - 1) / kSmallTileBlocks;   // rows or columns per block
    if (t.rows > cap) t.rows = cap;
    if (t.solve_cols > cap) t.solve_cols = cap;
    const int ccap = Np / kSmallTileBlocks > 1 ? Np / kSmallTileBlocks : 1;   // a power of two
    if (t.conv_cols > ccap) t.conv_cols = ccap;
  }
  // FP32 at N' = 8192: the three-pass column convolution (conv_cols = -1)
  if (sizeof(T) == 4 && Np == 8192) t.conv_cols = kConvThreePass;
  return t;
}

template <typename T>
bool tiles_valid(const Geom& g, const Tiles& t) {
  const size_t vbytes = (size_t)vstride<T>(g.Np) * sizeof(cx<T>);
  const size_t lim = 227 * 1024;
  if (t.rows < 1 || t.solve_cols < 1) return false;
  if (t.conv_cols == kConvThreePass) {
    if (sizeof(T) != 4 || !conv3_supported(g.logNp)) return false;
  } else if (t.conv_cols < 1 || g.Np % t.conv_cols != 0 || 2 * t.conv_cols * vbytes > lim) {
    return false;
  }
  if (t.rows * (g.Np / 2) > kMaxPairs * kThreads) return false;
  if (t.rows * vbytes > lim || t.solve_cols * vbytes > lim) return false;
  return true;
}

// Block size of the dense form's Bn kernel: 512 threads from N' = 4096 on,
// where its long-latency loads need more warps than the one to three
// 256-thread blocks the shared-memory vectors leave room for (N' = 8192:
// 1446 -> 1081 us; N' = 4096: 295 -> 270 us).  The kernels that also run
// Algorithm 1 and the row FFT ran slower with 512 and keep 256.
template <typename T>
bool wide_rows(const Geom& g) {
  return sizeof(T) == 4 && g.Np >= 4096;
}

// The y sweep runs on the transpose for the FP32 compensated form (state in
// place: u_next == u_cur), where the spectrum scratch holds W^T and uhat^T.
template <typename T>
bool transposed_y_sweep(const T* u_lo) {
  return sizeof(T) == 4 && u_lo != nullptr;
}

// The column convolution: the three-pass form for conv_cols = kConvThreePass
// (its buffers in tb.c3), else the single-pass shared-memory kernel with CTc
// slots per block.
template <typename T>
cudaError_t launch_cols_conv(const Geom& g, const StepTables<T>& tb, int CTc, cx<T>* S, cudaStream_t st) {
  if (CTc == kConvThreePass) {
    if constexpr (sizeof(T) == 4) {
      if (tb.c3) return launch_conv3(*tb.c3, g.N, g.Np, S, tb.tw, st);
    }
    return cudaErrorInvalidValue;
  }
  const size_t vbytes = (size_t)vstride<T>(g.Np) * sizeof(cx<T>);
  return launch_dependent(k_cols_conv<T>, dim3(g.Np / CTc), dim3(kThreads), 2 * CTc * vbytes, st, S, g,
                          reinterpret_cast<const cx<T>*>(tb.stw), reinterpret_cast<const cx<T>*>(tb.tw), tb.lpb, CTc);
}

template <typename T>
cudaError_t launch_step(const Geom& g, const StepTables<T>& tb, const Tiles& tl, const RhsParams& rp, const T* u_cur,
                        T* u_prev, T* u_next, T* u_lo, const T* phi2, void* Sv, T* W, cudaStream_t st,
                        cudaEvent_t* ev, float* Ch, float* Cl) {
  const cx<T>* stw = reinterpret_cast<const cx<T>*>(tb.stw);
  const cx<T>* tw = reinterpret_cast<const cx<T>*>(tb.tw);
  const cx<T>* ls = reinterpret_cast<const cx<T>*>(tb.lam_s);
  const cx<T>* lc = reinterpret_cast<const cx<T>*>(tb.lam_c);
  cx<T>* S = reinterpret_cast<cx<T>*>(Sv);
  const size_t vbytes = (size_t)vstride<T>(g.Np) * sizeof(cx<T>);
  if (!tiles_valid<T>(g, tl)) return cudaErrorInvalidConfiguration;
  const int NR = tl.rows, CTc = tl.conv_cols, CTs = tl.solve_cols;
  const int rblocks = (g.N + NR - 1) / NR;
  if (ev) cudaEventRecord(ev[0], st);
  // incremental remainder (Ch != nullptr): transform the increment d = u_prev
  // FP64 diffusion step (n >= 1): transform u~ = u^n + (u^n - u^{n-1})/2
  const bool extrap = !Ch && rp.eq == 1 && !rp.first;
  // every kernel of the step a programmatic dependent of the one before it
  const dim3 rg(rblocks), kt(kThreads);
  const size_t rsm = NR * vbytes;
  unsigned short* const no_bf16 = nullptr;
  cudaError_t ce = extrap ? launch_dependent(k_rows_r2c<T, true>, rg, kt, rsm, st, u_cur, S, g, stw, tw, NR,
                                             static_cast<const T*>(u_prev), T(0.5))
                          : launch_dependent(k_rows_r2c<T>, rg, kt, rsm, st, static_cast<const T*>(Ch ? u_prev : u_cur),
                                             S, g, stw, tw, NR, static_cast<const T*>(nullptr), T(0));
  if (ce != cudaSuccess) return ce;
  if (ev) cudaEventRecord(ev[1], st);
  ce = launch_cols_conv<T>(g, tb, CTc, S, st);
  if (ce != cudaSuccess) return ce;
  if (ev) cudaEventRecord(ev[2], st);
  ce = rp.eq == 1 ? launch_dependent(k_rows_solve<T, false, kThreads, true>, rg, kt, rsm, st, S, u_cur,
                                     static_cast<const T*>(u_prev), phi2, W, g, rp, stw, tw, ls, lc, tb.G, NR, Ch, Cl,
                                     no_bf16, no_bf16, 0)
                  : launch_dependent(k_rows_solve<T>, rg, kt, rsm, st, S, u_cur, static_cast<const T*>(u_prev), phi2,
                                     W, g, rp, stw, tw, ls, lc, tb.G, NR, Ch, Cl, no_bf16, no_bf16, 0);
  if (ce != cudaSuccess) return ce;
  if (ev) cudaEventRecord(ev[3], st);
  if (transposed_y_sweep<T>(u_lo)) {
    // FP32 compensated form: the y sweep on rows of W^T (S is free scratch)
    float* WT = reinterpret_cast<float*>(S);
    float* UT = WT + (size_t)g.N * g.N;
    const dim3 tg((g.N + kTT - 1) / kTT, (g.N + kTT - 1) / kTT), tb8(kTT, 8);
    ce = launch_dependent(k_transpose_f32, tg, tb8, 0, st, reinterpret_cast<const float*>(W), WT, g.N);
    if (ce == cudaSuccess)
      ce = launch_dependent(k_rows_gs<T>, rg, kt, rsm, st, reinterpret_cast<const T*>(WT), reinterpret_cast<T*>(UT), g,
                            stw, tw, ls, lc, tb.G, NR);
    if (ce == cudaSuccess)
      ce = launch_dependent(k_transpose_leapfrog, tg, tb8, 0, st, static_cast<const float*>(UT),
                            reinterpret_cast<float*>(const_cast<T*>(u_cur)), reinterpret_cast<float*>(u_prev),
                            reinterpret_cast<float*>(u_lo), g.N, rp.first);
  } else {
    ce = launch_dependent(k_cols_solve<T>, dim3((g.N + CTs - 1) / CTs), kt, CTs * vbytes, st,
                          static_cast<const T*>(W), u_cur, u_prev, u_next, u_lo, g, rp.first, stw, tw, ls, lc, tb.G,
                          CTs);
  }
  if (ce != cudaSuccess) return ce;
  if (ev) cudaEventRecord(ev[4], st);
  return cudaSuccess;
}

template cudaError_t step_setup_attributes<float>();
template cudaError_t step_setup_attributes<double>();
template Tiles default_tiles<float>(int, int);
template Tiles default_tiles<double>(int, int);
template bool tiles_valid<float>(const Geom&, const Tiles&);
template bool tiles_valid<double>(const Geom&, const Tiles&);
template cudaError_t launch_step<float>(const Geom&, const StepTables<float>&, const Tiles&, const RhsParams&,
                                        const float*, float*, float*, float*, const float*, void*, float*,
                                        cudaStream_t, cudaEvent_t*, float*, float*);
template cudaError_t launch_step<double>(const Geom&, const StepTables<double>&, const Tiles&, const RhsParams&,
                                         const double*, double*, double*, double*, const double*, void*, double*,
                                         cudaStream_t, cudaEvent_t*, float*, float*);

template <typename T>
cudaError_t launch_remainder(const Geom& g, const StepTables<T>& tb, const Tiles& tl, const T* u, void* Sv, float* Ch,
                             float* Cl, cudaStream_t st) {
  const cx<T>* stw = reinterpret_cast<const cx<T>*>(tb.stw);
  const cx<T>* tw = reinterpret_cast<const cx<T>*>(tb.tw);
  cx<T>* S = reinterpret_cast<cx<T>*>(Sv);
  const size_t vbytes = (size_t)vstride<T>(g.Np) * sizeof(cx<T>);
  if (!tiles_valid<T>(g, tl)) return cudaErrorInvalidConfiguration;
  const int NR = tl.rows, CTc = tl.conv_cols;
  const int rblocks = (g.N + NR - 1) / NR;
  k_rows_r2c<T><<<rblocks, kThreads, NR * vbytes, st>>>(u, S, g, stw, tw, NR);
  cudaError_t ce = launch_cols_conv<T>(g, tb, CTc, S, st);
  if (ce != cudaSuccess) return ce;
  k_rows_remainder<T><<<rblocks, kThreads, NR * vbytes, st>>>(S, g, stw, tw, NR, Ch, Cl);
  return cudaGetLastError();
}
template cudaError_t launch_remainder<float>(const Geom&, const StepTables<float>&, const Tiles&, const float*, void*,
                                             float*, float*, cudaStream_t);
template cudaError_t launch_remainder<double>(const Geom&, const StepTables<double>&, const Tiles&, const double*,
                                              void*, float*, float*, cudaStream_t);

cudaError_t launch_dense_rows(const Geom& g, const StepTables<float>& tb, const Tiles& tl, const RhsParams& rp,
                              const float* u_cur, const float* d, const float* phi2, void* Sv, float* W,
                              float* Ch, float* Cl, unsigned short* Bh, unsigned short* Bl, int ldp, cudaStream_t st,
                              cudaEvent_t* ev) {
  using T = float;
  const cx<T>* stw = reinterpret_cast<const cx<T>*>(tb.stw);
  const cx<T>* tw = reinterpret_cast<const cx<T>*>(tb.tw);
  const cx<T>* ls = reinterpret_cast<const cx<T>*>(tb.lam_s);
  const cx<T>* lc = reinterpret_cast<const cx<T>*>(tb.lam_c);
  cx<T>* S = reinterpret_cast<cx<T>*>(Sv);
  const size_t vbytes = (size_t)vstride<T>(g.Np) * sizeof(cx<T>);
  if (!tiles_valid<T>(g, tl)) return cudaErrorInvalidConfiguration;
  const int NR = tl.rows, CTc = tl.conv_cols;
  const int rblocks = (g.N + NR - 1) / NR;
  if (ev) cudaEventRecord(ev[0], st);
  // every kernel a programmatic dependent of the one before it
  const dim3 rg(rblocks);
  const size_t rsm = NR * vbytes;
  cudaError_t ce = launch_dependent(k_rows_r2c<T>, rg, dim3(kThreads), rsm, st, d, S, g, stw, tw, NR,
                                    static_cast<const T*>(nullptr), T(0));
  if (ce != cudaSuccess) return ce;
  if (ev) cudaEventRecord(ev[1], st);
  ce = launch_cols_conv<T>(g, tb, CTc, S, st);
  if (ce != cudaSuccess) return ce;
  if (ev) cudaEventRecord(ev[2], st);
  const bool diff = rp.eq == 1;
  const dim3 kt(kThreads), kt2(2 * kThreads);
  if (wide_rows<T>(g) && diff)
    return launch_dependent(k_rows_solve<T, true, 2 * kThreads, true>, rg, kt2, rsm, st, S, u_cur, d, phi2, W, g, rp,
                            stw, tw, ls, lc, tb.G, NR, Ch, Cl, Bh, Bl, ldp);
  if (wide_rows<T>(g))
    return launch_dependent(k_rows_solve<T, true, 2 * kThreads>, rg, kt2, rsm, st, S, u_cur, d, phi2, W, g, rp, stw,
                            tw, ls, lc, tb.G, NR, Ch, Cl, Bh, Bl, ldp);
  if (diff)
    return launch_dependent(k_rows_solve<T, true, kThreads, true>, rg, kt, rsm, st, S, u_cur, d, phi2, W, g, rp, stw,
                            tw, ls, lc, tb.G, NR, Ch, Cl, Bh, Bl, ldp);
  return launch_dependent(k_rows_solve<T, true>, rg, kt, rsm, st, S, u_cur, d, phi2, W, g, rp, stw, tw, ls, lc, tb.G,
                          NR, Ch, Cl, Bh, Bl, ldp);
}

}  // namespace sadi
