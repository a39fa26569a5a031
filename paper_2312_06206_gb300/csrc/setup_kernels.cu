// setup_kernels.cu -- once-per-context FP64 setup of the S-ADI scheme
// (arXiv 2312.06206):
//   * twiddle table exp(-2 pi i k / P);
//   * 1D Riesz weights a_i (Sec. 2, eq. "single coefficient discrete Riesz"),
//     by the ratio a_{i+1}/a_i = (i - alpha/2)/(i + 1 + alpha/2) of the Gamma form;
//   * 2D weights a_ij (Sec. 2, eq. "center discretization"): Fourier
//     coefficients of (4 sin^2(eta/2) + 4 sin^2(xi/2))^(alpha/2) by the
//     trapezoid rule on M x M and 2M x 2M grids and one Richardson step on the
//     leading M^-(2+alpha) term; each 1D pass is an output-pruned DFT (only
//     the first N coefficients), computed as M/Np FFTs of length Np;
//   * symbol of the block-circulant embedding of L_h (Sec. 3), separably;
//   * Gohberg-Semencul generator c' = H'^-1 e_1 (Proposition 1) by the Durbin
//     recursion (the paper uses PCG with a tau-algebra preconditioner; any
//     exact solver gives the same c'), the spectra lambda_c = fft(c'),
//     lambda_s = fft(Q s') (eq. "eigenvalue of CS"), and the correction that
//     turns the bordered solve into H^-1.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fft.cuh"
#include "sadi_internal.h"

namespace sadi {

namespace {

__global__ void k_twiddles(double2* tw64, float2* tw32, int P) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  double s, c;
  sincospi(2.0 * (double)k / (double)P, &s, &c);
  tw64[k] = make_double2(c, -s);
  tw32[k] = make_float2((float)c, (float)-s);
}

// Per-stage twiddles of the length-2^logL plan: entry (q-1) * m + j of the
// stage with span S and radix R (m = S/R) is exp(-2 pi i j brev_R(q) / S).
__global__ void k_stage_twiddles(double2* out64, float2* out32, int logL) {
  const int ns = plan_stages(logL);
  const int total = fft_plan(logL).total;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int s = ns - 1;
  while (s > 0 && e < plan_stage(logL, s).off) --s;
  const Stage stg = plan_stage(logL, s);
  const int local = e - stg.off;
  const int logm = stg.logS - stg.logR;
  const int q = (local >> logm) + 1;
  const int j = local & ((1 << logm) - 1);
  const int lr = stg.logR;
  const int bq = lr == 1 ? q : lr == 2 ? (((q & 1) << 1) | (q >> 1)) : (((q & 1) << 2) | (q & 2) | (q >> 2));
  const long long ex = (long long)j * bq;                 // < S
  double sn, cs;
  sincospi(2.0 * (double)ex / (double)(1 << stg.logS), &sn, &cs);
  out64[e] = make_double2(cs, -sn);
  out32[e] = make_float2((float)cs, (float)-sn);
}

__global__ void k_unit_roots(double2* w, int M) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  double s, c;
  sincospi(2.0 * (double)k / (double)M, &s, &c);
  w[k] = make_double2(c, -s);
}

__global__ void k_sinsq(double* s2, int M) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > M / 2) return;
  const double s = sinpi((double)k / (double)M);
  s2[k] = 4.0 * s * s;
}

__global__ void k_riesz1d(double* a, int n, double alpha) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double h = 0.5 * alpha;
  const double g1 = tgamma(h + 1.0);
  double v = tgamma(alpha + 1.0) / (g1 * g1);
  for (int i = 0; i < n; ++i) {
    a[i] = v;
    v = v * ((double)i - h) / ((double)i + 1.0 + h);
  }
}

// Output-pruned DFT of an even real sequence f[0..Mg-1]:
//   X[i] = sum_k f[k] exp(-2 pi i i k / Mg),  0 <= i < N,
// as sum_d exp(-2 pi i d i / Mg) F_d[i], F_d = DFT_Np(f[q D + d]), D = Mg/Np,
// with two decimated sequences packed in one complex FFT.
//   mode 0: block = grid row l in [0, Mg/2]; f[k] = (s2[k] + s2[l])^(alpha/2);
//           writes GT[i * ldg + l].
//   mode 1: block = i in [0, N); f[l] = GT[i * ldg + l] (folded);
//           writes A[i * N + j] = X[j] * outscale.
__global__ void k_trap_pass(int mode, double alpha, int Mg, const double* __restrict__ s2,
                            const double2* __restrict__ twM, Geom g, const double2* __restrict__ stw,
                            double* GT, int ldg, double* A, double outscale, int NVB) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* buf = reinterpret_cast<double2*>(smem_raw);
  const int L = g.Np, logL = g.logNp, N = g.N;
  const int vs = vec_stride(L);
  double* acc = reinterpret_cast<double*>(buf + NVB * vs);
  const int D = Mg >> logL;
  const int npairs = D / 2;
  const int b = blockIdx.x;
  const double ex = 0.5 * alpha;
  const double sl = (mode == 0) ? s2[b] : 0.0;
  for (int p = threadIdx.x; p < L; p += blockDim.x) acc[p] = 0.0;
  for (int c0 = 0; c0 < npairs; c0 += NVB) {
    const int nb = min(NVB, npairs - c0);
    for (int t = threadIdx.x; t < (nb << logL); t += blockDim.x) {
      const int bv = t >> logL, q = t & (L - 1);
      const int k0 = q * D + 2 * (c0 + bv);
      const int k1 = k0 + 1;
      const int f0i = min(k0, Mg - k0), f1i = min(k1, Mg - k1);
      double f0, f1;
      if (mode == 0) {
        f0 = pow(s2[f0i] + sl, ex);
        f1 = pow(s2[f1i] + sl, ex);
      } else {
        f0 = GT[(size_t)b * ldg + f0i];
        f1 = GT[(size_t)b * ldg + f1i];
      }
      buf[bv * vs + padi(q)] = make_double2(f0, f1);
    }
    __syncthreads();
    fft_dif<double>(buf, logL, nb, vs, stw);
    for (int p = threadIdx.x; p < L; p += blockDim.x) {
      const int i = brev(p, logL);
      if (i >= N) continue;
      const int pp = brev((L - i) & (L - 1), logL);
      double sum = 0.0;
      for (int bv = 0; bv < nb; ++bv) {
        const double2 Z = buf[bv * vs + padi(p)];
        const double2 Zc = cconj(buf[bv * vs + padi(pp)]);
        const double2 F0 = cscale(cadd(Z, Zc), 0.5);
        const double2 F1 = cscale(cmul_mi(csub(Z, Zc)), 0.5);
        const long long d0 = 2LL * (c0 + bv);
        const double2 w0 = twM[(int)((d0 * i) & (Mg - 1))];
        const double2 w1 = twM[(int)(((d0 + 1) * i) & (Mg - 1))];
        sum += (w0.x * F0.x - w0.y * F0.y) + (w1.x * F1.x - w1.y * F1.y);
      }
      acc[p] += sum;
    }
    __syncthreads();
  }
  for (int p = threadIdx.x; p < L; p += blockDim.x) {
    const int i = brev(p, logL);
    if (i >= N) continue;
    if (mode == 0) GT[(size_t)i * ldg + b] = acc[p];
    else A[(size_t)b * N + i] = acc[p] * outscale;
  }
}

__global__ void k_richardson(const double* A1, const double* A2, double* out, size_t n, double q) {
  const size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  out[k] = (q * A2[k] - A1[k]) / (q - 1.0);
}

// One real even sequence of length P = 2Np per block, transformed by the
// packed real FFT; writes the (real) transform X[k], 0 <= k <= Np, in
// natural order.
//   mode 0: block j in [0, N):   x[m] = a2d[dist(m) * N + j]       -> dst[j * (Np+1) + k]
//   mode 1: block k1 in [0, Np]: x[m] = src[dist(m) * (Np+1) + k1] -> dst[k1 * (Np+1) + k]
// dist(m) = min(m, P - m), entries with dist > N - 1 are zero.
__global__ void k_lambda_pass(int mode, const double* __restrict__ src, Geom g, const double2* __restrict__ stw,
                              const double2* __restrict__ tw, double* __restrict__ dst) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* buf = reinterpret_cast<double2*>(smem_raw);
  const int N = g.N, Np = g.Np, logNp = g.logNp, P = g.P;
  const int b = blockIdx.x;
  const int lds = (mode == 0) ? N : Np + 1;
  for (int n = threadIdx.x; n < Np; n += blockDim.x) {
    double v[2];
    for (int e = 0; e < 2; ++e) {
      const int m = 2 * n + e;
      const int d = min(m, P - m);
      v[e] = (d <= N - 1) ? src[(size_t)d * lds + b] : 0.0;
    }
    buf[padi(n)] = make_double2(v[0], v[1]);
  }
  __syncthreads();
  fft_dif<double>(buf, logNp, 1, vec_stride(Np), stw);
  for (int s = threadIdx.x; s < Np; s += blockDim.x) {
    const int k = brev(s, logNp);
    const int sp = brev((Np - k) & (Np - 1), logNp);
    const double2 Z = buf[padi(s)];
    const double2 Zc = cconj(buf[padi(sp)]);
    const double2 E = cscale(cadd(Z, Zc), 0.5);
    const double2 O = cscale(cmul_mi(csub(Z, Zc)), 0.5);
    double* row = dst + (size_t)b * (Np + 1);
    if (s == 0) {
      row[0] = E.x + O.x;
      row[Np] = E.x - O.x;
    } else {
      const double2 X = cadd(E, cmul(tw[k], O));
      row[k] = X.x;
    }
  }
}

__global__ void k_lambda_arrange(const double* __restrict__ lnat, Geom g, double scale, double* lpb64,
                                 float* lpb32) {
  const int Np = g.Np, logNp = g.logNp, P = g.P;
  const size_t total = (size_t)(Np + 1) * 2 * Np;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int p = (int)(idx % Np);
  const int h = (int)((idx / Np) % 2);
  const int slot = (int)(idx / (2 * (size_t)Np));
  int k2 = 2 * brev(p, logNp) + h;
  if (k2 > Np) k2 = P - k2;
  double val;
  // slot 0 carries the k1 = 0 symbol, the extra slot Np the k1 = Np symbol
  if (slot >= 1 && slot < Np) val = lnat[(size_t)brev(slot, logNp) * (Np + 1) + k2];
  else if (slot == 0) val = lnat[k2];
  else val = lnat[(size_t)Np * (Np + 1) + k2];
  val *= scale;
  lpb64[idx] = val;
  lpb32[idx] = (float)val;
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Durbin recursion (normalised Yule-Walker) for the symmetric Toeplitz H'
// with t_0 = 1 + s a_0, t_k = s a_k: c' = [1; y] / (t_0 sigma).
__global__ void k_durbin(const double* __restrict__ a1, int Np, double s, double* c, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* y = reinterpret_cast<double*>(smem_raw);
  double* r = y + Np;
  double* red = r + Np + 1;
  const double t0 = 1.0 + s * a1[0];
  for (int k = threadIdx.x; k < Np; k += blockDim.x) r[k] = (k == 0) ? 1.0 : s * a1[k] / t0;
  __syncthreads();
  const int n = Np - 1;
  int bad = 0;
  if (n == 0) {
    if (threadIdx.x == 0) { c[0] = 1.0 / t0; *status = 0; }
    return;
  }
  if (threadIdx.x == 0) y[0] = -r[1];
  double beta = 1.0, al = -r[1];
  __syncthreads();
  for (int k = 1; k < n; ++k) {
    beta = (1.0 - al * al) * beta;
    if (!(beta > 0.0)) bad = 1;
    double part = 0.0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) part += r[k - i] * y[i];
    const double dot = block_sum(part, red);
    al = -(r[k + 1] + dot) / beta;
    for (int i = threadIdx.x; i < (k + 1) / 2; i += blockDim.x) {
      const int i2 = k - 1 - i;
      const double yi = y[i], yi2 = y[i2];
      y[i] = yi + al * yi2;
      if (i2 != i) y[i2] = yi2 + al * yi;
    }
    if (threadIdx.x == 0) y[k] = al;
    __syncthreads();
  }
  double part = 0.0;
  for (int k = 1 + threadIdx.x; k <= n; k += blockDim.x) part += r[k] * y[k - 1];
  const double sigma = 1.0 + block_sum(part, red);
  if (!(sigma > 0.0) || !isfinite(sigma)) bad = 1;
  const double inv = 1.0 / (t0 * sigma);
  for (int k = threadIdx.x; k < Np; k += blockDim.x) c[k] = (k == 0) ? inv : y[k - 1] * inv;
  if (threadIdx.x == 0) *status = bad;
}

// which = 0: lambda_c = fft(c') / (2 p1 Np); which = 1: lambda_s = fft(Q s') / Np;
// bit-reversed order, s' = [p1, -p_Np, ..., -p_2], Q = diag(exp(-i pi k / Np)).
__global__ void k_gs_table(int which, const double* __restrict__ c, Geom g, const double2* __restrict__ stw,
                           const double2* __restrict__ tw, double2* out64, float2* out32) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* buf = reinterpret_cast<double2*>(smem_raw);
  const int Np = g.Np;
  for (int k = threadIdx.x; k < Np; k += blockDim.x) {
    if (which == 0) {
      buf[padi(k)] = make_double2(c[k], 0.0);
    } else {
      const double sk = (k == 0) ? c[0] : -c[Np - k];
      buf[padi(k)] = cscale(tw[k], sk);
    }
  }
  __syncthreads();
  fft_dif<double>(buf, g.logNp, 1, vec_stride(Np), stw);
  const double sc = (which == 0) ? 1.0 / (2.0 * c[0] * (double)Np) : 1.0 / (double)Np;
  for (int p = threadIdx.x; p < Np; p += blockDim.x) {
    const double2 a = cscale(buf[padi(p)], sc);
    out64[p] = a;
    out32[p] = make_float2((float)a.x, (float)a.y);
  }
}

// X[i][q] = (H'^-1)[i][N + q] from the Gohberg-Semencul form
// H'^-1 = (1/p1) (L(c) L(c)^T - L(yh) L(yh)^T), yh = Z J c'.
__global__ void k_border_X(const double* __restrict__ c, Geom g, double* X) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.Np * g.r) return;
  const int i = idx / g.r, q = idx % g.r, j = g.N + q, Np = g.Np;
  const int mm = min(i, j);
  double acc = 0.0;
  for (int m = 0; m <= mm; ++m) {
    const int a = i - m, b = j - m;
    const double ya = (a == 0) ? 0.0 : c[Np - a];
    const double yb = (b == 0) ? 0.0 : c[Np - b];
    acc += c[a] * c[b] - ya * yb;
  }
  X[idx] = acc / c[0];
}

// In-place Gauss-Jordan inverse of the SPD r x r matrix M (no pivoting).
__global__ void k_gauss_jordan(double* M, double* Inv, int r) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* fcol = reinterpret_cast<double*>(smem_raw);
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) Inv[e] = (e / r == e % r) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    const double piv = M[k * r + k];
    __syncthreads();
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
      M[k * r + j] /= piv;
      Inv[k * r + j] /= piv;
    }
    for (int i = threadIdx.x; i < r; i += blockDim.x) fcol[i] = M[i * r + k];
    __syncthreads();
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      if (i == k) continue;
      const double f = (i == k) ? 0.0 : fcol[i];
      M[e] -= f * M[k * r + j];
      Inv[e] -= f * Inv[k * r + j];
    }
    __syncthreads();
  }
}

// G = -X_top X_bot^-1  (N x r), FP64 and FP32.
__global__ void k_border_G(const double* __restrict__ X, const double* __restrict__ Dinv, Geom g, double* G64,
                           float* G32) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.N * g.r) return;
  const int k = idx / g.r, q = idx % g.r;
  double acc = 0.0;
  for (int t = 0; t < g.r; ++t) acc += X[k * g.r + t] * Dinv[t * g.r + q];
  G64[idx] = -acc;
  G32[idx] = (float)(-acc);
}

// Register-path tables.  tw1: exp(-2 pi i t k1 / Np) at [k1 * TT + t] with
// TT = 2^floor(logNp/2); lreg[(k1 * 2 + h) * Np + m] = scale * Lambda(k1, 2m + h)
// (natural order, k2 folded into [0, Np]); lam*_nat[k] = lam*[brev(k)].
__global__ void k_reg_tables(Geom g, const double* __restrict__ lnat, double scale,
                             const double2* __restrict__ lamc64, const double2* __restrict__ lams64, float2* tw1,
                             float* lreg, float2* lamc_nat, float2* lams_nat) {
  const int Np = g.Np, logNp = g.logNp, P = g.P;
  const int logT = logNp / 2;
  const int TT = 1 << logT;
  const size_t nl = (size_t)(Np + 1) * 2 * Np;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx < (size_t)Np) {
    const int k = (int)idx;
    const int t = k & (TT - 1), k1 = k >> logT;
    double sn, cs;
    sincospi(2.0 * (double)((long long)t * k1 % Np) / (double)Np, &sn, &cs);
    tw1[k] = make_float2((float)cs, (float)-sn);
    const double2 a = lamc64[brev(k, logNp)], b = lams64[brev(k, logNp)];
    lamc_nat[k] = make_float2((float)a.x, (float)a.y);
    lams_nat[k] = make_float2((float)b.x, (float)b.y);
  }
  if (idx < nl) {
    const int m = (int)(idx % Np);
    const int h = (int)((idx / Np) % 2);
    const int k1 = (int)(idx / (2 * (size_t)Np));
    int k2 = 2 * m + h;
    if (k2 > Np) k2 = P - k2;
    lreg[idx] = (float)(scale * lnat[(size_t)k1 * (Np + 1) + k2]);
  }
}

// Element-wise conversions over a rows x cols array (source rows sld apart,
// destination rows dld apart): thread -> column blockIdx.x * blockDim.x +
// threadIdx.x of rows blockIdx.y, blockIdx.y + gridDim.y, ... (no index
// division per element).
struct Pitch2 {
  int rows, cols, sld, dld;
};
template <typename F>
__device__ __forceinline__ void for_each_element(const Pitch2& p, F f) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.cols) return;
  for (int r = blockIdx.y; r < p.rows; r += gridDim.y) f((size_t)r * p.sld + c, (size_t)r * p.dld + c);
}
__global__ void k_d2f(const double* __restrict__ s, float* __restrict__ d, Pitch2 p) {
  for_each_element(p, [&](size_t si, size_t di) { d[di] = (float)s[si]; });
}
__global__ void k_f2d(const float* __restrict__ s, double* __restrict__ d, Pitch2 p) {
  for_each_element(p, [&](size_t si, size_t di) { d[di] = (double)s[si]; });
}
__global__ void k_split_d2ff(const double* __restrict__ s, float* __restrict__ hi, float* __restrict__ lo, Pitch2 p) {
  for_each_element(p, [&](size_t si, size_t di) {
    const double v = s[si];
    const float h = (float)v;
    hi[di] = h;
    lo[di] = (float)(v - (double)h);
  });
}
__global__ void k_join_ff2d(const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ d,
                            Pitch2 p) {
  for_each_element(p, [&](size_t si, size_t di) { d[di] = (double)hi[si] + (double)lo[si]; });
}
__global__ void k_join_ff2f(const float* __restrict__ hi, const float* __restrict__ lo, float* __restrict__ d,
                            Pitch2 p) {
  for_each_element(p, [&](size_t si, size_t di) { d[di] = hi[si] + lo[si]; });
}
// grid of a conversion: 256 threads a block across a row, rows over y
inline dim3 pitch_grid(int rows, int cols) {
  return dim3((unsigned)((cols + 255) / 256), (unsigned)(rows < 65535 ? rows : 65535));
}

inline unsigned nblk(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_twiddles(double2* tw64, float2* tw32, int P, cudaStream_t st) {
  k_twiddles<<<nblk(P, 256), 256, 0, st>>>(tw64, tw32, P);
  return cudaGetLastError();
}

cudaError_t launch_stage_twiddles(double2* stw64, float2* stw32, int logL, cudaStream_t st) {
  const int total = fft_plan(logL).total;
  k_stage_twiddles<<<nblk(total, 256), 256, 0, st>>>(stw64, stw32, logL);
  return cudaGetLastError();
}

cudaError_t run_reg_tables(const Geom& g, const double* lnat, double scale, const double2* lamc64,
                           const double2* lams64, float2* tw1, float* lreg, float2* lamc_nat, float2* lams_nat,
                           cudaStream_t st) {
  const size_t nl = (size_t)(g.Np + 1) * 2 * g.Np;
  k_reg_tables<<<nblk(nl, 256), 256, 0, st>>>(g, lnat, scale, lamc64, lams64, tw1, lreg, lamc_nat, lams_nat);
  return cudaGetLastError();
}

cudaError_t launch_riesz1d(double* a, int n, double alpha, cudaStream_t st) {
  k_riesz1d<<<1, 32, 0, st>>>(a, n, alpha);
  return cudaGetLastError();
}

cudaError_t launch_convert_d2f(const double* s, float* d, int rows, int cols, int sld, int dld, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  k_d2f<<<pitch_grid(rows, cols), 256, 0, st>>>(s, d, Pitch2{rows, cols, sld, dld});
  return cudaGetLastError();
}
cudaError_t launch_split_d2ff(const double* s, float* hi, float* lo, int rows, int cols, int sld, int dld,
                              cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  k_split_d2ff<<<pitch_grid(rows, cols), 256, 0, st>>>(s, hi, lo, Pitch2{rows, cols, sld, dld});
  return cudaGetLastError();
}
cudaError_t launch_join_ff2d(const float* hi, const float* lo, double* d, int rows, int cols, int sld, int dld,
                             cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  k_join_ff2d<<<pitch_grid(rows, cols), 256, 0, st>>>(hi, lo, d, Pitch2{rows, cols, sld, dld});
  return cudaGetLastError();
}
cudaError_t launch_join_ff2f(const float* hi, const float* lo, float* d, int rows, int cols, int sld, int dld,
                             cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  k_join_ff2f<<<pitch_grid(rows, cols), 256, 0, st>>>(hi, lo, d, Pitch2{rows, cols, sld, dld});
  return cudaGetLastError();
}

cudaError_t launch_convert_f2d(const float* s, double* d, int rows, int cols, int sld, int dld, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  k_f2d<<<pitch_grid(rows, cols), 256, 0, st>>>(s, d, Pitch2{rows, cols, sld, dld});
  return cudaGetLastError();
}

// H^-1 - I from the generator c = H^-1 e_1 of the symmetric Toeplitz H (n x n),
// by the Gohberg-Semencul identity H^-1 = (1/c_0)(L(c) L(c)^T - L(y) L(y)^T),
// y = (0, c_{n-1}, ..., c_1), read along diagonals:
//   (H^-1)[d + j][j] = (H^-1)[d + j - 1][j - 1] + (c_{d+j} c_j - y_{d+j} y_j) / c_0,
//   (H^-1)[d][0] = c_d.
// One thread per diagonal d; both triangles written (symmetry), as BF16 pairs.
__global__ void k_dense_inverse(const double* __restrict__ c, int n, int npad, unsigned short* Eh,
                                unsigned short* El) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const double c0 = c[0];
  double v = c[d];
  for (int j = 0; j < n - d; ++j) {
    if (j > 0) v += (c[d + j] * c[j] - c[n - d - j] * c[n - j]) / c0;
    const double e = (d == 0) ? v - 1.0 : v;
    const float ef = (float)e;
    const __nv_bfloat16 h = __float2bfloat16_rn(ef);
    const unsigned short hb = __bfloat16_as_ushort(h);
    const unsigned short lb = __bfloat16_as_ushort(__float2bfloat16_rn((float)(e - (double)__bfloat162float(h))));
    const size_t a = (size_t)(d + j) * npad + j, b = (size_t)j * npad + (d + j);
    Eh[a] = hb;
    El[a] = lb;
    Eh[b] = hb;
    El[b] = lb;
  }
}

#define SADI_TRY(x)                        \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) { err = e_; goto done; } \
  } while (0)

cudaError_t run_weights2d(double* a2d, const Geom& g, double alpha, int M, const double2* stw64, cudaStream_t st) {
  cudaError_t err = cudaSuccess;
  const int M2 = 2 * M;
  const int ldg = M2 / 2 + 1;
  const size_t nn = (size_t)g.N * g.N;
  double *s2 = nullptr, *GT = nullptr, *A1 = nullptr, *A2 = nullptr;
  double2* twM = nullptr;
  const int vs = vec_stride(g.Np);
  const size_t vbytes = (size_t)vs * sizeof(double2);
  const size_t accbytes = (size_t)g.Np * sizeof(double);
  const size_t budget = 200 * 1024;
  int NVB = (int)((budget - accbytes) / vbytes);
  if (NVB < 1) NVB = 1;
  if (NVB > 8) NVB = 8;
  SADI_TRY(cudaFuncSetAttribute(k_trap_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  SADI_TRY(cudaMalloc(&s2, sizeof(double) * (M2 / 2 + 1)));
  SADI_TRY(cudaMalloc(&twM, sizeof(double2) * M2));
  SADI_TRY(cudaMalloc(&GT, sizeof(double) * (size_t)g.N * ldg));
  SADI_TRY(cudaMalloc(&A1, sizeof(double) * nn));
  SADI_TRY(cudaMalloc(&A2, sizeof(double) * nn));
  for (int pass = 0; pass < 2; ++pass) {
    const int Mg = (pass == 0) ? M : M2;
    double* A = (pass == 0) ? A1 : A2;
    k_sinsq<<<nblk(Mg / 2 + 1, 256), 256, 0, st>>>(s2, Mg);
    k_unit_roots<<<nblk(Mg, 256), 256, 0, st>>>(twM, Mg);
    const int nb = NVB;
    k_trap_pass<<<Mg / 2 + 1, 256, nb * vbytes + accbytes, st>>>(0, alpha, Mg, s2, twM, g, stw64, GT, ldg, nullptr,
                                                                   0.0, nb);
    k_trap_pass<<<g.N, 256, nb * vbytes + accbytes, st>>>(1, alpha, Mg, s2, twM, g, stw64, GT, ldg, A,
                                                          1.0 / ((double)Mg * (double)Mg), nb);
    SADI_TRY(cudaGetLastError());
  }
  k_richardson<<<nblk(nn, 256), 256, 0, st>>>(A1, A2, a2d, nn, pow(2.0, 2.0 + alpha));
  SADI_TRY(cudaGetLastError());
  SADI_TRY(cudaStreamSynchronize(st));
done:
  cudaFree(s2);
  cudaFree(twM);
  cudaFree(GT);
  cudaFree(A1);
  cudaFree(A2);
  return err;
}

cudaError_t run_lambda(const double* a2d, const Geom& g, const double2* stw64, const double2* tw64, double scale,
                       double* lnat, double* lpb64, float* lpb32, cudaStream_t st) {
  cudaError_t err = cudaSuccess;
  double* TA = nullptr;
  const size_t sm = (size_t)vec_stride(g.Np) * sizeof(double2);
  SADI_TRY(cudaFuncSetAttribute(k_lambda_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  SADI_TRY(cudaMalloc(&TA, sizeof(double) * (size_t)g.N * (g.Np + 1)));
  k_lambda_pass<<<g.N, 256, sm, st>>>(0, a2d, g, stw64, tw64, TA);
  k_lambda_pass<<<g.Np + 1, 256, sm, st>>>(1, TA, g, stw64, tw64, lnat);
  {
    const size_t total = (size_t)(g.Np + 1) * 2 * g.Np;
    k_lambda_arrange<<<nblk(total, 256), 256, 0, st>>>(lnat, g, scale, lpb64, lpb32);
  }
  SADI_TRY(cudaGetLastError());
  SADI_TRY(cudaStreamSynchronize(st));
done:
  cudaFree(TA);
  return err;
}

cudaError_t run_generator(const double* a1, const Geom& g, double s, const double2* stw64, const double2* tw64,
                          double* cgen,
                          double2* lamc64, double2* lams64, float2* lamc32, float2* lams32, double* G64,
                          float* G32, int* status_host, cudaStream_t st) {
  cudaError_t err = cudaSuccess;
  int* dstat = nullptr;
  double *X = nullptr, *Mb = nullptr, *Inv = nullptr;
  *status_host = 1;
  const size_t smd = sizeof(double) * (2 * (size_t)g.Np + 1 + 32);
  const size_t smt = (size_t)vec_stride(g.Np) * sizeof(double2);
  SADI_TRY(cudaFuncSetAttribute(k_durbin, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  SADI_TRY(cudaFuncSetAttribute(k_gs_table, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  SADI_TRY(cudaFuncSetAttribute(k_gauss_jordan, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  SADI_TRY(cudaMalloc(&dstat, sizeof(int)));
  k_durbin<<<1, 1024, smd, st>>>(a1, g.Np, s, cgen, dstat);
  SADI_TRY(cudaGetLastError());
  if (smt > 227 * 1024) { err = cudaErrorInvalidConfiguration; goto done; }
  k_gs_table<<<1, 256, smt, st>>>(0, cgen, g, stw64, tw64, lamc64, lamc32);
  k_gs_table<<<1, 256, smt, st>>>(1, cgen, g, stw64, tw64, lams64, lams32);
  SADI_TRY(cudaGetLastError());
  if (g.r > 0) {
    const int r = g.r;
    SADI_TRY(cudaMalloc(&X, sizeof(double) * (size_t)g.Np * r));
    SADI_TRY(cudaMalloc(&Mb, sizeof(double) * (size_t)r * r));
    SADI_TRY(cudaMalloc(&Inv, sizeof(double) * (size_t)r * r));
    k_border_X<<<nblk((size_t)g.Np * r, 128), 128, 0, st>>>(cgen, g, X);
    SADI_TRY(cudaMemcpyAsync(Mb, X + (size_t)g.N * r, sizeof(double) * (size_t)r * r, cudaMemcpyDeviceToDevice, st));
    k_gauss_jordan<<<1, 1024, sizeof(double) * r, st>>>(Mb, Inv, r);
    k_border_G<<<nblk((size_t)g.N * r, 128), 128, 0, st>>>(X, Inv, g, G64, G32);
    SADI_TRY(cudaGetLastError());
  }
  SADI_TRY(cudaMemcpyAsync(status_host, dstat, sizeof(int), cudaMemcpyDeviceToHost, st));
  SADI_TRY(cudaStreamSynchronize(st));
done:
  cudaFree(dstat);
  cudaFree(X);
  cudaFree(Mb);
  cudaFree(Inv);
  return err;
}

cudaError_t run_dense_inverse(const double* a1, int N, double s, int npad, void* Eh, void* El, int* status_host,
                              cudaStream_t st) {
  cudaError_t err = cudaSuccess;
  int* dstat = nullptr;
  double* c = nullptr;
  *status_host = 1;
  const size_t smd = sizeof(double) * (2 * (size_t)N + 1 + 32);
  const size_t ne = (size_t)npad * npad * sizeof(unsigned short);
  SADI_TRY(cudaFuncSetAttribute(k_durbin, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  if (smd > 227 * 1024) { err = cudaErrorInvalidConfiguration; goto done; }
  SADI_TRY(cudaMalloc(&dstat, sizeof(int)));
  SADI_TRY(cudaMalloc(&c, sizeof(double) * N));
  k_durbin<<<1, 1024, smd, st>>>(a1, N, s, c, dstat);
  SADI_TRY(cudaGetLastError());
  SADI_TRY(cudaMemsetAsync(Eh, 0, ne, st));
  SADI_TRY(cudaMemsetAsync(El, 0, ne, st));
  k_dense_inverse<<<nblk(N, 128), 128, 0, st>>>(c, N, npad, static_cast<unsigned short*>(Eh),
                                                static_cast<unsigned short*>(El));
  SADI_TRY(cudaGetLastError());
  SADI_TRY(cudaMemcpyAsync(status_host, dstat, sizeof(int), cudaMemcpyDeviceToHost, st));
  SADI_TRY(cudaStreamSynchronize(st));
done:
  cudaFree(dstat);
  cudaFree(c);
  return err;
}

}  // namespace sadi
