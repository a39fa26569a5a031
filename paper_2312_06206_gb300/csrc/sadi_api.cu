// sadi_api.cu -- the C ABI declared in include/sadi.h: context lifetime,
// argument validation, FP64 setup orchestration and the step loop.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <array>
#include <memory>
#include <string>
#include <vector>

#include "../../include/sadi.h"
#include "fft.cuh"
#include "sadi_ctx.h"
#include "sadi_internal.h"

using namespace sadi;

static thread_local std::string g_create_err;

namespace sadi_api {

sadi_status fail(sadi_ctx* c, sadi_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

sadi_status cuda_fail(sadi_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (c) {
    c->err = m;
    c->broken = true;
  }
  return SADI_ECUDA;
}

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e__ = (call);                            \
    if (e__ != cudaSuccess) return cuda_fail(c, e__, what); \
  } while (0)

template <typename T>
T* dalloc(size_t n, cudaError_t* e) {
  void* p = nullptr;
  *e = cudaMalloc(&p, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
  return static_cast<T*>(p);
}

void free_all(sadi_ctx* c) {
  void* ptrs[] = {c->rtw1, c->rlreg, c->rlamc, c->rlams, c->stw64, c->stw32, c->a1,     c->a2d,    c->cgen,   c->lnat,   c->tw64,   c->tw32, c->lpb64,
                  c->lpb32,  c->lamc64, c->lams64, c->lamc32, c->lams32, c->G64,  c->G32,
                  c->ubuf[0], c->ubuf[1], c->ulo, c->F, c->phi2, c->S,      c->W,      c->stage};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  conv3_free(&c->c3);
  void* dense[] = {c->Eh, c->El, c->Bh, c->Bl, c->WTh, c->WTl, c->tcerr, c->tcdep, c->Chi, c->Clo, c->wd, c->Fconv};
  for (void* p : dense)
    if (p) cudaFree(p);
  for (auto& a : c->ev_pool)
    for (auto e : a) cudaEventDestroy(e);
  for (auto& a : c->ev_free)
    for (auto e : a) cudaEventDestroy(e);
  c->ev_pool.clear();
  c->ev_free.clear();
  if (c->order_ev) cudaEventDestroy(c->order_ev);
  if (c->ev_staged) cudaEventDestroy(c->ev_staged);
  if (c->ev_copied) cudaEventDestroy(c->ev_copied);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
}

// Fold recorded per-kernel events into the accumulators (waits for them).
cudaError_t fold_events(sadi_ctx* c) {
  for (auto& a : c->ev_pool) {
    cudaError_t e = cudaEventSynchronize(a[4]);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < 4; ++k) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, a[k], a[k + 1]);
      if (e != cudaSuccess) return e;
      c->phase_ms[k] += ms;
    }
    c->phase_steps += 1;
    c->ev_free.push_back(a);
  }
  c->ev_pool.clear();
  return cudaSuccess;
}

int log2i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

size_t esize(int prec) { return prec == SADI_PREC_FP64 ? sizeof(double) : sizeof(float); }

// The FFT engine of the context's precision: the register path where it
// serves that precision (both FP32 forms up to N' = 1024, the dense form's FFT
// part up to N' = 2048), except that explicit tiles keep the dense form on
// the shared-memory engine at lengths where the GS form runs there too.  The
// state's row pitch follows the engine (alloc_state).
bool wants_reg_path(const sadi_ctx* c) {
  if (!reg_path_supported(c->g.logNp, c->prec)) return false;
  return !(c->tiles_explicit && !reg_path_supported(c->g.logNp, SADI_PREC_FP32));
}

sadi_status alloc_state(sadi_ctx* c) {
  // row pitch of the N x N arrays: the FP32 forms on the register path pad
  // their rows to 128 bytes (16-byte vector accesses in the sweep GEMM's
  // epilogue and the row kernels), everything else keeps rows of N
  c->g.ld = (c->prec != SADI_PREC_FP64 && c->reg_path) ? (c->g.N + kPitchAlign - 1) / kPitchAlign * kPitchAlign
                                                        : c->g.N;
  const size_t nn = (size_t)c->g.ld * c->g.N;
  const size_t es = esize(c->prec);
  cudaError_t e;
  for (int k = 0; k < 2; ++k) {
    if (c->ubuf[k]) cudaFree(c->ubuf[k]);
    c->ubuf[k] = nullptr;
    CK(cudaMalloc(&c->ubuf[k], nn * es), "cudaMalloc(state)");
  }
  float** fbufs[] = {&c->ulo, &c->Chi, &c->Clo};
  for (auto b : fbufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
    if (c->prec != SADI_PREC_FP64) CK(cudaMalloc(b, nn * sizeof(float)), "cudaMalloc(state)");
  }
  if (c->phi2) cudaFree(c->phi2);
  if (c->S) cudaFree(c->S);
  if (c->W) cudaFree(c->W);
  c->phi2 = c->S = c->W = nullptr;
  CK(cudaMalloc(&c->phi2, nn * es), "cudaMalloc(phi2)");
  // the FP32 forms start their incremental remainder from an FP64 evaluation
  // (N' <= 4096), which needs the spectrum scratch at double size
  const size_t ses = (c->prec != SADI_PREC_FP64 && c->g.Np <= 4096) ? sizeof(double) : es;
  CK(cudaMalloc(&c->S, (size_t)c->g.N * c->g.Np * 2 * ses), "cudaMalloc(spectrum)");
  CK(cudaMalloc(&c->W, nn * es), "cudaMalloc(sweep)");
  if (c->g.ld != c->g.N) {
    // the padding columns stay zero: no kernel writes them, and the state
    // watchdog sums whole padded arrays
    void* pbufs[] = {c->ubuf[0], c->ubuf[1], c->ulo, c->Chi, c->Clo, c->phi2, c->W};
    for (void* b : pbufs) CK(cudaMemsetAsync(b, 0, nn * es, c->stream), "zero state");
    CK(cudaStreamSynchronize(c->stream), "zero state");
  }
  // FP32 forms whose tiles select the three-pass column convolution (the
  // default at N' = 8192): its buffers and tables (kept once allocated)
  if (c->prec != SADI_PREC_FP64 && c->tiles32.conv_cols == kConvThreePass) {
    const sadi_status s3 = ensure_conv3(c);
    if (s3 != SADI_OK) return s3;
  }
  (void)e;
  return SADI_OK;
}

// The three-pass column convolution's buffers and tables (once per context).
sadi_status ensure_conv3(sadi_ctx* c) {
  if (c->c3.ZE) return SADI_OK;
  if (c->reg_path || !conv3_supported(c->g.logNp))
    return fail(c, SADI_EINVAL, "the three-pass convolution serves FFT lengths 2048 .. 8192");
  const cudaError_t e = conv3_setup(c->g.Np, c->g.logNp, c->lpb32, &c->c3, c->stream);
  if (e == cudaErrorMemoryAllocation) return fail(c, SADI_ENOMEM, "cudaMalloc(three-pass convolution) failed");
  if (e != cudaSuccess) return cuda_fail(c, e, "three-pass convolution setup");
  return SADI_OK;
}

// The three-pass column convolution of a context, where it has one.
const Conv3* c3_of(const sadi_ctx* c) { return c->c3.ZE ? &c->c3 : nullptr; }

// Buffers, dense inverse and GEMM tensor maps of the dense-inverse form (once).
sadi_status setup_dense(sadi_ctx* c) {
  if (c->Eh) return SADI_OK;
  const int np = (c->g.N + kTcTileN - 1) / kTcTileN * kTcTileN;
  const size_t bytes = (size_t)np * np * sizeof(unsigned short);
  unsigned short** bufs[] = {&c->Eh, &c->El, &c->Bh, &c->Bl, &c->WTh, &c->WTl};
  for (auto b : bufs) {
    if (cudaMalloc(reinterpret_cast<void**>(b), bytes) != cudaSuccess)
      return fail(c, SADI_ENOMEM, "cudaMalloc(dense-inverse buffers) failed");
  }
  CK(cudaMalloc(&c->tcerr, sizeof(int)), "cudaMalloc(error flag)");
  // the per-panel counters and, after them, the GEMM launch's tile counter
  CK(cudaMalloc(&c->tcdep, sizeof(int) * (np / kTcBox + 1)), "cudaMalloc(panel counters)");
  cudaStream_t st = c->stream;
  CK(cudaMemsetAsync(c->tcerr, 0, sizeof(int), st), "error flag");
  for (int k = 2; k < 6; ++k) CK(cudaMemsetAsync(*bufs[k], 0, bytes, st), "dense padding");
  int stat = 1;
  CK(run_dense_inverse(c->a1, c->g.N, c->s, np, c->Eh, c->El, &stat, st), "dense inverse");
  if (stat != 0) return fail(c, SADI_ENOTSPD, "Durbin recursion of the N x N generator broke down");
  c->tc_x.reset(new (std::nothrow) TcInst());
  c->tc_y.reset(new (std::nothrow) TcInst());
  if (!c->tc_x || !c->tc_y) return fail(c, SADI_ENOMEM, "host allocation failed");
  // x sweep: ACC[j][i] = sum_k B[j][k] E[i][k]; y sweep: ACC[j][i] = sum_k E[j][k] W^T[i][k]
  CK(tc_set_operands(c->tc_x.get(), c->Bh, c->Bl, c->Eh, c->El, np, np, np), "tensor maps (x sweep)");
  CK(tc_set_operands(c->tc_y.get(), c->Eh, c->El, c->WTh, c->WTl, np, np, np), "tensor maps (y sweep)");
  CK(cudaStreamSynchronize(st), "dense setup");
  c->npad = np;
  return SADI_OK;
}

}  // namespace sadi_api

using namespace sadi_api;

namespace sadi_api {

// sadi_create and sadi_create_diffusion: eq 0 (wave) scales the ADI factor
// and the symbol by tau^2, eq 1 (diffusion) by tau.
sadi_status create_impl(int eq, int N, double alpha, double kappa, double tau, const double domain[2],
                        sadi_ctx** out) {
  if (!out) {
    g_create_err = "sadi_create: out is NULL";
    return SADI_EINVAL;
  }
  *out = nullptr;
  if (!domain) { g_create_err = "sadi_create: domain is NULL"; return SADI_EINVAL; }
  if (N < 1 || N > 8192) { g_create_err = "sadi_create: N must be in [1, 8192]"; return SADI_EINVAL; }
  if (!std::isfinite(alpha) || !(alpha > 1.0) || alpha > 2.0) {
    g_create_err = "sadi_create: alpha must be in (1, 2]";
    return SADI_EINVAL;
  }
  if (!std::isfinite(kappa) || !(kappa > 0.0)) { g_create_err = "sadi_create: kappa must be > 0"; return SADI_EINVAL; }
  if (!std::isfinite(tau) || !(tau > 0.0)) { g_create_err = "sadi_create: tau must be > 0"; return SADI_EINVAL; }
  if (!std::isfinite(domain[0]) || !std::isfinite(domain[1]) || !(domain[0] < domain[1])) {
    g_create_err = "sadi_create: domain must satisfy a < b (finite)";
    return SADI_EINVAL;
  }
  sadi_ctx* c = new (std::nothrow) sadi_ctx();
  if (!c) { g_create_err = "sadi_create: host allocation failed"; return SADI_ENOMEM; }
  auto bail = [&](sadi_status st) {
    g_create_err = c->err;
    free_all(c);
    delete c;
    return st;
  };
  c->eq = eq;
  c->alpha = alpha;
  c->kappa = kappa;
  c->tau = tau;
  c->a = domain[0];
  c->b = domain[1];
  c->h = (c->b - c->a) / (N + 1);
  const double tp = eq == 0 ? tau * tau : tau;   // tau^2 (wave) or tau (diffusion)
  c->s = kappa * tp / (2.0 * std::pow(c->h, alpha));
  Geom& g = c->g;
  g.N = N;
  g.ld = N;
  g.logNp = log2i(N < 8 ? 8 : N);
  g.Np = 1 << g.logNp;
  g.P = 2 * g.Np;
  g.logP = g.logNp + 1;
  g.r = g.Np - N;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaGetDevice"));
  e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamCreate"));
  c->stream = c->own_stream;
  const int Np = g.Np, P = g.P;
  const size_t nn = (size_t)N * N;
  const size_t nlpb = (size_t)(Np + 1) * 2 * Np;
  struct A { void** p; size_t bytes; } allocs[] = {
      {(void**)&c->a1, sizeof(double) * Np},
      {(void**)&c->a2d, sizeof(double) * nn},
      {(void**)&c->cgen, sizeof(double) * Np},
      {(void**)&c->lnat, sizeof(double) * (size_t)(Np + 1) * (Np + 1)},
      {(void**)&c->tw64, sizeof(double2) * P},
      {(void**)&c->tw32, sizeof(float2) * P},
      {(void**)&c->stw64, sizeof(double2) * fft_plan(g.logNp).total},
      {(void**)&c->stw32, sizeof(float2) * fft_plan(g.logNp).total},
      {(void**)&c->lpb64, sizeof(double) * nlpb},
      {(void**)&c->lpb32, sizeof(float) * nlpb},
      {(void**)&c->lamc64, sizeof(double2) * Np},
      {(void**)&c->lams64, sizeof(double2) * Np},
      {(void**)&c->lamc32, sizeof(float2) * Np},
      {(void**)&c->lams32, sizeof(float2) * Np},
      {(void**)&c->G64, sizeof(double) * ((size_t)N * g.r + 1)},
      {(void**)&c->G32, sizeof(float) * ((size_t)N * g.r + 1)},
      {(void**)&c->stage, sizeof(double) * nn},
      {(void**)&c->rtw1, sizeof(float2) * Np},
      {(void**)&c->rlreg, sizeof(float) * nlpb},
      {(void**)&c->rlamc, sizeof(float2) * Np},
      {(void**)&c->rlams, sizeof(float2) * Np},
      {(void**)&c->wd, sizeof(WdState)},
  };
  for (auto& al : allocs) {
    e = cudaMalloc(al.p, al.bytes);
    if (e != cudaSuccess) {
      c->err = std::string("sadi_create: cudaMalloc failed: ") + cudaGetErrorString(e);
      return bail(SADI_ENOMEM);
    }
  }
  cudaStream_t st = c->stream;
  if ((e = cudaMemsetAsync(c->wd, 0, sizeof(WdState), st))) return bail(cuda_fail(c, e, "watchdog record"));
  if ((e = launch_twiddles(c->tw64, c->tw32, P, st))) return bail(cuda_fail(c, e, "twiddles"));
  if ((e = launch_stage_twiddles(c->stw64, c->stw32, g.logNp, st))) return bail(cuda_fail(c, e, "stage twiddles"));
  if ((e = launch_riesz1d(c->a1, Np, alpha, st))) return bail(cuda_fail(c, e, "riesz weights"));
  const int M = (8 * Np > 1024) ? 8 * Np : 1024;
  if ((e = run_weights2d(c->a2d, g, alpha, M, c->stw64, st))) return bail(cuda_fail(c, e, "2D weights"));
  const double scale = -kappa * tp * std::pow(c->h, -alpha) / ((double)P * (double)Np);
  if ((e = run_lambda(c->a2d, g, c->stw64, c->tw64, scale, c->lnat, c->lpb64, c->lpb32, st)))
    return bail(cuda_fail(c, e, "symbol"));
  int gstat = 1;
  if ((e = run_generator(c->a1, g, c->s, c->stw64, c->tw64, c->cgen, c->lamc64, c->lams64, c->lamc32, c->lams32, c->G64,
                         c->G32, &gstat, st)))
    return bail(cuda_fail(c, e, "generator"));
  if (gstat != 0) {
    c->err = "sadi_create: Durbin recursion broke down (H not numerically SPD)";
    return bail(SADI_ENOTSPD);
  }
  c->reg_path = wants_reg_path(c);
  if ((e = run_reg_tables(g, c->lnat, scale, c->lamc64, c->lams64, c->rtw1, c->rlreg, c->rlamc, c->rlams, st)))
    return bail(cuda_fail(c, e, "register-path tables"));
  if ((e = step_setup_attributes<float>())) return bail(cuda_fail(c, e, "kernel attributes"));
  if ((e = step_setup_attributes<double>())) return bail(cuda_fail(c, e, "kernel attributes"));
  c->tiles64 = default_tiles<double>(Np, N);
  c->tiles32 = default_tiles<float>(Np, N);
  sadi_status sst = alloc_state(c);
  if (sst != SADI_OK) return bail(sst);
  if ((e = cudaStreamSynchronize(st))) return bail(cuda_fail(c, e, "setup"));
  *out = c;
  return SADI_OK;
}

}  // namespace sadi_api

extern "C" {

sadi_status sadi_create(int N, double alpha, double kappa, double tau, const double domain[2], sadi_ctx** out) {
  return create_impl(0, N, alpha, kappa, tau, domain, out);
}

sadi_status sadi_create_diffusion(int N, double alpha, double kappa, double tau, const double domain[2],
                                  sadi_ctx** out) {
  return create_impl(1, N, alpha, kappa, tau, domain, out);
}

sadi_status sadi_get_equation(const sadi_ctx* c, int* eq) {
  if (!c || !eq) return SADI_EINVAL;
  *eq = c->eq;
  return SADI_OK;
}

sadi_status sadi_set_options(sadi_ctx* c, int g, int prec) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (c->initialized) return fail(c, SADI_ESTATE, "sadi_set_options must precede sadi_set_initial");
  if (g < SADI_G_ZERO || g > SADI_G_GENERAL) return fail(c, SADI_EINVAL, "g must be 0, 1, 2 or 3");
  if (prec != SADI_PREC_FP64 && prec != SADI_PREC_FP32 && prec != SADI_PREC_FP32_DENSE)
    return fail(c, SADI_EINVAL, "prec must be 0, 1 or 2");
  if (prec == SADI_PREC_FP64 && c->g.N > 4096)
    return fail(c, SADI_EUNSUPPORTED, "the FP64 step path supports N <= 4096");
  if (prec == SADI_PREC_FP32_DENSE && c->g.N > 8192)
    return fail(c, SADI_EUNSUPPORTED, "the dense-inverse form supports N <= 8192");
  if (prec != c->prec && c->F) return fail(c, SADI_ESTATE, "set the precision before sadi_set_source");
  if (prec == SADI_PREC_FP32_DENSE) {
    const sadi_status ds = setup_dense(c);
    if (ds != SADI_OK) return ds;
  }
  c->gkind = g;
  if (prec != c->prec) {
    if (c->F) return fail(c, SADI_ESTATE, "set the precision before sadi_set_source");
    c->prec = prec;
    c->reg_path = wants_reg_path(c);
    if (c->Fconv) cudaFree(c->Fconv);
    c->Fconv = nullptr;
    return alloc_state(c);
  }
  return SADI_OK;
}

sadi_status sadi_set_nonlinearity(sadi_ctx* c, double c1, double c3, double cs) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (c->initialized) return fail(c, SADI_ESTATE, "sadi_set_nonlinearity must precede sadi_set_initial");
  if (!std::isfinite(c1) || !std::isfinite(c3) || !std::isfinite(cs))
    return fail(c, SADI_EINVAL, "the coefficients of g must be finite");
  c->gc[0] = c1;
  c->gc[1] = c3;
  c->gc[2] = cs;
  c->gkind = SADI_G_GENERAL;
  return SADI_OK;
}

sadi_status sadi_get_options(const sadi_ctx* c, int* g, int* prec) {
  if (!c) return SADI_EINVAL;
  if (g) *g = c->gkind;
  if (prec) *prec = c->prec;
  return SADI_OK;
}

sadi_status sadi_set_source(sadi_ctx* c, const double* F, double omega, double phase) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (!std::isfinite(omega) || !std::isfinite(phase)) return fail(c, SADI_EINVAL, "omega and phase must be finite");
  if (c->F) {
    CK(cudaStreamSynchronize(c->stream), "sadi_set_source");
    cudaFree(c->F);
    c->F = nullptr;
  }
  if (!F) return SADI_OK;
  const int N = c->g.N, ld = c->g.ld;
  const size_t nn = (size_t)N * N;
  CK(cudaMalloc(&c->F, (size_t)ld * N * esize(c->prec)), "cudaMalloc(source)");
  cudaStream_t st = c->stream;
  CK(stage_acquire(c), "order after the last asynchronous read");
  CK(cudaMemcpyAsync(c->stage, F, nn * sizeof(double), cudaMemcpyHostToDevice, st), "copy source");
  if (c->prec == SADI_PREC_FP64)
    CK(cudaMemcpyAsync(c->F, c->stage, nn * sizeof(double), cudaMemcpyDeviceToDevice, st), "source");
  else
    CK(launch_convert_d2f(c->stage, static_cast<float*>(c->F), N, N, N, ld, st), "source convert");
  CK(cudaStreamSynchronize(st), "sadi_set_source");
  c->f_omega = omega;
  c->f_phase = phase;
  return SADI_OK;
}

sadi_status sadi_set_stream(sadi_ctx* c, void* stream) {
  if (!c) return SADI_EINVAL;
  c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own_stream;
  return SADI_OK;
}

sadi_status sadi_set_initial(sadi_ctx* c, const double* phi1, const double* phi2) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (!phi1) return fail(c, SADI_EINVAL, "phi1 is NULL");
  if (c->eq == 1 && phi2) return fail(c, SADI_EINVAL, "the diffusion equation has no phi2 (pass NULL)");
  if (c->prec == SADI_PREC_FP64 && c->g.N > 4096)
    return fail(c, SADI_EUNSUPPORTED, "the FP64 step path supports N <= 4096; select SADI_PREC_FP32");
  const int N = c->g.N, ld = c->g.ld;
  const size_t nn = (size_t)N * N;
  cudaStream_t st = c->stream;
  c->cur = 0;
  CK(stage_acquire(c), "order after the last asynchronous read");
  CK(cudaMemcpyAsync(c->stage, phi1, nn * sizeof(double), cudaMemcpyHostToDevice, st), "copy phi1");
  if (c->prec == SADI_PREC_FP64) {
    CK(cudaMemcpyAsync(c->ubuf[0], c->stage, nn * sizeof(double), cudaMemcpyDeviceToDevice, st), "phi1");
  } else {
    CK(launch_split_d2ff(c->stage, static_cast<float*>(c->ubuf[0]), c->ulo, N, N, N, ld, st), "phi1 split");
    CK(cudaMemsetAsync(c->ubuf[1], 0, (size_t)ld * N * sizeof(float), st), "increment zero");
    // starting remainder C^0 = -kappa tau^2 L_h phi1: FP64 where the FP64
    // engine applies (N' <= 4096), else FP32 from the hi part
    if (c->g.Np <= 4096) {
      StepTables<double> tb{c->stw64, c->tw64, c->lpb64, c->lams64, c->lamc64, c->G64};
      CK(launch_remainder<double>(c->g, tb, default_tiles<double>(c->g.Np, c->g.N), c->stage, c->S, c->Chi, c->Clo, st),
         "starting remainder");
    } else {
      StepTables<float> tb{c->stw32, c->tw32, c->lpb32, c->lams32, c->lamc32, c->G32, c3_of(c)};
      CK(launch_remainder<float>(c->g, tb, default_tiles<float>(c->g.Np, c->g.N), static_cast<const float*>(c->ubuf[0]),
                                 c->S, c->Chi, c->Clo, st),
         "starting remainder");
    }
  }
  if (phi2) {
    CK(cudaMemcpyAsync(c->stage, phi2, nn * sizeof(double), cudaMemcpyHostToDevice, st), "copy phi2");
    if (c->prec == SADI_PREC_FP64)
      CK(cudaMemcpyAsync(c->phi2, c->stage, nn * sizeof(double), cudaMemcpyDeviceToDevice, st), "phi2");
    else
      CK(launch_convert_d2f(c->stage, static_cast<float*>(c->phi2), N, N, N, ld, st), "phi2 convert");
  } else {
    CK(cudaMemsetAsync(c->phi2, 0, (size_t)ld * N * esize(c->prec), st), "phi2 zero");
  }
  CK(cudaMemsetAsync(c->wd, 0, sizeof(WdState), st), "watchdog record");
  CK(cudaStreamSynchronize(st), "set_initial");
  c->n = 0;
  c->initialized = true;
  return SADI_OK;
}

}  // extern "C"

namespace sadi_api {

// Profiling events for one step of ctx (nullptr when not profiling).
sadi_status next_events(sadi_ctx* c, cudaEvent_t** out) {
  *out = nullptr;
  if (!c->profiling) return SADI_OK;
  if (c->ev_pool.size() >= 512) CK(fold_events(c), "profile events");
  if (c->ev_free.empty()) {
    std::array<cudaEvent_t, 5> a{};
    for (auto& e : a) CK(cudaEventCreate(&e), "cudaEventCreate");
    c->ev_free.push_back(a);
  }
  c->ev_pool.push_back(c->ev_free.back());
  c->ev_free.pop_back();
  *out = c->ev_pool.back().data();
  return SADI_OK;
}

// B^n scalars of the next step of c (time level n): g, the source term (the
// field of sadi_step_source, else the separable one) and the n = 0 switch
RhsParams rhs_of(const sadi_ctx* c, long long n) {
  RhsParams rp{};
  rp.eq = c->eq;
  rp.tau = c->tau;
  rp.tau2 = c->eq == 0 ? c->tau * c->tau : c->tau;
  rp.g = c->gkind;
  rp.first = n == 0 ? 1 : 0;
  if (c->F_step) {
    rp.F = c->F_step;
    rp.fsc = 1.0;
  } else if (c->F) {
    // the wave step samples f at t_n, the diffusion step at t_{n+1/2}
    const double t = ((double)n + (c->eq == 0 ? 0.0 : 0.5)) * c->tau;
    rp.F = c->F;
    rp.fsc = std::cos(c->f_omega * t + c->f_phase);
  }
  rp.gc1 = c->gc[0];
  rp.gc3 = c->gc[1];
  rp.gcs = c->gc[2];
  return rp;
}

RegInst reg_inst(const sadi_ctx* c) {
  RegInst r{};
  r.tw1 = c->rtw1;
  r.tw = c->tw32;
  r.lam_s = c->rlams;
  r.lam_c = c->rlamc;
  r.lreg = c->rlreg;
  r.G = c->G32;
  r.u_hi = static_cast<float*>(c->ubuf[0]);
  r.u_d = static_cast<float*>(c->ubuf[1]);
  r.u_lo = c->ulo;
  r.phi2 = static_cast<const float*>(c->phi2);
  r.S = static_cast<float2*>(c->S);
  r.W = static_cast<float*>(c->W);
  r.N = c->g.N;
  r.ld = c->g.ld;
  r.r = c->g.r;
  r.tau = (float)c->tau;
  r.tau2 = (float)(c->eq == 0 ? c->tau * c->tau : c->tau);
  r.eq = c->eq;
  r.gkind = c->gkind;
  r.first = c->n == 0 ? 1 : 0;
  const RhsParams rp = rhs_of(c, c->n);
  r.F = static_cast<const float*>(rp.F);
  r.fsc = (float)rp.fsc;
  r.gc1 = (float)c->gc[0];
  r.gc3 = (float)c->gc[1];
  r.gcs = (float)c->gc[2];
  r.C_hi = c->Chi;
  r.C_lo = c->Clo;
  r.Bh = c->Bh;
  r.Bl = c->Bl;
  r.ldp = c->npad;
  r.dep = c->prec == SADI_PREC_FP32_DENSE ? c->tcdep : nullptr;
  r.ndep = c->npad / kTcBox + 1;
  return r;
}

bool uses_reg_path(const sadi_ctx* c) { return c->prec == SADI_PREC_FP32 && c->reg_path; }
bool is_dense(const sadi_ctx* c) { return c->prec == SADI_PREC_FP32_DENSE; }

// One step of a context on the shared-memory engine (FP64, or FP32 N' > 1024),
// on stream st.
sadi_status step_smem(sadi_ctx* c, cudaEvent_t* ev, cudaStream_t st) {
  const RhsParams rp = rhs_of(c, c->n);
  cudaError_t e;
  if (c->prec == SADI_PREC_FP64) {
    void* ucur = c->ubuf[c->cur];
    void* uoth = c->ubuf[1 - c->cur];
    StepTables<double> tb{c->stw64, c->tw64, c->lpb64, c->lams64, c->lamc64, c->G64};
    e = launch_step<double>(c->g, tb, c->tiles64, rp, static_cast<const double*>(ucur), static_cast<double*>(uoth),
                            static_cast<double*>(uoth), nullptr, static_cast<const double*>(c->phi2), c->S,
                            static_cast<double*>(c->W), st, ev);
  } else {
    StepTables<float> tb{c->stw32, c->tw32, c->lpb32, c->lams32, c->lamc32, c->G32, c3_of(c)};
    float* hi = static_cast<float*>(c->ubuf[0]);
    e = launch_step<float>(c->g, tb, c->tiles32, rp, hi, static_cast<float*>(c->ubuf[1]), hi, c->ulo,
                           static_cast<const float*>(c->phi2), c->S, static_cast<float*>(c->W), st, ev, c->Chi,
                           c->Clo);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
  if (c->prec == SADI_PREC_FP64) c->cur = 1 - c->cur;
  c->n += 1;
  return SADI_OK;
}

// One step of up to kMaxBatch register-path contexts with equal FFT length,
// in one launch per kernel on stream st.
sadi_status step_reg_group(sadi_ctx* const* cs, int count, cudaStream_t st_) {
  static thread_local RegBatch b;
  b.count = count;
  int max_n = 0;
  for (int k = 0; k < count; ++k) {
    b.in[k] = reg_inst(cs[k]);
    if (cs[k]->g.N > max_n) max_n = cs[k]->g.N;
  }
  sadi_ctx* c = cs[0];
  cudaEvent_t* ev = nullptr;
  sadi_status st = next_events(c, &ev);
  if (st != SADI_OK) return st;
  const cudaError_t e = launch_step_reg(b, c->g.logNp, max_n, st_, ev);
  if (e != cudaSuccess) {
    for (int k = 0; k < count; ++k) cuda_fail(cs[k], e, "step launch");
    return SADI_ECUDA;
  }
  for (int k = 0; k < count; ++k) cs[k]->n += 1;
  return SADI_OK;
}

// One step of count dense-form contexts with equal FFT length on stream st:
// the FFT part batched (register path, N' <= 2048), or one member after
// another (shared-memory engine), then
// the x-sweep and y-sweep GEMMs batched (at most kTcMaxBatch per launch).
sadi_status step_dense_group(sadi_ctx* const* cs, int count, cudaStream_t st_) {
  sadi_ctx* c = cs[0];
  cudaEvent_t* ev = nullptr;
  sadi_status st = next_events(c, &ev);
  if (st != SADI_OK) return st;
  cudaError_t e;
  if (c->reg_path) {
    static thread_local RegBatch b;
    b.count = count;
    int max_n = 0;
    for (int k = 0; k < count; ++k) {
      b.in[k] = reg_inst(cs[k]);
      if (cs[k]->g.N > max_n) max_n = cs[k]->g.N;
    }
    e = launch_step_reg(b, c->g.logNp, max_n, st_, ev, true);
  } else {
    // shared-memory engine: the FFT part one member after another (a
    // profiled group has one member, so the events time its kernels), then
    // the sweeps of all members batched below
    if (ev && count != 1) return fail(c, SADI_EINVAL, "internal: profiled shared-memory dense group of more than one");
    e = cudaSuccess;
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
      sadi_ctx* ck = cs[k];
      const RhsParams rp = rhs_of(ck, ck->n);
      StepTables<float> tb{ck->stw32, ck->tw32, ck->lpb32, ck->lams32, ck->lamc32, ck->G32, c3_of(ck)};
      e = launch_dense_rows(ck->g, tb, ck->tiles32, rp, static_cast<const float*>(ck->ubuf[0]),
                            static_cast<const float*>(ck->ubuf[1]), static_cast<const float*>(ck->phi2), ck->S,
                            static_cast<float*>(ck->W), ck->Chi, ck->Clo, ck->Bh, ck->Bl, ck->npad, st_, ev);
    }
  }
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[3], st_);
  // Both sweeps of up to kTcMaxBatch / 2 members per launch: the x-sweep
  // problems first, then the y-sweep problems, whose tiles wait per
  // 128-column panel for the x-sweep tiles that store W (and its transposed
  // split) there, so that the y sweep of one member runs beside the x sweep
  // of the next.
  static thread_local TcBatch tb;
  constexpr int kPer = kTcMaxBatch / 2;
  for (int k0 = 0; e == cudaSuccess && k0 < count; k0 += kPer) {
    const int m = count - k0 < kPer ? count - k0 : kPer;
    tb.count = 2 * m;
    tb.wait_ns = 0;
    tb.tile_next = cs[k0]->tcdep + cs[k0]->npad / kTcBox;
    // register path: the B^n kernel zeroed the counters, and the first GEMM
    // follows it directly in the stream (unless profiling events sit
    // between), so it is launched as its programmatic dependent; otherwise
    // the counters are zeroed here
    tb.pdl = (c->reg_path && k0 == 0 && !ev) ? 1 : 0;
    for (int k = 0; k < m && e == cudaSuccess; ++k) {
      const sadi_ctx* ck = cs[k0 + k];
      if (!c->reg_path) e = cudaMemsetAsync(ck->tcdep, 0, sizeof(int) * (ck->npad / kTcBox + 1), st_);
      for (int pass = 0; pass < 2; ++pass) {
        TcInst& in = tb.in[pass * m + k];
        in = pass == 0 ? *ck->tc_x : *ck->tc_y;
        TcEpi& ep = in.e;
        ep = TcEpi{};
        ep.m_valid = ep.n_valid = ck->g.N;
        ep.C = static_cast<float*>(ck->W);
        ep.ldc = ck->g.ld;
        ep.err = ck->tcerr;
        if (pass == 0) {
          ep.mode = kTcSweepX;
          ep.t_hi = ck->WTh;
          ep.t_lo = ck->WTl;
          ep.ldt = ck->npad;
          in.dep_wait = nullptr;
          in.dep_need = 0;
          in.dep_signal = ck->tcdep;
        } else {
          ep.mode = kTcSweepY;
          ep.u_hi = static_cast<float*>(ck->ubuf[0]);
          ep.u_lo = ck->ulo;
          ep.u_d = static_cast<float*>(ck->ubuf[1]);
          ep.ldu = ck->g.ld;
          ep.first = ck->n == 0 ? 1 : 0;
          in.dep_wait = ck->tcdep;
          in.dep_need = ck->tc_x->tiles_m;   // x-sweep tiles per column panel
          in.dep_signal = nullptr;
          if (ck->dbg_expire_ns > 0) {
            // sadi_debug_expire_waits: a panel count that no x-sweep tile
            // reaches, and a short limit for every wait of the launch
            in.dep_need = ck->tc_x->tiles_m + 1;
            tb.wait_ns = (unsigned long long)ck->dbg_expire_ns;
          }
        }
      }
    }
    for (int k = 0; k < 2 * m; ++k) tb.in[k].e.vec = tc_vec_ok(tb.in[k].e) ? 1 : 0;
    for (int k = 0; k < m; ++k) cs[k0 + k]->dbg_expire_ns = 0;
    if (e == cudaSuccess) e = launch_tc_gemm(tb, cs[k0]->tcerr, st_);
  }
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[4], st_);
  if (e != cudaSuccess) {
    for (int k = 0; k < count; ++k) cuda_fail(cs[k], e, "dense step launch");
    return SADI_ECUDA;
  }
  for (int k = 0; k < count; ++k) cs[k]->n += 1;
  return SADI_OK;
}

// The tensor-core sweeps' device error flag (a bounded wait ran out): the
// context's state is then invalid.
sadi_status check_gemm_flag(sadi_ctx* c) {
  if (!c->tcerr) return SADI_OK;
  int flag = 0;
  CK(cudaMemcpy(&flag, c->tcerr, sizeof(int), cudaMemcpyDeviceToHost), "error flag");
  if (flag) {
    c->broken = true;
    return fail(c, SADI_ETIMEOUT, "a bounded wait in a tensor-core sweep ran out; the state is invalid");
  }
  return SADI_OK;
}

cudaError_t stage_acquire(sadi_ctx* c) {
  return c->ev_copied ? cudaStreamWaitEvent(c->stream, c->ev_copied, 0) : cudaSuccess;
}

sadi_status check_steppable(sadi_ctx* c) {
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (!c->initialized) return fail(c, SADI_ESTATE, "sadi_step before sadi_set_initial");
  return SADI_OK;
}

}  // namespace sadi_api

extern "C" {

sadi_status sadi_step(sadi_ctx* c, int nsteps) {
  if (!c) return SADI_EINVAL;
  sadi_status st = check_steppable(c);
  if (st != SADI_OK) return st;
  if (nsteps < 0) return fail(c, SADI_EINVAL, "nsteps must be >= 0");
  const long long n_before = c->n;
  for (int it = 0; it < nsteps; ++it) {
    if (is_dense(c)) {
      st = step_dense_group(&c, 1, c->stream);
    } else if (uses_reg_path(c)) {
      st = step_reg_group(&c, 1, c->stream);
    } else {
      cudaEvent_t* ev = nullptr;
      st = next_events(c, &ev);
      if (st == SADI_OK) st = step_smem(c, ev, c->stream);
    }
    if (st != SADI_OK) return st;
  }
  return watchdog_after(c, n_before, c->stream);
}

}  // extern "C"

namespace sadi_api {

sadi_status batch_issue(sadi_ctx** ctxs, int count, int nsteps) {
  // group register-path contexts by FFT length (insertion order kept)
  // (dense-form contexts on the register path form their own groups), and
  // dense-form contexts on the shared-memory engine by FFT length too (their
  // FFT kernels run one member after another, their sweep GEMMs batched; a
  // profiled one steps alone, so that its events time its own kernels)
  std::vector<std::vector<sadi_ctx*>> groups;
  std::vector<sadi_ctx*> others;
  for (int k = 0; k < count; ++k) {
    sadi_ctx* c = ctxs[k];
    const bool dense_reg = is_dense(c) && c->reg_path;
    const bool dense_smem = is_dense(c) && !c->reg_path && !c->profiling;
    if (!uses_reg_path(c) && !dense_reg && !dense_smem) {
      others.push_back(c);
      continue;
    }
    bool placed = false;
    for (auto& gr : groups)
      if (gr[0]->g.logNp == c->g.logNp && is_dense(gr[0]) == is_dense(c) && gr[0]->reg_path == c->reg_path &&
          (int)gr.size() < kMaxBatch) {
        gr.push_back(c);
        placed = true;
        break;
      }
    if (!placed) groups.push_back({c});
  }
  // everything runs on the first context's stream, ordered after and before
  // the pending work of the other contexts' streams
  cudaStream_t s0 = ctxs[0]->stream;
  for (int k = 0; k < count; ++k) {
    sadi_ctx* c = ctxs[k];
    if (c->stream == s0) continue;
    if (!c->order_ev) CK(cudaEventCreateWithFlags(&c->order_ev, cudaEventDisableTiming), "cudaEventCreate");
    CK(cudaEventRecord(c->order_ev, c->stream), "cudaEventRecord");
    CK(cudaStreamWaitEvent(s0, c->order_ev, 0), "cudaStreamWaitEvent");
  }
  for (int it = 0; it < nsteps; ++it) {
    for (auto& gr : groups) {
      sadi_status st = is_dense(gr[0]) ? step_dense_group(gr.data(), (int)gr.size(), s0)
                                       : step_reg_group(gr.data(), (int)gr.size(), s0);
      if (st != SADI_OK) return st;
    }
    for (sadi_ctx* c : others) {
      if (is_dense(c)) {
        sadi_status st = step_dense_group(&c, 1, s0);
        if (st != SADI_OK) return st;
        continue;
      }
      cudaEvent_t* ev = nullptr;
      sadi_status st = next_events(c, &ev);
      if (st == SADI_OK) st = step_smem(c, ev, s0);
      if (st != SADI_OK) return st;
    }
  }
  sadi_ctx* c0 = ctxs[0];
  bool any_other = false;
  for (int k = 0; k < count; ++k) any_other |= ctxs[k]->stream != s0;
  if (any_other) {
    sadi_ctx* c = c0;
    if (!c0->order_ev) CK(cudaEventCreateWithFlags(&c0->order_ev, cudaEventDisableTiming), "cudaEventCreate");
    CK(cudaEventRecord(c0->order_ev, s0), "cudaEventRecord");
    for (int k = 0; k < count; ++k)
      if (ctxs[k]->stream != s0) CK(cudaStreamWaitEvent(ctxs[k]->stream, c0->order_ev, 0), "cudaStreamWaitEvent");
  }
  return SADI_OK;
}

sadi_status zero_initial(sadi_ctx* c) {
  const size_t nn = (size_t)c->g.ld * c->g.N;
  const size_t es = esize(c->prec);
  cudaStream_t st = c->stream;
  void* bufs[] = {c->ubuf[0], c->ubuf[1], c->phi2};
  for (void* b : bufs)
    if (b) CK(cudaMemsetAsync(b, 0, nn * es, st), "zero state");
  float* fb[] = {c->ulo, c->Chi, c->Clo};
  for (float* b : fb)
    if (b) CK(cudaMemsetAsync(b, 0, nn * sizeof(float), st), "zero state");
  CK(cudaMemsetAsync(c->wd, 0, sizeof(WdState), st), "watchdog record");
  c->cur = 0;
  c->n = 0;
  c->initialized = true;
  return SADI_OK;
}

sadi_status watchdog_after(sadi_ctx* c, long long n_before, cudaStream_t st) {
  if (c->wd_every <= 0 || c->n / c->wd_every == n_before / c->wd_every) return SADI_OK;
  const size_t nn = (size_t)c->g.ld * c->g.N;   // padding columns (zero) included
  const bool f64 = c->prec == SADI_PREC_FP64;
  // FP64: u^n; FP32 forms: the hi part of the double-float pair, finite
  // exactly when u^n is
  CK(launch_watchdog(f64 ? c->ubuf[c->cur] : c->ubuf[0], f64, nn, c->wd, c->n, st), "watchdog");
  return SADI_OK;
}

sadi_status check_watchdog(sadi_ctx* c) {
  WdState h;
  CK(cudaMemcpy(&h, c->wd, offsetof(WdState, ticket), cudaMemcpyDeviceToHost), "watchdog record");
  if (h.nonfinite) {
    c->initialized = false;
    return fail(c, SADI_ENONFINITE,
                "the watchdog found a non-finite value in u^n at step " + std::to_string(h.nonfinite_step) +
                    "; set new initial data (sadi_set_initial or sadi_load_state) to continue");
  }
  return SADI_OK;
}

}  // namespace sadi_api

extern "C" {

sadi_status sadi_batch_step(sadi_ctx** ctxs, int count, int nsteps) {
  if (!ctxs || count < 1 || nsteps < 0) return SADI_EINVAL;
  for (int k = 0; k < count; ++k) {
    if (!ctxs[k]) return SADI_EINVAL;
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return fail(ctxs[k], SADI_EINVAL, "a context appears twice in the batch");
    sadi_status st = check_steppable(ctxs[k]);
    if (st != SADI_OK) return st;
  }
  std::vector<long long> n_before(count);
  for (int k = 0; k < count; ++k) n_before[k] = ctxs[k]->n;
  sadi_status st = batch_issue(ctxs, count, nsteps);
  for (int k = 0; k < count && st == SADI_OK; ++k) {
    // on the stream of the context, after the batch (batch_issue ordered it)
    st = watchdog_after(ctxs[k], n_before[k], ctxs[k]->stream);
  }
  return st;
}

sadi_status sadi_get(sadi_ctx* c, double* u_out, long long* n_out) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (!c->initialized) return fail(c, SADI_ESTATE, "sadi_get before sadi_set_initial");
  if (!u_out) return fail(c, SADI_EINVAL, "u_out is NULL");
  const size_t nn = (size_t)c->g.N * c->g.N;
  cudaStream_t st = c->stream;
  if (c->prec == SADI_PREC_FP64) {
    CK(cudaMemcpyAsync(u_out, c->ubuf[c->cur], nn * sizeof(double), cudaMemcpyDeviceToHost, st), "copy u");
  } else {
    CK(stage_acquire(c), "order after the last asynchronous read");
    CK(launch_join_ff2d(static_cast<const float*>(c->ubuf[0]), c->ulo, c->stage, c->g.N, c->g.N, c->g.ld, c->g.N,
                        st),
       "u join");
    CK(cudaMemcpyAsync(u_out, c->stage, nn * sizeof(double), cudaMemcpyDeviceToHost, st), "copy u");
  }
  CK(cudaStreamSynchronize(st), "sadi_get");
  sadi_status es = check_gemm_flag(c);
  if (es == SADI_OK) es = check_watchdog(c);
  if (es != SADI_OK) return es;
  if (n_out) *n_out = c->n;
  return SADI_OK;
}

sadi_status sadi_get_async(sadi_ctx* c, double* u_out) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (!c->initialized) return fail(c, SADI_ESTATE, "sadi_get_async before sadi_set_initial");
  if (!u_out) return fail(c, SADI_EINVAL, "u_out is NULL");
  if (!c->copy_stream) {
    CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "cudaStreamCreate(copies)");
    CK(cudaEventCreateWithFlags(&c->ev_staged, cudaEventDisableTiming), "cudaEventCreate");
    CK(cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming), "cudaEventCreate");
  }
  const size_t nn = (size_t)c->g.N * c->g.N;
  cudaStream_t st = c->stream;
  // u^n into the staging buffer on the step stream (after the previous copy
  // out of it), then the copy to the host on the copy stream, so that later
  // steps on the step stream run while it is in flight
  CK(stage_acquire(c), "order after the last asynchronous read");
  if (c->prec == SADI_PREC_FP64)
    CK(cudaMemcpyAsync(c->stage, c->ubuf[c->cur], nn * sizeof(double), cudaMemcpyDeviceToDevice, st), "stage u");
  else
    CK(launch_join_ff2d(static_cast<const float*>(c->ubuf[0]), c->ulo, c->stage, c->g.N, c->g.N, c->g.ld, c->g.N,
                        st),
       "u join");
  CK(cudaEventRecord(c->ev_staged, st), "cudaEventRecord");
  CK(cudaStreamWaitEvent(c->copy_stream, c->ev_staged, 0), "cudaStreamWaitEvent");
  CK(cudaMemcpyAsync(u_out, c->stage, nn * sizeof(double), cudaMemcpyDeviceToHost, c->copy_stream), "copy u");
  CK(cudaEventRecord(c->ev_copied, c->copy_stream), "cudaEventRecord");
  return SADI_OK;
}

sadi_status sadi_wait(sadi_ctx* c) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  CK(cudaStreamSynchronize(c->stream), "sadi_wait");
  if (c->copy_stream) CK(cudaStreamSynchronize(c->copy_stream), "sadi_wait (copies)");
  const sadi_status es = check_gemm_flag(c);
  return es != SADI_OK || !c->initialized ? es : check_watchdog(c);
}

sadi_status sadi_get_device(sadi_ctx* c, void* dst, int dtype) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (!c->initialized) return fail(c, SADI_ESTATE, "sadi_get_device before sadi_set_initial");
  if (!dst) return fail(c, SADI_EINVAL, "dst is NULL");
  if (dtype != 0 && dtype != 1) return fail(c, SADI_EINVAL, "dtype must be 0 (double) or 1 (float)");
  const int N = c->g.N;
  const size_t nn = (size_t)N * N;
  cudaStream_t st = c->stream;
  const void* src = c->ubuf[c->cur];
  if (c->prec == SADI_PREC_FP64) {
    if (dtype == 0) CK(cudaMemcpyAsync(dst, src, nn * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy");
    else
      CK(launch_convert_d2f(static_cast<const double*>(src), static_cast<float*>(dst), N, N, N, N, st), "convert");
  } else {
    const float* hi = static_cast<const float*>(c->ubuf[0]);
    const int ld = c->g.ld;
    if (dtype == 1) CK(launch_join_ff2f(hi, c->ulo, static_cast<float*>(dst), N, N, ld, N, st), "join");
    else CK(launch_join_ff2d(hi, c->ulo, static_cast<double*>(dst), N, N, ld, N, st), "join");
  }
  return SADI_OK;
}

sadi_status sadi_get_setup(sadi_ctx* c, int which, double* out, size_t count) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (!out) return fail(c, SADI_EINVAL, "out is NULL");
  const double* src = nullptr;
  size_t n = 0;
  const size_t N = c->g.N, Np = c->g.Np;
  switch (which) {
    case 0: src = c->a1; n = N; break;
    case 1: src = c->a2d; n = N * N; break;
    case 2: src = c->cgen; n = Np; break;
    case 3: src = c->lnat; n = (Np + 1) * (Np + 1); break;
    case 4: {
      if (!c->Eh) return fail(c, SADI_ESTATE, "which = 4 needs SADI_PREC_FP32_DENSE selected");
      if (count != N * N) return fail(c, SADI_EINVAL, "count does not match the table size");
      const size_t np = (size_t)c->npad;
      std::vector<unsigned short> hi(np * np), lo(np * np);
      CK(cudaMemcpyAsync(hi.data(), c->Eh, np * np * 2, cudaMemcpyDeviceToHost, c->stream), "copy E");
      CK(cudaMemcpyAsync(lo.data(), c->El, np * np * 2, cudaMemcpyDeviceToHost, c->stream), "copy E");
      CK(cudaStreamSynchronize(c->stream), "sadi_get_setup");
      auto f = [](unsigned short b) {
        const unsigned int w = (unsigned int)b << 16;
        float v;
        std::memcpy(&v, &w, sizeof(v));
        return (double)v;
      };
      for (size_t i = 0; i < N; ++i)
        for (size_t j = 0; j < N; ++j) out[i * N + j] = f(hi[i * np + j]) + f(lo[i * np + j]);
      return SADI_OK;
    }
    default: return fail(c, SADI_EINVAL, "which must be 0..4");
  }
  if (count != n) return fail(c, SADI_EINVAL, "count does not match the table size");
  CK(cudaMemcpyAsync(out, src, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy setup table");
  CK(cudaStreamSynchronize(c->stream), "sadi_get_setup");
  return SADI_OK;
}

sadi_status sadi_get_info(const sadi_ctx* c, int* fft_len, int* border_rank) {
  if (!c) return SADI_EINVAL;
  if (fft_len) *fft_len = c->g.Np;
  if (border_rank) *border_rank = c->g.r;
  return SADI_OK;
}

sadi_status sadi_set_tiles(sadi_ctx* c, int rows, int conv_cols, int solve_cols) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  Tiles t{rows, conv_cols, solve_cols};
  const bool f64 = c->prec == SADI_PREC_FP64;
  const bool dflt = rows == 0 && conv_cols == 0 && solve_cols == 0;
  if (dflt) t = f64 ? default_tiles<double>(c->g.Np, c->g.N) : default_tiles<float>(c->g.Np, c->g.N);
  const bool ok = f64 ? tiles_valid<double>(c->g, t) : tiles_valid<float>(c->g, t);
  if (!ok) return fail(c, SADI_EINVAL, "tile sizes invalid for this N and precision");
  // the engine these tiles select (the dense form at N' = 2048: explicit
  // tiles the shared-memory engine, the defaults the register path); the
  // FP64 path's tiles leave the FP32 forms' choice alone
  const bool was_explicit = c->tiles_explicit;
  const bool expl = f64 ? was_explicit : !dflt;
  c->tiles_explicit = expl;
  const bool reg = wants_reg_path(c);
  c->tiles_explicit = was_explicit;
  if (!f64 && t.conv_cols == kConvThreePass && (reg || !conv3_supported(c->g.logNp)))
    return fail(c, SADI_EINVAL, "the three-pass convolution serves FFT lengths 2048 .. 8192");
  if (reg != c->reg_path) {
    if (c->initialized || c->F)
      return fail(c, SADI_ESTATE,
                  "tiles that change the FFT engine (dense form, N' = 2048) must precede sadi_set_initial and "
                  "sadi_set_source");
    c->tiles_explicit = expl;
    c->reg_path = reg;
    const sadi_status sa = alloc_state(c);
    if (sa != SADI_OK) return sa;
  }
  c->tiles_explicit = expl;
  if (!f64 && t.conv_cols == kConvThreePass) {
    const sadi_status s3 = ensure_conv3(c);
    if (s3 != SADI_OK) return s3;
  }
  if (f64) c->tiles64 = t;
  else c->tiles32 = t;
  return SADI_OK;
}

sadi_status sadi_get_tiles(const sadi_ctx* c, int tiles[3]) {
  if (!c || !tiles) return SADI_EINVAL;
  const Tiles& t = c->prec == SADI_PREC_FP64 ? c->tiles64 : c->tiles32;
  tiles[0] = t.rows;
  tiles[1] = t.conv_cols;
  tiles[2] = t.solve_cols;
  return SADI_OK;
}

sadi_status sadi_profile(sadi_ctx* c, int enable) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (enable && !c->profiling) {
    CK(fold_events(c), "profile events");
    for (double& v : c->phase_ms) v = 0.0;
    c->phase_steps = 0;
  }
  c->profiling = enable != 0;
  return SADI_OK;
}

sadi_status sadi_get_phase_times(sadi_ctx* c, double ms[4], long long* nsteps) {
  if (!c) return SADI_EINVAL;
  if (!ms) return fail(c, SADI_EINVAL, "ms is NULL");
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  CK(fold_events(c), "profile events");
  for (int k = 0; k < 4; ++k) {
    ms[k] = c->phase_ms[k];
    c->phase_ms[k] = 0.0;
  }
  if (nsteps) *nsteps = c->phase_steps;
  c->phase_steps = 0;
  return SADI_OK;
}

sadi_status sadi_set_watchdog(sadi_ctx* c, int every) {
  if (!c) return SADI_EINVAL;
  if (every < 0) return fail(c, SADI_EINVAL, "sadi_set_watchdog: every must be >= 0");
  c->wd_every = every;
  return SADI_OK;
}

sadi_status sadi_get_watchdog(sadi_ctx* c, double* l2norm, long long* step) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  CK(cudaStreamSynchronize(c->stream), "sadi_get_watchdog");
  WdState h;
  CK(cudaMemcpy(&h, c->wd, offsetof(WdState, ticket), cudaMemcpyDeviceToHost), "watchdog record");
  if (l2norm) *l2norm = c->h * std::sqrt(h.sumsq);
  if (step) *step = h.step;
  return SADI_OK;
}

sadi_status sadi_debug_expire_waits(sadi_ctx* c, long long wait_limit_ns) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (!is_dense(c)) return fail(c, SADI_EUNSUPPORTED, "sadi_debug_expire_waits: SADI_PREC_FP32_DENSE contexts only");
  if (wait_limit_ns < 100000 || wait_limit_ns > 1000000000)
    return fail(c, SADI_EINVAL, "sadi_debug_expire_waits: wait_limit_ns must be in [1e5, 1e9]");
  c->dbg_expire_ns = wait_limit_ns;
  return SADI_OK;
}

const char* sadi_last_error(const sadi_ctx* c) {
  if (!c) return g_create_err.c_str();
  return c->err.c_str();
}

void sadi_destroy(sadi_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

}  // extern "C"

// ---- sadi_step_noalloc: caller-owned state, fixed library scratch -----------

namespace {

// cuMemGetAddressRange of the driver API, looked up once through the runtime
// (the library does not link libcuda directly)
using AddressRangeFn = CUresult (*)(CUdeviceptr*, size_t*, CUdeviceptr);
AddressRangeFn address_range_fn() {
  static AddressRangeFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return static_cast<AddressRangeFn>(nullptr);
    }
    return reinterpret_cast<AddressRangeFn>(f);
  }();
  return fn;
}

// p must be device (or managed) memory on the context's device, and the
// allocation holding p must extend over all `bytes` bytes from p.
sadi_status check_device_buffer(sadi_ctx* c, const void* p, size_t bytes, const char* name) {
  cudaPointerAttributes a{};
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, SADI_EINVAL, std::string(name) + " is not a CUDA pointer");
  }
  if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != c->device)
    return fail(c, SADI_EINVAL, std::string(name) + " must be device memory on the context's device");
  AddressRangeFn range = address_range_fn();
  if (!range) return fail(c, SADI_EINVAL, std::string(name) + ": cannot query the size of its allocation");
  CUdeviceptr base = 0;
  size_t size = 0;
  const CUdeviceptr q = reinterpret_cast<CUdeviceptr>(p);
  if (range(&base, &size, q) != CUDA_SUCCESS)
    return fail(c, SADI_EINVAL, std::string(name) + ": cannot query the size of its allocation");
  if (q < base || q - base > size || size - (q - base) < bytes)
    return fail(c, SADI_EINVAL,
                std::string(name) + " is shorter than N*N doubles (" + std::to_string(bytes) + " bytes needed, " +
                    std::to_string(base + size > q ? size_t(base + size - q) : size_t(0)) +
                    " left in its allocation)");
  return SADI_OK;
}

bool ranges_overlap(const void* p, const void* q, size_t bytes) {
  const char* a = static_cast<const char*>(p);
  const char* b = static_cast<const char*>(q);
  return a < b + bytes && b < a + bytes;
}

}  // namespace

extern "C" sadi_status sadi_step_noalloc(sadi_ctx* c, const double* u_prev, const double* u_cur, double* u_next,
                                         long long n) {
  if (!c) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (c->prec != SADI_PREC_FP64)
    return fail(c, SADI_EUNSUPPORTED, "sadi_step_noalloc: FP64 contexts only (select SADI_PREC_FP64)");
  if (!u_prev || !u_cur || !u_next) return fail(c, SADI_EINVAL, "sadi_step_noalloc: a state pointer is NULL");
  if (n < 1) return fail(c, SADI_EINVAL, "sadi_step_noalloc: n (time level of u_cur) must be >= 1");
  const Geom& g = c->g;
  const size_t nn = (size_t)g.N * g.N;
  const size_t s_bytes = (size_t)g.N * g.Np * 2 * sizeof(double);
  const size_t w_off = (s_bytes + 255) & ~size_t(255);
  const size_t need = w_off + nn * sizeof(double);
  if (need > kNoallocScratchBytes)
    return fail(c, SADI_EINVAL,
                "sadi_step_noalloc: this N needs " + std::to_string(need) + " bytes of scratch, above the fixed " +
                    std::to_string(kNoallocScratchBytes) + " (N <= 1024 fits)");
  const size_t ub = nn * sizeof(double);
  if (ranges_overlap(u_next, u_cur, ub)) return fail(c, SADI_EINVAL, "sadi_step_noalloc: u_next overlaps u_cur");
  if (u_next != u_prev && ranges_overlap(u_next, u_prev, ub))
    return fail(c, SADI_EINVAL, "sadi_step_noalloc: u_next overlaps u_prev without being equal to it");
  int dev = -1;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != c->device) return fail(c, SADI_EINVAL, "sadi_step_noalloc: the context's device must be current");
  sadi_status st = check_device_buffer(c, u_prev, ub, "u_prev");
  if (st == SADI_OK) st = check_device_buffer(c, u_cur, ub, "u_cur");
  if (st == SADI_OK) st = check_device_buffer(c, u_next, ub, "u_next");
  if (st != SADI_OK) return st;
  void* scratch = nullptr;
  // a failed look-up (e.g. a first call made during a stream capture) is
  // reported without marking the context unusable; a later call retries it
  const cudaError_t se = noalloc_scratch_address(dev, &scratch);
  if (se != cudaSuccess) {
    cudaGetLastError();
    return fail(c, SADI_ESTATE,
                std::string("sadi_step_noalloc: looking up the scratch array's device address failed: ") +
                    cudaGetErrorName(se) + " (make the first call on a device outside any stream capture)");
  }
  const RhsParams rp = rhs_of(c, n);
  StepTables<double> tb{c->stw64, c->tw64, c->lpb64, c->lams64, c->lamc64, c->G64};
  double* W = reinterpret_cast<double*>(static_cast<char*>(scratch) + w_off);
  // u_prev is only read by the plain (uncompensated) leapfrog form
  CK(launch_step<double>(g, tb, c->tiles64, rp, u_cur, const_cast<double*>(u_prev), u_next, nullptr,
                         static_cast<const double*>(c->phi2), scratch, W, c->stream, nullptr),
     "step launch");
  return SADI_OK;
}

// ---- sadi_step_source: one step with a per-step source field ---------------

extern "C" sadi_status sadi_step_source(sadi_ctx* c, const void* f, int dtype) {
  if (!c) return SADI_EINVAL;
  sadi_status st = check_steppable(c);
  if (st != SADI_OK) return st;
  if (!f) return fail(c, SADI_EINVAL, "sadi_step_source: f is NULL");
  if (dtype != 0 && dtype != 1) return fail(c, SADI_EINVAL, "sadi_step_source: dtype must be 0 (double) or 1 (float)");
  if (c->F) return fail(c, SADI_ESTATE, "sadi_step_source: remove the separable source (sadi_set_source NULL) first");
  const size_t nn = (size_t)c->g.N * c->g.N;
  st = check_device_buffer(c, f, nn * (dtype == 0 ? sizeof(double) : sizeof(float)), "f");
  if (st != SADI_OK) return st;
  const bool f64 = c->prec == SADI_PREC_FP64;
  const int N = c->g.N, ld = c->g.ld;
  const void* field = f;
  // the caller's field is used in place when its type and row pitch are the
  // context's; else it is converted (and its rows spread to the padded pitch)
  if ((dtype == 0) != f64 || ld != N) {
    if (!c->Fconv) CK(cudaMalloc(&c->Fconv, (size_t)ld * N * esize(c->prec)), "cudaMalloc(source conversion)");
    if (f64)
      CK(launch_convert_f2d(static_cast<const float*>(f), static_cast<double*>(c->Fconv), N, N, N, ld, c->stream),
         "source convert");
    else if (dtype == 0)
      CK(launch_convert_d2f(static_cast<const double*>(f), static_cast<float*>(c->Fconv), N, N, N, ld, c->stream),
         "source convert");
    else
      CK(cudaMemcpy2DAsync(c->Fconv, (size_t)ld * sizeof(float), f, (size_t)N * sizeof(float), (size_t)N * sizeof(float),
                           N, cudaMemcpyDeviceToDevice, c->stream),
         "source copy");
    field = c->Fconv;
  }
  c->F_step = field;
  st = sadi_step(c, 1);
  c->F_step = nullptr;
  return st;
}

// ---- checkpoint / resume -----------------------------------------------------

namespace {

struct StateHeader {
  char magic[8];          // "SADIST02"
  int N, Np, prec, gkind, cur, initialized, eq;
  long long n;
  double alpha, kappa, tau, a, b;
  double gc[3];           // coefficients of SADI_G_GENERAL
  int narrays;            // arrays of N*N elements that follow
  int esz;                // bytes per element of the state arrays
};

// device arrays that make up the step state of c, in blob order
int state_arrays(sadi_ctx* c, void** out) {
  int k = 0;
  if (c->prec == SADI_PREC_FP64) {
    out[k++] = c->ubuf[c->cur];        // u^n
    out[k++] = c->ubuf[1 - c->cur];    // u^{n-1}
    out[k++] = c->phi2;
  } else {
    out[k++] = c->ubuf[0];             // u_hi
    out[k++] = c->ulo;                 // u_lo
    out[k++] = c->ubuf[1];             // d = u^n - u^{n-1}
    out[k++] = c->Chi;                 // remainder pair
    out[k++] = c->Clo;
    out[k++] = c->phi2;
  }
  return k;
}

}  // namespace

extern "C" sadi_status sadi_save_state(sadi_ctx* c, void* buf, size_t* bytes) {
  if (!c || !bytes) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  if (!c->initialized) return fail(c, SADI_ESTATE, "sadi_save_state before sadi_set_initial");
  void* arr[8];
  const int na = state_arrays(c, arr);
  const size_t es = c->prec == SADI_PREC_FP64 ? sizeof(double) : sizeof(float);
  const size_t nn = (size_t)c->g.N * c->g.N;
  const size_t need = sizeof(StateHeader) + (size_t)na * nn * es;
  if (!buf) {
    *bytes = need;
    return SADI_OK;
  }
  if (*bytes < need) {
    *bytes = need;
    return fail(c, SADI_EINVAL, "sadi_save_state: buffer too small (size returned in *bytes)");
  }
  StateHeader h{};
  std::memcpy(h.magic, "SADIST02", 8);
  for (int k = 0; k < 3; ++k) h.gc[k] = c->gc[k];
  h.N = c->g.N;
  h.Np = c->g.Np;
  h.prec = c->prec;
  h.gkind = c->gkind;
  h.eq = c->eq;
  h.cur = 0;
  h.initialized = 1;
  h.n = c->n;
  h.alpha = c->alpha;
  h.kappa = c->kappa;
  h.tau = c->tau;
  h.a = c->a;
  h.b = c->b;
  h.narrays = na;
  h.esz = (int)es;
  std::memcpy(buf, &h, sizeof h);
  char* p = static_cast<char*>(buf) + sizeof h;
  const size_t row = (size_t)c->g.N * es, pitch = (size_t)c->g.ld * es;
  for (int k = 0; k < na; ++k, p += nn * es)
    CK(cudaMemcpy2DAsync(p, row, arr[k], pitch, row, c->g.N, cudaMemcpyDeviceToHost, c->stream), "copy state");
  CK(cudaStreamSynchronize(c->stream), "sadi_save_state");
  *bytes = need;
  return SADI_OK;
}

extern "C" sadi_status sadi_load_state(sadi_ctx* c, const void* buf, size_t bytes) {
  if (!c || !buf) return SADI_EINVAL;
  if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
  StateHeader h;
  if (bytes < sizeof h) return fail(c, SADI_EINVAL, "sadi_load_state: blob too small");
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, "SADIST02", 8) != 0) return fail(c, SADI_EINVAL, "sadi_load_state: not a state blob");
  if (h.N != c->g.N || h.prec != c->prec || h.gkind != c->gkind || h.eq != c->eq || h.alpha != c->alpha ||
      h.kappa != c->kappa ||
      h.tau != c->tau || h.a != c->a || h.b != c->b || h.gc[0] != c->gc[0] || h.gc[1] != c->gc[1] ||
      h.gc[2] != c->gc[2])
    return fail(c, SADI_EINVAL,
                "sadi_load_state: the blob was saved by a context with another N, alpha, kappa, tau, domain, g or "
                "precision");
  void* arr[8];
  const int na = state_arrays(c, arr);
  const size_t es = c->prec == SADI_PREC_FP64 ? sizeof(double) : sizeof(float);
  const size_t nn = (size_t)c->g.N * c->g.N;
  if (h.narrays != na || h.esz != (int)es || bytes < sizeof h + (size_t)na * nn * es || h.n < 0)
    return fail(c, SADI_EINVAL, "sadi_load_state: blob size or layout does not match");
  c->cur = 0;   // saved in canonical order: arr[0] = u^n
  state_arrays(c, arr);
  const char* p = static_cast<const char*>(buf) + sizeof h;
  const size_t row = (size_t)c->g.N * es, pitch = (size_t)c->g.ld * es;
  for (int k = 0; k < na; ++k, p += nn * es)
    CK(cudaMemcpy2DAsync(arr[k], pitch, p, row, row, c->g.N, cudaMemcpyHostToDevice, c->stream), "copy state");
  CK(cudaMemsetAsync(c->wd, 0, sizeof(WdState), c->stream), "watchdog record");
  CK(cudaStreamSynchronize(c->stream), "sadi_load_state");
  c->n = h.n;
  c->initialized = true;
  return SADI_OK;
}
