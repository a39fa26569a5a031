// sadi_ctx.h -- the context object behind the opaque sadi_ctx of the C ABI,
// and the internal helpers shared by the translation units that implement
// the ABI (sadi_api.cu, graph_tune.cu).  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <memory>
#include <string>
#include <vector>

#include "../../include/sadi.h"
#include "sadi_internal.h"

// steps between watchdog checks of a new context
constexpr int kWatchdogDefaultEvery = 100;

struct sadi_ctx {
  using Geom = sadi::Geom;
  using Tiles = sadi::Tiles;
  using TcInst = sadi::TcInst;
  Geom g{};
  double alpha = 0, kappa = 0, tau = 0, a = 0, b = 0, h = 0, s = 0;
  int eq = 0;                       // 0 the wave equation, 1 the diffusion equation
  int gkind = SADI_G_ZERO;
  double gc[3] = {0.0, 0.0, 0.0};   // coefficients of SADI_G_GENERAL (u, u^3, sin u)
  int prec = SADI_PREC_FP64;
  int device = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  // FP64 setup products
  double* a1 = nullptr;      // Np
  double* a2d = nullptr;     // N x N
  double* cgen = nullptr;    // Np
  double* lnat = nullptr;    // (Np+1)^2
  double2* tw64 = nullptr;   // P
  float2* tw32 = nullptr;    // P
  double2* stw64 = nullptr;  // per-stage FFT twiddles
  float2* stw32 = nullptr;
  Tiles tiles64{}, tiles32{};
  // tiles set explicitly (not the defaults): at N' = 2048 they keep the
  // dense form on the shared-memory engine
  bool tiles_explicit = false;
  // FP32 register-FFT path tables (N' <= 2048)
  float2* rtw1 = nullptr;
  float* rlreg = nullptr;
  float2* rlamc = nullptr;
  float2* rlams = nullptr;
  bool reg_path = false;
  double* lpb64 = nullptr;   // (Np+1) 2 Np
  float* lpb32 = nullptr;
  double2* lamc64 = nullptr;
  double2* lams64 = nullptr;
  float2* lamc32 = nullptr;
  float2* lams32 = nullptr;
  double* G64 = nullptr;     // N x r
  float* G32 = nullptr;
  // state (element type per prec)
  // FP64: ubuf[cur] = u^n, ubuf[1-cur] = u^{n-1} (ping-pong).
  // FP32: ubuf[0] = hi part of u^n, ubuf[1] = d = u^n - u^{n-1}, ulo = lo part
  // (double-float state, updated in place; cur stays 0).
  void* ubuf[2] = {nullptr, nullptr};
  float* ulo = nullptr;
  // FP32 forms: the remainder C = -kappa tau^2 L_h u^n as a double-float pair,
  // advanced each step by the convolution of the increment d^n
  float* Chi = nullptr;
  float* Clo = nullptr;
  void* phi2 = nullptr;
  void* S = nullptr;         // N x Np complex
  void* W = nullptr;         // N x N
  double* stage = nullptr;   // N x N doubles (host <-> device staging)
  int cur = 0;
  long long n = 0;
  bool initialized = false;
  bool broken = false;
  std::string err;
  // per-kernel timing (sadi_profile)
  bool profiling = false;
  std::vector<std::array<cudaEvent_t, 5>> ev_pool;   // recorded, not yet folded
  std::vector<std::array<cudaEvent_t, 5>> ev_free;
  double phase_ms[4] = {0, 0, 0, 0};
  long long phase_steps = 0;
  cudaEvent_t order_ev = nullptr;   // cross-stream ordering in sadi_batch_step
  // sadi_get_async: device -> host copies of the staging buffer on their own
  // stream; ev_staged orders a copy after the staging, ev_copied orders later
  // writers of the staging buffer after the last copy
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_staged = nullptr, ev_copied = nullptr;
  // optional source term f^n = cos(omega t_n + phase) F(x)
  void* F = nullptr;                // T, N x N
  double f_omega = 0.0, f_phase = 0.0;
  // sadi_step_source: the source field of the step being issued (T, N x N;
  // the caller's buffer or Fconv, its conversion to T), nullptr otherwise
  const void* F_step = nullptr;
  void* Fconv = nullptr;
  // dense-inverse form (SADI_PREC_FP32_DENSE): BF16 pairs, npad x npad,
  // zero-padded: E = H^-1 - I, B^n rows, W^T rows; tensor maps of the two GEMMs
  int npad = 0;
  unsigned short *Eh = nullptr, *El = nullptr, *Bh = nullptr, *Bl = nullptr, *WTh = nullptr, *WTl = nullptr;
  int* tcerr = nullptr;             // device flag: a bounded wait in a GEMM ran out
  long long dbg_expire_ns = 0;      // sadi_debug_expire_waits: next dense step's waits run out (0: off)
  int* tcdep = nullptr;             // per 128-column panel: x-sweep tiles stored (zeroed each step)
  sadi::Conv3 c3;                   // FP32 forms, N' = 2048 .. 8192: three-pass column convolution
  std::unique_ptr<TcInst> tc_x, tc_y;
  std::string tune_log;             // choice of sadi_autotune
  // state watchdog: after a stepping call in which n reaches a multiple of
  // wd_every (0: off), sum u^2 on the device and latch non-finite results
  int wd_every = kWatchdogDefaultEvery;
  sadi::WdState* wd = nullptr;
};

namespace sadi_api {

// store msg in c (if any) and return st
sadi_status fail(sadi_ctx* c, sadi_status st, const std::string& msg);
// message from a CUDA error; the context becomes unusable; returns SADI_ECUDA
sadi_status cuda_fail(sadi_ctx* c, cudaError_t e, const char* what);
sadi_status check_steppable(sadi_ctx* c);
// order the context's stream after the last sadi_get_async copy (which reads
// the staging buffer) before the buffer is written again
cudaError_t stage_acquire(sadi_ctx* c);
// allocate and fill the three-pass convolution's buffers (FP32, N' 2048 .. 8192)
sadi_status ensure_conv3(sadi_ctx* c);
// SADI_ETIMEOUT (and the context marked unusable) if a tensor-core sweep's
// bounded wait ran out
sadi_status check_gemm_flag(sadi_ctx* c);
bool is_dense(const sadi_ctx* c);
// issue nsteps steps of count validated, distinct contexts (what
// sadi_batch_step does after its argument checks)
sadi_status batch_issue(sadi_ctx** ctxs, int count, int nsteps);
// zero state (u, increment, remainder, phi2) and n = 0: a context ready to
// step, for timing runs that need no data
sadi_status zero_initial(sadi_ctx* c);
// queue a watchdog check of c's state if n crossed a multiple of its period
// since n_before (the value before the stepping call)
sadi_status watchdog_after(sadi_ctx* c, long long n_before, cudaStream_t st);
// after the stream has been synchronised: SADI_ENONFINITE (and the state
// marked as needing sadi_set_initial) if a check found a non-finite value
sadi_status check_watchdog(sadi_ctx* c);

}  // namespace sadi_api
