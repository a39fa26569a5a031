// graph_tune.cu -- CUDA-graph replay of batched steps and the autotuner of
// the step form (FP32 Gohberg-Semencul FFT sweeps vs dense-inverse tensor-core
// sweeps) and of the shared-memory engine's work decomposition.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "sadi_ctx.h"

using namespace sadi;
using namespace sadi_api;

struct sadi_graph {
  std::vector<sadi_ctx*> ctxs;
  std::vector<int> cur;   // FP64 contexts: which ping-pong buffer held u^n at capture
  int nsteps = 0;
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// nsteps: steps per replay.  An FP64 context keeps u^n and u^{n-1} in two
// buffers that swap every step, so it replays only in graphs of an even
// number of steps, launched with the buffers as they were at capture (cur,
// when launching).
sadi_status graph_check(sadi_ctx* const* ctxs, int count, bool launching, int nsteps, const int* cur = nullptr) {
  cudaStream_t s0 = ctxs[0]->stream;
  for (int k = 0; k < count; ++k) {
    sadi_ctx* c = ctxs[k];
    sadi_status st = check_steppable(c);
    if (st != SADI_OK) return st;
    if (c->prec == SADI_PREC_FP64 && nsteps % 2 != 0)
      return fail(c, SADI_EUNSUPPORTED, "FP64 contexts replay in graphs of an even number of steps only");
    if (c->prec == SADI_PREC_FP64 && cur && c->cur != cur[k])
      return fail(c, SADI_ESTATE, "an odd number of steps since the capture: the FP64 buffers are swapped");
    if (c->n < 1) return fail(c, SADI_ESTATE, "take the n = 0 step before capturing or launching a graph");
    if (c->F) return fail(c, SADI_EUNSUPPORTED, "a source term changes every step; it cannot be replayed");
    if (c->profiling) return fail(c, SADI_ESTATE, "disable sadi_profile before capturing a graph");
    if (c->dbg_expire_ns) return fail(c, SADI_ESTATE, "a sadi_debug_expire_waits step is pending; step it first");
    if (c->stream != s0) return fail(c, SADI_EINVAL, "all contexts of a graph must share one stream");
    if (!launching)
      for (int j = 0; j < k; ++j)
        if (ctxs[j] == c) return fail(c, SADI_EINVAL, "a context appears twice");
  }
  return SADI_OK;
}

std::string fmt(const char* f, double a, double b = 0, double c = 0, double d = 0) {
  char buf[256];
  std::snprintf(buf, sizeof buf, f, a, b, c, d);
  return buf;
}

}  // namespace

extern "C" {

sadi_status sadi_graph_create(sadi_ctx** ctxs, int count, int nsteps, sadi_graph** out) {
  if (!out) return SADI_EINVAL;
  *out = nullptr;
  if (!ctxs || count < 1 || nsteps < 1) return SADI_EINVAL;
  for (int k = 0; k < count; ++k)
    if (!ctxs[k]) return SADI_EINVAL;
  sadi_status st = graph_check(ctxs, count, false, nsteps);
  if (st != SADI_OK) return st;
  sadi_graph* g = new (std::nothrow) sadi_graph();
  if (!g) return fail(ctxs[0], SADI_ENOMEM, "host allocation failed");
  g->ctxs.assign(ctxs, ctxs + count);
  for (int k = 0; k < count; ++k) g->cur.push_back(ctxs[k]->cur);
  g->nsteps = nsteps;
  g->stream = ctxs[0]->stream;
  std::vector<long long> n0(count);
  for (int k = 0; k < count; ++k) n0[k] = ctxs[k]->n;
  // the capture issues the steps without running them: the FP64 buffer swaps
  // it makes are undone below, with the step counters
  cudaError_t e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    delete g;
    return cuda_fail(ctxs[0], e, "cudaStreamBeginCapture");
  }
  st = batch_issue(ctxs, count, nsteps);
  e = cudaStreamEndCapture(g->stream, &g->graph);
  for (int k = 0; k < count; ++k) {
    ctxs[k]->n = n0[k];
    ctxs[k]->cur = g->cur[k];
  }
  if (st == SADI_OK && e != cudaSuccess) st = cuda_fail(ctxs[0], e, "cudaStreamEndCapture");
  if (st == SADI_OK) {
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) st = cuda_fail(ctxs[0], e, "cudaGraphInstantiate");
  }
  if (st != SADI_OK) {
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return st;
  }
  *out = g;
  return SADI_OK;
}

sadi_status sadi_graph_launch(sadi_graph* g, int reps) {
  if (!g || reps < 0) return SADI_EINVAL;
  sadi_status st = graph_check(g->ctxs.data(), (int)g->ctxs.size(), true, g->nsteps, g->cur.data());
  if (st != SADI_OK) return st;
  for (int r = 0; r < reps; ++r) {
    const cudaError_t e = cudaGraphLaunch(g->exec, g->stream);
    if (e != cudaSuccess) {
      for (sadi_ctx* c : g->ctxs) cuda_fail(c, e, "cudaGraphLaunch");
      return SADI_ECUDA;
    }
  }
  for (sadi_ctx* c : g->ctxs) {
    const long long n_before = c->n;
    c->n += (long long)g->nsteps * reps;
    st = watchdog_after(c, n_before, g->stream);
    if (st != SADI_OK) return st;
  }
  return SADI_OK;
}

sadi_status sadi_graph_kernels(const sadi_graph* g, int* kernels) {
  if (!g || !kernels) return SADI_EINVAL;
  size_t n = 0;
  if (cudaGraphGetNodes(g->graph, nullptr, &n) != cudaSuccess) return SADI_ECUDA;
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(g->graph, nodes.data(), &n) != cudaSuccess) return SADI_ECUDA;
  int k = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess) return SADI_ECUDA;
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  *kernels = k;
  return SADI_OK;
}

void sadi_graph_destroy(sadi_graph* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

}  // extern "C"

// ---- autotuner ----------------------------------------------------------------

namespace {

struct Cand {
  int prec;
  Tiles t;
};

// largest s a_0 for which the autotuner offers the dense form
constexpr double kDenseMaxSA0 = 0.2;

// ms per batched step of the group in its current configuration (zero data:
// the step's cost does not depend on the values)
sadi_status time_group(std::vector<sadi_ctx*>& grp, int reps, double* ms) {
  for (sadi_ctx* c : grp) {
    sadi_status st = zero_initial(c);
    if (st != SADI_OK) return st;
  }
  sadi_ctx* c0 = grp[0];
  sadi_status st = batch_issue(grp.data(), (int)grp.size(), 3);   // start step + warm-up
  if (st != SADI_OK) return st;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(c0, e, "cudaEventCreate");
  cudaEventRecord(e0, c0->stream);
  st = batch_issue(grp.data(), (int)grp.size(), reps);
  cudaEventRecord(e1, c0->stream);
  e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SADI_OK) return st;
  if (e != cudaSuccess) return cuda_fail(c0, e, "timing");
  *ms = t / reps;
  return SADI_OK;
}

sadi_status apply(std::vector<sadi_ctx*>& grp, int g, const Cand& cd) {
  for (sadi_ctx* c : grp) {
    c->initialized = false;
    c->n = 0;
    sadi_status st = sadi_set_options(c, g, cd.prec);
    if (st != SADI_OK) return st;
    // zero tiles restore the defaults (and, for the dense form at N' = 2048,
    // the register path that an earlier candidate's tiles may have left)
    st = sadi_set_tiles(c, cd.t.rows, cd.t.conv_cols, cd.t.solve_cols);
    if (st != SADI_OK) return st;
  }
  return SADI_OK;
}

const char* prec_name(int p) { return p == SADI_PREC_FP32 ? "fp32-gsfft" : "fp32-dense"; }

}  // namespace

extern "C" {

sadi_status sadi_autotune(sadi_ctx** ctxs, int count, int g, int flags) {
  if (!ctxs || count < 1) return SADI_EINVAL;
  for (int k = 0; k < count; ++k) {
    if (!ctxs[k]) return SADI_EINVAL;
    sadi_ctx* c = ctxs[k];
    if (c->broken) return fail(c, SADI_ESTATE, "context unusable after a CUDA error");
    if (c->initialized) return fail(c, SADI_ESTATE, "sadi_autotune must precede sadi_set_initial");
    if (c->F) return fail(c, SADI_ESTATE, "sadi_autotune must precede sadi_set_source");
    if (c->profiling) return fail(c, SADI_ESTATE, "disable sadi_profile before sadi_autotune");
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == c) return fail(c, SADI_EINVAL, "a context appears twice");
  }
  if (g < SADI_G_ZERO || g > SADI_G_GENERAL) return fail(ctxs[0], SADI_EINVAL, "g must be 0, 1, 2 or 3");
  // groups of equal N (they share a choice), at most one register-path batch each
  std::map<int, std::vector<sadi_ctx*>> by_n;
  for (int k = 0; k < count; ++k) by_n[ctxs[k]->g.N].push_back(ctxs[k]);
  for (auto& kv : by_n) {
    std::vector<sadi_ctx*>& all = kv.second;
    const int N = kv.first, Np = all[0]->g.Np, logNp = all[0]->g.logNp;
    std::vector<int> precs{SADI_PREC_FP32};
    // the dense form's split-BF16 error scales with E = H^-1 - I, i.e. with
    // s a_0 (s = kappa tau^2 / (2 h^alpha)); it is offered only while E is small
    double a0 = 0.0;
    if (cudaMemcpy(&a0, all[0]->a1, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return cuda_fail(all[0], cudaErrorUnknown, "reading a_0");
    const bool dense_ok = all[0]->s * a0 <= kDenseMaxSA0;
    if (!(flags & 1) && dense_ok) precs.push_back(SADI_PREC_FP32_DENSE);
    if (flags & 2) {
      // keep the precision the group was created with; tune its tiles only
      const int p0 = all[0]->prec;
      for (sadi_ctx* c : all)
        if (c->prec != p0) return fail(c, SADI_EINVAL, "flags bit 1: contexts of one N differ in precision");
      if (p0 == SADI_PREC_FP64) return fail(all[0], SADI_EUNSUPPORTED, "flags bit 1 tunes the FP32 forms only");
      precs.assign(1, p0);
    }
    // register-path contexts step in batches of up to kMaxBatch, the
    // shared-memory engine one context after another; every candidate is
    // timed on the same group (the step time of the whole group), as large
    // as a register-path candidate batches
    bool any_reg = false;
    for (int prec : precs) any_reg = any_reg || reg_path_supported(logNp, prec);
    const size_t cap = any_reg ? (size_t)kMaxBatch : 1;
    std::vector<sadi_ctx*> grp(all.begin(), all.begin() + std::min(all.size(), cap));
    std::string log = fmt("N=%.0f N'=%.0f batch=%.0f s*a0=%.3g:", N, Np, (double)grp.size(), grp[0]->s * a0);
    Cand best{SADI_PREC_FP32, Tiles{0, 0, 0}};
    double best_ms = 1e30;
    for (int prec : precs) {
      Cand cd{prec, Tiles{0, 0, 0}};
      sadi_status st = apply(grp, g, cd);
      if (st != SADI_OK) return st;
      double ms = 0;
      if ((st = time_group(grp, 5, &ms)) != SADI_OK) return st;
      if (!reg_path_supported(logNp, prec)) {
        // coordinate descent over the shared-memory engine's decomposition
        // (the dense form leaves the y-sweep tile unused); the column
        // convolution may also run as three passes (kConvThreePass)
        Tiles t = grp[0]->tiles32;
        const int nfields = prec == SADI_PREC_FP32 ? 3 : 2;
        const int opts[3][5] = {{1, 2, 4, 8, 0}, {kConvThreePass, 1, 2, 4, 8}, {1, 2, 4, 8, 0}};
        for (int f = 0; f < nfields; ++f) {
          for (int v : opts[f]) {
            if (v == 0) continue;
            Tiles tt = t;
            (f == 0 ? tt.rows : f == 1 ? tt.conv_cols : tt.solve_cols) = v;
            if ((f == 0 ? t.rows : f == 1 ? t.conv_cols : t.solve_cols) == v) continue;
            if (!tiles_valid<float>(grp[0]->g, tt)) continue;
            Cand c2{prec, tt};
            if ((st = apply(grp, g, c2)) != SADI_OK) return st;
            double m2 = 0;
            if ((st = time_group(grp, 5, &m2)) != SADI_OK) return st;
            if (m2 < ms) {
              ms = m2;
              t = tt;
            }
          }
        }
        cd.t = t;
        log += std::string(" ") + prec_name(prec) +
               fmt("(tiles %.0f/%.0f/%.0f) %.4f ms", t.rows, t.conv_cols, t.solve_cols, ms);
      } else {
        log += std::string(" ") + prec_name(prec) + fmt(" %.4f ms", ms);
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = cd;
      }
    }
    log += std::string(" -> ") + prec_name(best.prec);
    for (sadi_ctx* c : all) {
      std::vector<sadi_ctx*> one{c};
      sadi_status st = apply(one, g, best);
      if (st != SADI_OK) return st;
      c->initialized = false;
      c->n = 0;
      c->tune_log = log;
    }
  }
  return SADI_OK;
}

const char* sadi_tuning_log(const sadi_ctx* c) { return c ? c->tune_log.c_str() : ""; }

}  // extern "C"
