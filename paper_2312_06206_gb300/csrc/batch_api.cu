// batch_api.cu -- a batch of independent S-ADI instances behind one handle:
// create (with the step form chosen by the autotuner or given), set initial
// data per member, advance all members together, read a member back.
//
// The members are ordinary contexts on one stream.  sadi_batch_run advances
// them with the batched launches of sadi_batch_step and, once every member
// is past its n = 0 step and the members allow it (no source term, no
// profiling), by replaying a CUDA graph of one batched step (two when a
// member is FP64) that is captured on first use and kept until a member's
// set-up changes.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "sadi_ctx.h"

using namespace sadi;
using namespace sadi_api;

struct sadi_batch {
  std::vector<sadi_ctx*> ctxs;
  cudaStream_t own_stream = nullptr;
  sadi_graph* graph = nullptr;      // gsteps batched steps, captured on first use
  int gsteps = 1;                   // 2 when a member is FP64 (its buffers swap every step)
  bool graph_failed = false;        // the members cannot be replayed: launch directly
  std::string err;
};

namespace {

sadi_status bfail(sadi_batch* b, sadi_status st, const std::string& msg) {
  if (b) b->err = msg;
  return st;
}

// message of member k's last failure, kept on the batch
sadi_status member_fail(sadi_batch* b, int k, sadi_status st) {
  b->err = "member " + std::to_string(k) + ": " + sadi_last_error(b->ctxs[k]);
  return st;
}

void drop_graph(sadi_batch* b) {
  if (b->graph) sadi_graph_destroy(b->graph);
  b->graph = nullptr;
  b->graph_failed = false;
}

void destroy_batch(sadi_batch* b) {
  drop_graph(b);
  for (sadi_ctx* c : b->ctxs) sadi_destroy(c);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
}

thread_local std::string g_batch_create_err;

}  // namespace

extern "C" {

sadi_status sadi_batch_create(int count, const int* N, const double* alpha, const double* kappa, const double* tau,
                              const double* domains, int g, int prec, sadi_batch** out) {
  g_batch_create_err.clear();
  if (!out) return SADI_EINVAL;
  *out = nullptr;
  if (count < 1 || !N || !alpha || !kappa || !tau) {
    g_batch_create_err = "sadi_batch_create: count >= 1 and the N, alpha, kappa, tau arrays are required";
    return SADI_EINVAL;
  }
  if (prec != SADI_PREC_AUTO && prec != SADI_PREC_FP64 && prec != SADI_PREC_FP32 && prec != SADI_PREC_FP32_DENSE) {
    g_batch_create_err = "sadi_batch_create: prec must be SADI_PREC_AUTO, 0, 1 or 2";
    return SADI_EINVAL;
  }
  sadi_batch* b = new (std::nothrow) sadi_batch();
  if (!b) return SADI_ENOMEM;
  auto bail = [&](sadi_status st) {
    g_batch_create_err = b->err;
    destroy_batch(b);
    return st;
  };
  if (cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return bail(bfail(b, SADI_ECUDA, "sadi_batch_create: cudaStreamCreate failed"));
  }
  for (int k = 0; k < count; ++k) {
    const double dflt[2] = {-1.0, 1.0};
    sadi_ctx* c = nullptr;
    const sadi_status st = sadi_create(N[k], alpha[k], kappa[k], tau[k], domains ? domains + 2 * k : dflt, &c);
    if (st != SADI_OK)
      return bail(bfail(b, st, "member " + std::to_string(k) + ": " + sadi_last_error(nullptr)));
    b->ctxs.push_back(c);
    sadi_set_stream(c, b->own_stream);
  }
  if (prec == SADI_PREC_AUTO) {
    const sadi_status st = sadi_autotune(b->ctxs.data(), count, g, 0);
    if (st != SADI_OK) {
      for (int k = 0; k < count; ++k)
        if (*sadi_last_error(b->ctxs[k])) return bail(member_fail(b, k, st));
      return bail(bfail(b, st, "sadi_batch_create: autotune failed"));
    }
  } else {
    for (int k = 0; k < count; ++k) {
      const sadi_status st = sadi_set_options(b->ctxs[k], g, prec);
      if (st != SADI_OK) return bail(member_fail(b, k, st));
    }
  }
  *out = b;
  return SADI_OK;
}

sadi_status sadi_batch_set_initial(sadi_batch* b, int k, const double* phi1, const double* phi2) {
  if (!b) return SADI_EINVAL;
  if (k < 0 || k >= (int)b->ctxs.size()) return bfail(b, SADI_EINVAL, "sadi_batch_set_initial: k out of range");
  const sadi_status st = sadi_set_initial(b->ctxs[k], phi1, phi2);
  return st == SADI_OK ? SADI_OK : member_fail(b, k, st);
}

sadi_status sadi_batch_set_stream(sadi_batch* b, void* stream) {
  if (!b) return SADI_EINVAL;
  drop_graph(b);
  for (sadi_ctx* c : b->ctxs) sadi_set_stream(c, stream ? stream : b->own_stream);
  return SADI_OK;
}

sadi_status sadi_batch_run(sadi_batch* b, int nsteps) {
  if (!b) return SADI_EINVAL;
  if (nsteps < 0) return bfail(b, SADI_EINVAL, "sadi_batch_run: nsteps must be >= 0");
  const int count = (int)b->ctxs.size();
  sadi_ctx** cs = b->ctxs.data();
  for (int k = 0; k < count; ++k)
    if (!cs[k]->initialized) return bfail(b, SADI_ESTATE, "member " + std::to_string(k) + " has no initial data");
  while (nsteps > 0) {
    bool fresh = false;   // a member still takes its n = 0 step
    for (int k = 0; k < count; ++k) fresh = fresh || cs[k]->n == 0;
    bool fp64 = false;
    for (int k = 0; k < count; ++k) fp64 = fp64 || cs[k]->prec == SADI_PREC_FP64;
    const int gsteps = fp64 ? 2 : 1;
    if (fresh || b->graph_failed || nsteps < gsteps) {
      const int m = fresh ? 1 : nsteps;
      // a direct step swaps FP64 buffers: a graph captured before is replayed
      // only after an even number of them, so capture anew
      if (fp64 && (m % 2) != 0 && b->graph) {
        sadi_graph_destroy(b->graph);
        b->graph = nullptr;
      }
      const sadi_status st = sadi_batch_step(cs, count, m);
      if (st != SADI_OK) {
        for (int k = 0; k < count; ++k)
          if (*sadi_last_error(cs[k])) return member_fail(b, k, st);
        return bfail(b, st, "sadi_batch_run: batched step failed");
      }
      nsteps -= m;
      continue;
    }
    if (b->graph && b->gsteps != gsteps) drop_graph(b);
    if (!b->graph) {
      b->gsteps = gsteps;
      const sadi_status st = sadi_graph_create(cs, count, gsteps, &b->graph);
      if (st == SADI_EUNSUPPORTED || st == SADI_ESTATE) {
        // FP64 members, a source term or profiling: direct launches
        b->graph = nullptr;
        b->graph_failed = true;
        for (sadi_ctx* c : b->ctxs) c->err.clear();
        continue;
      }
      if (st != SADI_OK) return bfail(b, st, "sadi_batch_run: graph capture failed");
    }
    const sadi_status st = sadi_graph_launch(b->graph, nsteps / gsteps);
    if (st != SADI_OK) {
      drop_graph(b);
      for (int k = 0; k < count; ++k)
        if (*sadi_last_error(cs[k])) return member_fail(b, k, st);
      return bfail(b, st, "sadi_batch_run: graph launch failed");
    }
    nsteps %= gsteps;   // an odd last step of FP64 members: directly, above
  }
  return SADI_OK;
}

sadi_status sadi_batch_get(sadi_batch* b, int k, double* u_out, long long* n_out) {
  if (!b) return SADI_EINVAL;
  if (k < 0 || k >= (int)b->ctxs.size()) return bfail(b, SADI_EINVAL, "sadi_batch_get: k out of range");
  const sadi_status st = sadi_get(b->ctxs[k], u_out, n_out);
  return st == SADI_OK ? SADI_OK : member_fail(b, k, st);
}

sadi_status sadi_batch_member(sadi_batch* b, int k, sadi_ctx** ctx) {
  if (!b || !ctx) return SADI_EINVAL;
  if (k < 0 || k >= (int)b->ctxs.size()) return bfail(b, SADI_EINVAL, "sadi_batch_member: k out of range");
  // the caller may change a member's set-up through its context: capture anew
  drop_graph(b);
  *ctx = b->ctxs[k];
  return SADI_OK;
}

sadi_status sadi_batch_count(const sadi_batch* b, int* count) {
  if (!b || !count) return SADI_EINVAL;
  *count = (int)b->ctxs.size();
  return SADI_OK;
}

const char* sadi_batch_last_error(const sadi_batch* b) { return b ? b->err.c_str() : g_batch_create_err.c_str(); }

void sadi_batch_destroy(sadi_batch* b) {
  if (!b) return;
  if (b->own_stream) cudaStreamSynchronize(b->own_stream);
  destroy_batch(b);
}

}  // extern "C"
