// Batches of independent aggregation jobs (hgf_batch_* in include/hgf.h).
//
// Every job gets its own guidance handle; jobs are assigned to `streams` internal streams,
// largest work (H*W*L) first onto the least-loaded stream, and each internal stream owns a context
// whose workspaces are sized at creation for its largest job. A run records an event on the
// caller's stream, makes every internal stream wait on it, enqueues each job's precompute and
// aggregation on its stream, and makes the caller's stream wait on an event from each internal
// stream: a fork/join that CUDA graph capture follows, so the whole batch becomes one graph.
#include "hgf_internal.cuh"

#include <algorithm>
#include <new>
#include <vector>

using namespace hgf;

struct hgf_batch {
  hgf_ctx *owner = nullptr;
  struct Lane {
    hgf_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<int> jobs;
    double work = 0.0;
  };
  std::vector<hgf_job> jobs;
  std::vector<hgf_guidance *> guid;
  std::vector<AggregatePlan> plans;
  std::vector<Lane> lanes;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t exec_stream = nullptr;
};

namespace {

void destroy_batch(hgf_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto *g : b->guid) free_guidance(g);
  for (auto &l : b->lanes) {
    if (l.done) cudaEventDestroy(l.done);
    if (l.stream) cudaStreamDestroy(l.stream);
    hgf_destroy(l.ctx);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

hgf_status set_ws(Workspace &w, size_t bytes) {
  if (w.size >= bytes) return HGF_OK;
  if (w.ptr) cudaFree(w.ptr);
  w.ptr = nullptr;
  w.size = 0;
  if (cudaMalloc(&w.ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    return HGF_ENOMEM;
  }
  w.size = bytes;
  return HGF_OK;
}

}  // namespace

extern "C" {

hgf_status hgf_batch_create(hgf_ctx *ctx, const hgf_job *jobs, int njobs, int streams,
                            hgf_batch **out) {
  if (!ctx || !jobs || njobs < 1 || streams < 1 || streams > 32 || !out) return HGF_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return HGF_ECUDA;
  hgf_batch *b = new (std::nothrow) hgf_batch;
  if (!b) return HGF_ENOMEM;
  b->owner = ctx;
  b->jobs.assign(jobs, jobs + njobs);
  hgf_status st = HGF_OK;
  for (int i = 0; i < njobs && st == HGF_OK; ++i) {
    const hgf_job &j = jobs[i];
    if (!j.img || !j.cost || (!j.labels && !j.best && !j.filtered) || j.L < 1 ||
        (j.cost_dtype != HGF_F32 && j.cost_dtype != HGF_BF16 && j.cost_dtype != HGF_F16)) {
      st = HGF_EINVAL;
      break;
    }
    hgf_guidance *g = nullptr;
    st = alloc_guidance_checked(ctx, j.C, j.H, j.W, &j.params, &g);
    if (st == HGF_OK && !aggregate_fits(g)) {
      free_guidance(g);
      st = HGF_EUNSUPPORTED;
    }
    if (st == HGF_OK) b->guid.push_back(g);
  }
  if (st != HGF_OK) {
    destroy_batch(b);
    return st;
  }
  // largest first onto the least-loaded lane
  const int nl = std::min(streams, njobs);
  b->lanes.resize(nl);
  std::vector<int> order(njobs);
  for (int i = 0; i < njobs; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int c) {
    return (double)jobs[a].H * jobs[a].W * jobs[a].L > (double)jobs[c].H * jobs[c].W * jobs[c].L;
  });
  for (int i : order) {
    auto it = std::min_element(b->lanes.begin(), b->lanes.end(),
                               [](const hgf_batch::Lane &x, const hgf_batch::Lane &y) {
                                 return x.work < y.work;
                               });
    it->jobs.push_back(i);
    it->work += (double)jobs[i].H * jobs[i].W * jobs[i].L;
  }
  b->plans.resize(njobs);
  for (auto &l : b->lanes) {
    if (hgf_create(ctx->device, &l.ctx) != HGF_OK ||
        cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) != cudaSuccess) {
      destroy_batch(b);
      return HGF_ECUDA;
    }
    l.ctx->tuning = ctx->tuning;
    size_t prep = 0, coef = 0, keys = 0;
    for (int i : l.jobs) {
      const hgf_guidance *g = b->guid[i];
      AggregatePlan p = plan_aggregate(g, jobs[i].L, ctx->tuning, ctx->num_sms);
      // at most 64 labels of coefficients per chunk keep the lane workspaces bounded
      p.chunk = std::min(p.chunk, 64);
      b->plans[i] = p;
      prep = std::max(prep, prepare_workspace_bytes(g->n, g->H, g->W));
      coef = std::max(coef, aggregate_coef_bytes(g, p));
      keys = std::max(keys, (size_t)g->H * g->W * sizeof(unsigned long long));
    }
    if (set_ws(l.ctx->ws_prepare, prep) != HGF_OK || set_ws(l.ctx->ws_coef, coef) != HGF_OK ||
        set_ws(l.ctx->ws_keys, keys) != HGF_OK) {
      destroy_batch(b);
      return HGF_ENOMEM;
    }
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    destroy_batch(b);
    return HGF_ECUDA;
  }
  *out = b;
  return HGF_OK;
}

hgf_status hgf_batch_run(hgf_batch *b, void *stream) {
  if (!b) return HGF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaEventRecord(b->fork, s);
  for (auto &l : b->lanes) {
    if (e == cudaSuccess) e = cudaStreamWaitEvent(l.stream, b->fork, 0);
    for (int i : l.jobs) {
      if (e != cudaSuccess) break;
      const hgf_job &j = b->jobs[i];
      hgf_guidance *g = b->guid[i];
      e = launch_prepare(g, j.img, l.ctx->ws_prepare.ptr, l.ctx->ws_prepare.size, l.stream,
                         &b->owner->prof);
      if (e == cudaSuccess)
        e = launch_aggregate(g, j.cost, j.cost_dtype, j.L, j.filtered, j.labels, j.best,
                             (float *)l.ctx->ws_coef.ptr,
                             (unsigned long long *)l.ctx->ws_keys.ptr, b->plans[i], l.stream,
                             &b->owner->prof);
    }
    if (e == cudaSuccess) e = cudaEventRecord(l.done, l.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, l.done, 0);
  }
  if (e != cudaSuccess) {
    b->owner->sticky.store(HGF_ECUDA);
    b->owner->err = std::string("hgf_batch_run: ") + cudaGetErrorString(e);
    return HGF_ECUDA;
  }
  return HGF_OK;
}

hgf_status hgf_batch_launch_graph(hgf_batch *b, void *stream) {
  if (!b) return HGF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!b->exec) {
    // capture on a private stream so the caller's stream is never left in capture mode
    cudaStream_t cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    hgf_status st = HGF_OK;
    if (e == cudaSuccess) st = hgf_batch_run(b, cap);
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && st == HGF_OK) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (st != HGF_OK) return st;
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) {
    b->owner->sticky.store(HGF_ECUDA);
    b->owner->err = std::string("hgf_batch_launch_graph: ") + cudaGetErrorString(e);
    return HGF_ECUDA;
  }
  return HGF_OK;
}

hgf_status hgf_batch_destroy(hgf_batch *b) {
  if (!b) return HGF_OK;
  cudaSetDevice(b->owner->device);
  cudaDeviceSynchronize();
  destroy_batch(b);
  return HGF_OK;
}

}  // extern "C"
