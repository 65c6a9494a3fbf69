// Batches of independent aggregation jobs (hgf_batch_* in include/hgf.h).
//
// Every job gets its own guidance handle; jobs are assigned to `streams` internal streams,
// largest work (H*W*L) first onto the least-loaded stream, and each internal stream owns a context
// whose workspaces are sized at creation for its largest job. A run records an event on the
// caller's stream, makes every internal stream wait on it, enqueues each job's precompute and
// aggregation on its stream, and makes the caller's stream wait on an event from each internal
// stream: a fork/join that CUDA graph capture follows, so the whole batch becomes one graph.
// With the context tuned to the single-pass kernel (hgf_tuning.kernel = 1), the jobs that kernel
// takes in a batch (RGB degree 1 or 2) are aggregated together instead: after every precompute,
// one persistent launch on the caller's stream takes their work items from one counter (per 40
// jobs), followed by their WTA unpacking; the other jobs run on their streams as before.
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
  // persistent single-pass launch over the eligible jobs
  std::vector<int> joint;                   // job indices in the joint launch
  std::vector<cudaEvent_t> prepared;        // per lane: its precomputes are done
  void *joint_mem = nullptr;                // ring slots | work counters | WTA keys
  float *ring = nullptr;
  size_t ring_stride = 0;
  unsigned long long *counters = nullptr;
  int n_counters = 0;
  std::vector<unsigned long long *> keys;   // per joint job
  int grid = 0;
};

namespace {

void destroy_batch(hgf_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto *g : b->guid) free_guidance(g);
  for (cudaEvent_t e : b->prepared)
    if (e) cudaEventDestroy(e);
  if (b->joint_mem) cudaFree(b->joint_mem);
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
  if (ctx->tuning.kernel == 1) {
    for (int i = 0; i < njobs; ++i)
      if (b->plans[i].onepass && onepass_batch_eligible(b->guid[i])) b->joint.push_back(i);
  }
  if (!b->joint.empty()) {
    b->grid = std::max(1, ctx->num_sms) * kFusedCtasPerSm;
    for (int i : b->joint) b->ring_stride = std::max(b->ring_stride,
                                                     onepass_batch_ring_floats(b->guid[i]));
    b->n_counters = ((int)b->joint.size() + kOnepassBatchJobsPerLaunch - 1) /
                    kOnepassBatchJobsPerLaunch;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    size_t bytes = up((size_t)b->grid * b->ring_stride * sizeof(float)) +
                   up((size_t)b->n_counters * sizeof(unsigned long long));
    for (int i : b->joint) bytes += up((size_t)jobs[i].H * jobs[i].W * 8);
    if (cudaMalloc(&b->joint_mem, bytes) != cudaSuccess) {
      cudaGetLastError();
      destroy_batch(b);
      return HGF_ENOMEM;
    }
    char *p = (char *)b->joint_mem;
    b->ring = (float *)p;
    p += up((size_t)b->grid * b->ring_stride * sizeof(float));
    b->counters = (unsigned long long *)p;
    p += up((size_t)b->n_counters * sizeof(unsigned long long));
    for (int i : b->joint) {
      b->keys.push_back((unsigned long long *)p);
      p += up((size_t)jobs[i].H * jobs[i].W * 8);
    }
    b->prepared.resize(b->lanes.size(), nullptr);
    for (auto &e : b->prepared)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        destroy_batch(b);
        return HGF_ECUDA;
      }
  }
  *out = b;
  return HGF_OK;
}

hgf_status hgf_batch_run(hgf_batch *b, void *stream) {
  if (!b) return HGF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<char> in_joint(b->jobs.size(), 0);
  for (int i : b->joint) in_joint[i] = 1;
  cudaError_t e = cudaEventRecord(b->fork, s);
  for (size_t li = 0; li < b->lanes.size(); ++li) {
    auto &l = b->lanes[li];
    if (e == cudaSuccess) e = cudaStreamWaitEvent(l.stream, b->fork, 0);
    // every precompute first (the joint launch waits for them), then the lane's own jobs
    for (int i : l.jobs) {
      if (e != cudaSuccess) break;
      e = launch_prepare(b->guid[i], b->jobs[i].img, l.ctx->ws_prepare.ptr,
                         l.ctx->ws_prepare.size, l.stream, &b->owner->prof);
    }
    if (e == cudaSuccess && !b->prepared.empty()) {
      e = cudaEventRecord(b->prepared[li], l.stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->prepared[li], 0);
    }
    for (int i : l.jobs) {
      if (e != cudaSuccess) break;
      if (in_joint[i]) continue;
      const hgf_job &j = b->jobs[i];
      e = launch_aggregate(b->guid[i], j.cost, j.cost_dtype, j.L, j.filtered, j.labels, j.best,
                           (float *)l.ctx->ws_coef.ptr,
                           (unsigned long long *)l.ctx->ws_keys.ptr, b->plans[i], l.stream,
                           &b->owner->prof);
    }
    if (e == cudaSuccess) e = cudaEventRecord(l.done, l.stream);
  }
  if (e == cudaSuccess && !b->joint.empty()) {
    // the joint launch on the caller's stream, after every lane's precomputes
    std::vector<OnepassBatchJob> jj;
    for (size_t k = 0; k < b->joint.size() && e == cudaSuccess; ++k) {
      const int i = b->joint[k];
      const hgf_job &j = b->jobs[i];
      const bool wta = j.labels || j.best;
      if (wta)
        e = cudaMemsetAsync(b->keys[k], 0xff, (size_t)j.H * j.W * sizeof(unsigned long long), s);
      jj.push_back(OnepassBatchJob{b->guid[i], j.cost, j.cost_dtype, j.L, j.filtered,
                                   wta ? b->keys[k] : nullptr, b->plans[i].nominal});
    }
    if (e == cudaSuccess)
      e = cudaMemsetAsync(b->counters, 0, (size_t)b->n_counters * sizeof(unsigned long long), s);
    int *status = device_status_ptr();
    if (e == cudaSuccess && !status) e = cudaErrorInvalidValue;
    if (e == cudaSuccess)
      e = launch_onepass_batch(jj.data(), (int)jj.size(), b->ring, b->ring_stride, b->grid,
                               b->owner->tuning.band_rows, b->counters, status, s,
                               &b->owner->prof);
    for (size_t k = 0; k < b->joint.size() && e == cudaSuccess; ++k) {
      const hgf_job &j = b->jobs[b->joint[k]];
      if (j.labels || j.best)
        e = launch_wta_finalize(b->keys[k], j.H * j.W, j.labels, j.best, s, &b->owner->prof);
    }
  }
  for (auto &l : b->lanes)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, l.done, 0);
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
