// Request loop for multi-label aggregation (hgf_serve_* in include/hgf.h).
//
// One background thread admits queued requests in arrival order whenever a slot (a CUDA stream
// with its own pre-sized workspace) is free and the device-memory budget allows the request's
// guidance. Guidances (the resident inverse of hgf_prepare) are cached by (guidance_key, image
// shape, parameters), reference-counted by the requests using them and evicted least-recently-used
// when the budget needs room. A request's work is enqueued on its slot's stream: the prepare (on a
// cache miss) or a wait on the cached guidance's ready event, the fused aggregation + WTA, and a
// host callback that timestamps completion. Different requests therefore overlap on the device,
// and each request's arithmetic is the same kernels on the same inputs as hgf_aggregate, so its
// results do not depend on what else is in flight.
#include "hgf_internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

using namespace hgf;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct CacheKey {
  uint64_t key;
  int C, H, W, degree, basis, r, prec, combine, form, comp;
  double eps;
  bool operator<(const CacheKey &o) const {
    return std::tie(key, C, H, W, degree, basis, r, prec, combine, form, comp, eps) <
           std::tie(o.key, o.C, o.H, o.W, o.degree, o.basis, o.r, o.prec, o.combine, o.form,
                    o.comp, o.eps);
  }
};

struct CacheEntry {
  CacheKey key;
  hgf_guidance g;
  void *base = nullptr;
  size_t bytes = 0;
  int refs = 0;
  cudaEvent_t ready = nullptr;
  uint64_t last_use = 0;
};

enum ReqState { Q_QUEUED, Q_RUNNING, Q_DONE, Q_FAILED };

struct Req {
  uint64_t id = 0;
  hgf_request r{};
  int n = 0;
  size_t guidance_bytes = 0;
  Clock::time_point t_submit, t_admit, t_done;
  bool prepared_here = false;  // a cache miss: the slot ran the precompute
  std::atomic<int> finished{0};   // set by the host callback once the slot's work completed
  int state = Q_QUEUED;
  hgf_status status = HGF_EAGAIN;
  CacheEntry *entry = nullptr;
  int slot = -1;
  struct hgf_server *server = nullptr;
};

struct Slot {
  cudaStream_t stream = nullptr;
  hgf_ctx *ctx = nullptr;  // owns this slot's prepare / coefficient / key workspaces
  Req *req = nullptr;
  // timing events of the running request: start, precompute done, aggregation done
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
};

// Guidance-size class of the statistics: 0 for n <= 3, 1 for n <= 9, 2 above.
int size_class(int n) { return n <= 3 ? 0 : n <= 9 ? 1 : 2; }

size_t guidance_bytes_for(int C, int H, int W, int n, int r) {
  const size_t HW = (size_t)H * W;
  return (HW * ((size_t)C + n + packed_size(n) + n) + record_total_floats(H, W, n) + 64) *
         sizeof(float);
}

}  // namespace

struct hgf_server {
  int device = 0;
  size_t budget = 0, slot_bytes = 0, cache_bytes = 0, peak = 0;
  int max_queue = 0, max_pixels = 0, max_n = 0, num_sms = 0;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req *> queue;
  std::map<uint64_t, std::unique_ptr<Req>> reqs;
  std::map<CacheKey, std::unique_ptr<CacheEntry>> cache;
  uint64_t next_id = 1, use_clock = 0;
  bool stop = false;
  hgf_status sticky = HGF_OK;
  int inject_alloc_failures = 0;
  std::thread worker;
  // statistics
  uint64_t submitted = 0, completed = 0, failed = 0, rejected_busy = 0, rejected_nomem = 0;
  uint64_t hits = 0, misses = 0, evictions = 0;
  std::vector<double> latencies, queue_waits;
  double prep_ms[3] = {0, 0, 0}, agg_ms[3] = {0, 0, 0};
  uint64_t done_by_class[3] = {0, 0, 0};
  int running_big = 0;  // running requests with n = 19
  double units_done = 0.0;
  bool have_first = false;
  Clock::time_point first_submit, last_done;
  int running = 0, max_running = 0;

  size_t resident() const { return slot_bytes + cache_bytes; }

  // Frees least-recently-used unreferenced guidances until `need` more bytes fit the budget.
  bool make_room(size_t need) {
    while (resident() + need > budget) {
      CacheEntry *victim = nullptr;
      for (auto &kv : cache)
        if (kv.second->refs == 0 && (!victim || kv.second->last_use < victim->last_use))
          victim = kv.second.get();
      if (!victim) return false;
      cudaFreeAsync(victim->base, slots[0].stream);  // unreferenced: all its work has completed
      cudaEventDestroy(victim->ready);
      cache_bytes -= victim->bytes;
      ++evictions;
      cache.erase(victim->key);
    }
    return true;
  }

  void fail_request(Req *q, hgf_status st) {
    q->state = Q_FAILED;
    q->status = st;
    q->t_done = Clock::now();
    ++failed;
  }

  static void CUDART_CB on_done(void *p) {
    Req *q = static_cast<Req *>(p);
    q->t_done = Clock::now();
    q->finished.store(1, std::memory_order_release);
    q->server->cv_work.notify_all();
  }

  // Tries to start the request at the head of the queue on slot `si`: returns false when it has
  // to wait for memory (it stays queued).
  bool admit(Req *q, int si) {
    Slot &sl = slots[si];
    const hgf_request &r = q->r;
    CacheKey key{r.guidance_key, r.C, r.H, r.W, r.params.degree, r.params.basis, r.params.r,
                 r.params.inv_precision, r.params.combine, r.params.form,
                 r.params.compensated, r.params.eps};
    auto it = cache.find(key);
    CacheEntry *e = nullptr;
    // the request's device time starts here (a failed record fails the request below)
    cudaError_t err = cudaEventRecord(sl.ev[0], sl.stream);
    q->prepared_here = false;
    if (err == cudaSuccess && it != cache.end()) {
      e = it->second.get();
      ++hits;
      err = cudaStreamWaitEvent(sl.stream, e->ready, 0);
    } else if (err == cudaSuccess) {
      if (!make_room(q->guidance_bytes)) {
        if (running == 0) {  // nothing in flight will free memory: it cannot run
          fail_request(q, HGF_ENOMEM);
          return true;
        }
        return false;
      }
      ++misses;
      auto ent = std::make_unique<CacheEntry>();
      ent->key = key;
      ent->bytes = q->guidance_bytes;
      if (inject_alloc_failures > 0) {
        --inject_alloc_failures;
        fail_request(q, HGF_ENOMEM);
        return true;
      }
      if (cudaMallocAsync(&ent->base, ent->bytes, sl.stream) != cudaSuccess) {
        cudaGetLastError();
        fail_request(q, HGF_ENOMEM);
        return true;
      }
      hgf_guidance &g = ent->g;
      g.ctx = sl.ctx;
      g.C = r.C;
      g.H = r.H;
      g.W = r.W;
      g.n = q->n;
      g.degree = r.params.degree;
      g.basis = r.params.basis;
      g.r = std::min(r.params.r, std::max(r.H, r.W) - 1);
      g.eps = r.params.eps;
      g.inv_precision = r.params.inv_precision;
      g.combine = r.params.combine;
      g.form = r.params.form;
      g.compensated = r.params.compensated;
      const size_t HW = (size_t)r.H * r.W;
      g.rec = (float *)ent->base;
      g.img = g.rec + record_total_floats(r.H, r.W, g.n);
      g.G = g.img + (size_t)g.C * HW;
      g.minv = g.G + (size_t)g.n * HW;
      g.mu = g.minv + (size_t)packed_size(g.n) * HW;
      g.shift = g.mu + (size_t)g.n * HW;
      err = cudaEventCreateWithFlags(&ent->ready, cudaEventDisableTiming);
      if (err == cudaSuccess)
        err = launch_prepare(&g, r.img, sl.ctx->ws_prepare.ptr, sl.ctx->ws_prepare.size,
                             sl.stream, &sl.ctx->prof);
      if (err == cudaSuccess) err = cudaEventRecord(ent->ready, sl.stream);
      q->prepared_here = true;
      cache_bytes += ent->bytes;
      peak = std::max(peak, resident());
      e = ent.get();
      cache[key] = std::move(ent);
    }
    if (err == cudaSuccess) err = cudaEventRecord(sl.ev[1], sl.stream);
    if (err == cudaSuccess && e) {
      hgf_tuning t = sl.ctx->tuning;
      AggregatePlan plan = plan_aggregate(&e->g, r.L, t, num_sms);
      const size_t per_label = coef_plane_floats(q->n, (size_t)r.H * r.W) * sizeof(float);
      plan.chunk = std::max(1, std::min(plan.chunk, (int)(sl.ctx->ws_coef.size / per_label)));
      if (plan.onepass)  // the ring slots that fit the slot's workspace
        plan.onepass_ctas = std::max(
            1, std::min(plan.onepass_ctas,
                        (int)(sl.ctx->ws_coef.size / onepass_ring_bytes(q->n, e->g.r, 1))));
      err = launch_aggregate(&e->g, r.cost, r.cost_dtype, r.L, nullptr, r.labels, r.best,
                             (float *)sl.ctx->ws_coef.ptr,
                             (unsigned long long *)sl.ctx->ws_keys.ptr, plan, sl.stream,
                             &sl.ctx->prof);
    }
    if (err == cudaSuccess) err = cudaEventRecord(sl.ev[2], sl.stream);
    if (err == cudaSuccess) err = cudaLaunchHostFunc(sl.stream, on_done, q);
    if (!e) {
      sticky = HGF_ECUDA;
      fail_request(q, HGF_ECUDA);
      return true;
    }
    e->refs += 1;
    e->last_use = ++use_clock;
    q->entry = e;
    if (err != cudaSuccess) {
      sticky = HGF_ECUDA;
      fail_request(q, HGF_ECUDA);
      e->refs -= 1;
      return true;
    }
    q->state = Q_RUNNING;
    q->slot = si;
    q->t_admit = Clock::now();
    sl.req = q;
    ++running;
    if (size_class(q->n) == 2) ++running_big;
    max_running = std::max(max_running, running);
    return true;
  }

  // An n = 19 request waits while n = 19 requests hold slots - 1 slots (two or more slots).
  bool degree_blocked(const Req *q) const {
    return size_class(q->n) == 2 && slots.size() >= 2 &&
           running_big >= (int)slots.size() - 1;
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      for (auto &sl : slots) {  // completions
        Req *q = sl.req;
        if (q && q->finished.load(std::memory_order_acquire)) {
          q->state = Q_DONE;
          q->status = HGF_OK;
          q->entry->refs -= 1;
          latencies.push_back(ms_between(q->t_submit, q->t_done));
          queue_waits.push_back(ms_between(q->t_submit, q->t_admit));
          const int cls = size_class(q->n);
          float pm = 0.f, am = 0.f;
          if (cudaEventElapsedTime(&pm, sl.ev[0], sl.ev[1]) != cudaSuccess ||
              cudaEventElapsedTime(&am, sl.ev[1], sl.ev[2]) != cudaSuccess) {
            cudaGetLastError();
            pm = am = 0.f;
          }
          if (q->prepared_here) prep_ms[cls] += pm;
          agg_ms[cls] += am;
          ++done_by_class[cls];
          if (cls == 2) --running_big;
          units_done += (double)q->r.H * q->r.W * q->r.L;
          last_done = std::max(last_done, q->t_done);
          ++completed;
          sl.req = nullptr;
          --running;
          cv_done.notify_all();
        }
      }
      while (!queue.empty()) {  // admissions, in arrival order (but see degree_blocked)
        int free_slot = -1;
        for (size_t i = 0; i < slots.size(); ++i)
          if (!slots[i].req) {
            free_slot = (int)i;
            break;
          }
        if (free_slot < 0) break;
        auto pos = queue.begin();
        if (sticky == HGF_OK && degree_blocked(*pos)) {
          // the head waits for an n = 19 slot: a later request with n <= 9 may start first
          auto alt = std::next(pos);
          for (int k = 0; alt != queue.end() && k < 16 && size_class((*alt)->n) == 2; ++k) ++alt;
          if (alt == queue.end() || size_class((*alt)->n) == 2) break;
          pos = alt;
        }
        Req *q = *pos;
        if (sticky != HGF_OK) {
          fail_request(q, sticky);
          queue.erase(pos);
          cv_done.notify_all();
          continue;
        }
        if (!admit(q, free_slot)) break;
        queue.erase(pos);
        if (q->state == Q_FAILED) cv_done.notify_all();
      }
      if (stop && queue.empty() && running == 0) break;
      cv_work.wait_for(lk, std::chrono::microseconds(200));
    }
  }
};

extern "C" {

hgf_status hgf_serve_create(int device, size_t budget_bytes, int slots, int max_queue,
                            int max_pixels, int max_n, hgf_server **out) {
  if (!out || slots < 1 || slots > 16 || max_queue < 1 || max_pixels < 1 || max_n < 1 ||
      max_n > kMaxChannels)
    return HGF_EINVAL;
  *out = nullptr;
  hgf_server *s = new (std::nothrow) hgf_server;
  if (!s) return HGF_ENOMEM;
  s->device = device;
  s->budget = budget_bytes;
  s->max_queue = max_queue;
  s->max_pixels = max_pixels;
  s->max_n = max_n;
  auto cleanup = [&](hgf_status st) {
    for (auto &sl : s->slots) {
      for (auto ev : sl.ev)
        if (ev) cudaEventDestroy(ev);
      if (sl.stream) cudaStreamDestroy(sl.stream);
      hgf_destroy(sl.ctx);
    }
    delete s;
    return st;
  };
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(HGF_EINVAL);
  }
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t keep = ~0ull;  // keep freed guidance memory in the pool for the next admission
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  // per-slot workspaces for the largest admitted request: prepare scratch, 16 labels of
  // coefficient records at n = max_n (fewer labels per chunk are used when a request is bigger)
  // or the single-pass kernel's ring buffer at its largest (n = 9, r = 15), and the WTA keys
  const size_t prep = prepare_workspace_bytes(max_n, 1, max_pixels);
  const size_t coef =
      std::max((size_t)16 * coef_plane_floats(max_n, (size_t)max_pixels) * sizeof(float),
               onepass_ring_bytes(9, 15, s->num_sms * kFusedCtasPerSm));
  const size_t keys = (size_t)max_pixels * sizeof(unsigned long long);
  s->slot_bytes = (size_t)slots * (prep + coef + keys);
  if (s->slot_bytes > budget_bytes) return cleanup(HGF_ENOMEM);
  s->slots.resize(slots);
  for (auto &sl : s->slots) {
    if (hgf_create(device, &sl.ctx) != HGF_OK) return cleanup(HGF_ECUDA);
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess)
      return cleanup(HGF_ECUDA);
    for (auto &ev : sl.ev)
      if (cudaEventCreate(&ev) != cudaSuccess) return cleanup(HGF_ECUDA);
    for (auto pr : {std::make_pair(&sl.ctx->ws_prepare, prep), std::make_pair(&sl.ctx->ws_coef, coef),
                    std::make_pair(&sl.ctx->ws_keys, keys)}) {
      if (cudaMalloc(&pr.first->ptr, pr.second) != cudaSuccess) {
        cudaGetLastError();
        pr.first->ptr = nullptr;
        return cleanup(HGF_ENOMEM);
      }
      pr.first->size = pr.second;
    }
  }
  s->peak = s->resident();
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return HGF_OK;
}

hgf_status hgf_serve_submit(hgf_server *s, const hgf_request *req, uint64_t *id) {
  if (!s || !req || !id) return HGF_EINVAL;
  const hgf_request &r = *req;
  if (!r.img || !r.cost || !r.labels || r.L < 1 || r.H < 1 || r.W < 1 ||
      (r.C != 1 && r.C != 3) || r.params.r < 0 || !(r.params.eps > 0.0) ||
      (r.cost_dtype != HGF_F32 && r.cost_dtype != HGF_BF16 && r.cost_dtype != HGF_F16) ||
      (r.params.inv_precision != HGF_F64 && r.params.inv_precision != HGF_F32 &&
       r.params.inv_precision != HGF_DF64) ||
      (r.params.combine != HGF_COMBINE_ALPHA && r.params.combine != HGF_COMBINE_W3) ||
      (r.params.form != HGF_FORM_CENTRED && r.params.form != HGF_FORM_PAPER) ||
      (r.params.compensated != 0 && r.params.compensated != 1))
    return HGF_EINVAL;
  const int n = hgf_num_channels(r.C, r.params.degree, r.params.basis);
  if (n < 1 || !aggregate_supported(n)) return HGF_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(s->mu);
  ++s->submitted;
  if (s->sticky != HGF_OK) return s->sticky;
  hgf_guidance probe;
  probe.C = r.C;
  probe.n = n;
  probe.r = std::min(r.params.r, std::max(r.H, r.W) - 1);
  if ((long long)r.H * r.W > s->max_pixels || n > s->max_n || !aggregate_fits(&probe)) {
    ++s->rejected_nomem;
    return HGF_EUNSUPPORTED;
  }
  const size_t gb = guidance_bytes_for(r.C, r.H, r.W, n, probe.r);
  if (s->slot_bytes + gb > s->budget) {
    ++s->rejected_nomem;
    return HGF_ENOMEM;
  }
  if ((int)s->queue.size() >= s->max_queue) {
    ++s->rejected_busy;
    return HGF_EBUSY;
  }
  auto q = std::make_unique<Req>();
  q->id = s->next_id++;
  q->r = r;
  q->n = n;
  q->guidance_bytes = gb;
  q->server = s;
  q->t_submit = Clock::now();
  if (!s->have_first) {
    s->have_first = true;
    s->first_submit = q->t_submit;
  }
  *id = q->id;
  s->queue.push_back(q.get());
  s->reqs[q->id] = std::move(q);
  s->cv_work.notify_all();
  return HGF_OK;
}

hgf_status hgf_serve_poll(hgf_server *s, uint64_t id) {
  if (!s) return HGF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return HGF_EINVAL;
  const Req *q = it->second.get();
  if (q->state == Q_DONE) return HGF_OK;
  if (q->state == Q_FAILED) return q->status;
  return HGF_EAGAIN;
}

hgf_status hgf_serve_wait(hgf_server *s, uint64_t id, int timeout_ms) {
  if (!s) return HGF_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return HGF_EINVAL;
  Req *q = it->second.get();
  auto done = [&] { return q->state == Q_DONE || q->state == Q_FAILED; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    return HGF_ETIMEOUT;
  }
  return q->state == Q_DONE ? HGF_OK : q->status;
}

hgf_status hgf_serve_stats(hgf_server *s, hgf_serve_stats_t *o, int reset) {
  if (!s || !o) return HGF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *o = hgf_serve_stats_t{};
  o->submitted = s->submitted;
  o->completed = s->completed;
  o->failed = s->failed;
  o->rejected_busy = s->rejected_busy;
  o->rejected_nomem = s->rejected_nomem;
  o->cache_hits = s->hits;
  o->cache_misses = s->misses;
  o->evictions = s->evictions;
  std::vector<double> lat = s->latencies;
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) {
      size_t i = (size_t)std::ceil(p * lat.size()) - 1;
      return lat[std::min(i, lat.size() - 1)];
    };
    o->p50_ms = pct(0.50);
    o->p99_ms = pct(0.99);
    double sum = 0;
    for (double v : lat) sum += v;
    o->mean_ms = sum / lat.size();
    o->max_ms = lat.back();
  }
  if (s->have_first && s->completed > 0) {
    const double secs = ms_between(s->first_submit, s->last_done) / 1e3;
    o->mpixel_labels_per_s = secs > 0 ? s->units_done / secs / 1e6 : 0.0;
  }
  o->budget_bytes = s->budget;
  o->resident_bytes = s->resident();
  o->peak_bytes = s->peak;
  o->slots = (int)s->slots.size();
  o->max_concurrent = s->max_running;
  std::vector<double> qw = s->queue_waits;
  if (!qw.empty()) {
    std::sort(qw.begin(), qw.end());
    double sum = 0;
    for (double v : qw) sum += v;
    o->queue_mean_ms = sum / qw.size();
    o->queue_p99_ms = qw[std::min(qw.size() - 1, (size_t)std::ceil(0.99 * qw.size()) - 1)];
  }
  for (int c = 0; c < 3; ++c) {
    o->prepare_ms_total[c] = s->prep_ms[c];
    o->aggregate_ms_total[c] = s->agg_ms[c];
    o->completed_by_class[c] = s->done_by_class[c];
  }
  if (reset) {
    s->submitted = s->completed = s->failed = s->rejected_busy = s->rejected_nomem = 0;
    s->hits = s->misses = s->evictions = 0;
    s->latencies.clear();
    s->queue_waits.clear();
    for (int c = 0; c < 3; ++c) {
      s->prep_ms[c] = s->agg_ms[c] = 0;
      s->done_by_class[c] = 0;
    }
    s->units_done = 0;
    s->have_first = false;
    s->max_running = s->running;
  }
  return HGF_OK;
}

hgf_status hgf_serve_inject_alloc_failures(hgf_server *s, int count) {
  if (!s || count < 0) return HGF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->inject_alloc_failures = count;
  return HGF_OK;
}

hgf_status hgf_serve_destroy(hgf_server *s) {
  if (!s) return HGF_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  for (auto &kv : s->cache) {
    cudaFree(kv.second->base);
    if (kv.second->ready) cudaEventDestroy(kv.second->ready);
  }
  for (auto &sl : s->slots) {
    for (auto ev : sl.ev)
      if (ev) cudaEventDestroy(ev);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    hgf_destroy(sl.ctx);
  }
  delete s;
  return HGF_OK;
}

}  // extern "C"
