// C ABI of libhgf: argument checks, error mapping, context workspaces and dispatch to the
// kernels in hgf_prepare.cu, hgf_aggregate.cu and hgf_plain.cu.
#include "hgf_internal.cuh"

#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>
#include <new>

using namespace hgf;

namespace {

hgf_status set_err(hgf_ctx *ctx, hgf_status st, const char *fmt, ...) {
  if (!ctx) return st;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  ctx->err = buf;
  return st;
}

// " in <step>" for the launch or set-up call that failed (failed_step), consumed here.
std::string failed_suffix() {
  const char *st = failed_step();
  failed_step() = nullptr;
  return st ? std::string(" in ") + st : std::string();
}

hgf_status cuda_fail(hgf_ctx *ctx, cudaError_t e, const char *where) {
  ctx->sticky.store(HGF_ECUDA);
  const std::string in = failed_suffix();
  return set_err(ctx, HGF_ECUDA, "%s: %s (%s)%s", where, cudaGetErrorName(e),
                 cudaGetErrorString(e), in.c_str());
}

// Enters an API call on ctx: refuses work after a CUDA failure, clears a non-sticky error that
// an earlier call left on this thread (a sticky one comes back from the next call anyway) and
// makes the device current.
hgf_status enter(hgf_ctx *ctx) {
  if (!ctx) return HGF_EINVAL;
  if (ctx->sticky.load() != HGF_OK)
    return HGF_ECUDA;
  cudaGetLastError();
  failed_step() = nullptr;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  return HGF_OK;
}

bool is_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
  return st != cudaStreamCaptureStatusNone;
}

// Grows a workspace to at least `bytes` (caller holds ctx->mu). Growing waits for all work on
// the device (the old buffer may still be in use), so it is refused while `s` is being captured
// into a graph: make one uncaptured call of the same shape first.
hgf_status grow(hgf_ctx *ctx, Workspace &w, size_t bytes, cudaStream_t s) {
  if (w.size >= bytes) return HGF_OK;
  if (is_capturing(s)) {
    ctx->err = "workspace must grow to " + std::to_string(bytes) +
               " bytes; make one uncaptured call first";
    return HGF_EINVAL;
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    ctx->sticky.store(HGF_ECUDA);
    ctx->err = std::string("cudaDeviceSynchronize: ") + cudaGetErrorString(e);
    return HGF_ECUDA;
  }
  if (w.ptr) cudaFree(w.ptr);
  w.ptr = nullptr;
  w.size = 0;
  e = cudaMalloc(&w.ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();  // allocation failures are not sticky
    w.ptr = nullptr;
    ctx->err = "cannot allocate " + std::to_string(bytes) + " bytes of workspace";
    return HGF_ENOMEM;
  }
  w.size = bytes;
  return HGF_OK;
}

// CUDA failure with ctx->mu held.
hgf_status cuda_fail_locked(hgf_ctx *ctx, cudaError_t e, const char *where) {
  ctx->sticky.store(HGF_ECUDA);
  ctx->err = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")" +
             failed_suffix();
  return HGF_ECUDA;
}

bool valid_dtype_cost(int d) { return d == HGF_F32 || d == HGF_BF16 || d == HGF_F16; }

size_t dtype_size(int d) { return d == HGF_F32 ? 4 : d == HGF_F64 ? 8 : 2; }

hgf_status check_params(hgf_ctx *ctx, int C, int H, int W, const hgf_params *p, int *n_out) {
  if (!p) return set_err(ctx, HGF_EINVAL, "params is NULL");
  if (C != 1 && C != 3) return set_err(ctx, HGF_EINVAL, "C must be 1 or 3 (got %d)", C);
  if (H < 1 || W < 1) return set_err(ctx, HGF_EINVAL, "H and W must be >= 1 (got %d x %d)", H, W);
  if ((long long)H * W > (1ll << 31) / 64)
    return set_err(ctx, HGF_EUNSUPPORTED, "image of %d x %d pixels is too large", H, W);
  if (p->r < 0) return set_err(ctx, HGF_EINVAL, "r must be >= 0 (got %d)", p->r);
  if (!(p->eps > 0.0)) return set_err(ctx, HGF_EINVAL, "eps must be > 0 (the recursion divides by it)");
  if (p->degree < 1) return set_err(ctx, HGF_EINVAL, "degree must be >= 1");
  if (p->basis != HGF_BASIS_MONOMIAL && p->basis != HGF_BASIS_POWERS)
    return set_err(ctx, HGF_EINVAL, "unknown basis %d", p->basis);
  if (p->inv_precision != HGF_F64 && p->inv_precision != HGF_F32 &&
      p->inv_precision != HGF_DF64)
    return set_err(ctx, HGF_EINVAL, "inv_precision must be HGF_F64, HGF_DF64 or HGF_F32");
  if (p->combine != HGF_COMBINE_ALPHA && p->combine != HGF_COMBINE_W3)
    return set_err(ctx, HGF_EINVAL, "unknown combine %d", p->combine);
  if (p->form != HGF_FORM_CENTRED && p->form != HGF_FORM_PAPER)
    return set_err(ctx, HGF_EINVAL, "unknown form %d", p->form);
  if (p->compensated != 0 && p->compensated != 1)
    return set_err(ctx, HGF_EINVAL, "compensated must be 0 or 1");
  int n = hgf_num_channels(C, p->degree, p->basis);
  if (n < 1) return set_err(ctx, HGF_EUNSUPPORTED, "C=%d degree=%d basis=%d gives n > %d", C,
                            p->degree, p->basis, kMaxChannels);
  if (!aggregate_supported(n))
    return set_err(ctx, HGF_EUNSUPPORTED, "n = %d guidance channels are not built", n);
  *n_out = n;
  return HGF_OK;
}

// Windows wider than the image behave like windows covering it: clamp r for the kernels.
int effective_radius(int r, int H, int W) { return std::min(r, std::max(H, W) - 1); }

hgf_status alloc_guidance(hgf_ctx *ctx, int C, int H, int W, int n, const hgf_params *p,
                          hgf_guidance **out) {
  hgf_guidance *g = new (std::nothrow) hgf_guidance;
  if (!g) return set_err(ctx, HGF_ENOMEM, "host allocation failed");
  g->ctx = ctx;
  g->C = C;
  g->H = H;
  g->W = W;
  g->n = n;
  g->degree = p->degree;
  g->basis = p->basis;
  g->r = effective_radius(p->r, H, W);
  g->eps = p->eps;
  g->inv_precision = p->inv_precision;
  g->combine = p->combine;
  g->form = p->form;
  g->compensated = p->compensated;
  const size_t HW = (size_t)H * W;
  const size_t rec_floats = record_total_floats(H, W, n);
  const size_t floats = HW * ((size_t)C + n + packed_size(n) + n) + rec_floats + 64;
  float *base = nullptr;
  cudaError_t e = cudaMalloc(&base, floats * sizeof(float));
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete g;
    return set_err(ctx, HGF_ENOMEM, "cannot allocate %zu bytes for the guidance",
                   floats * sizeof(float));
  }
  g->rec = base;  // first: tensor copies of record rows need the allocation's alignment
  g->img = g->rec + rec_floats;
  g->G = g->img + (size_t)C * HW;
  g->minv = g->G + (size_t)n * HW;
  g->mu = g->minv + (size_t)packed_size(n) * HW;
  g->shift = g->mu + (size_t)n * HW;
  *out = g;
  return HGF_OK;
}

bool same_shape(const hgf_guidance *g, int C, int H, int W, const hgf_params *p) {
  return g && g->C == C && g->H == H && g->W == W && g->degree == p->degree &&
         g->basis == p->basis && g->r == effective_radius(p->r, H, W) && g->eps == p->eps &&
         g->inv_precision == p->inv_precision && g->combine == p->combine && g->form == p->form &&
         g->compensated == p->compensated;
}

hgf_status prepare_locked(hgf_ctx *ctx, hgf_guidance *g, const float *img, cudaStream_t s) {
  hgf_status st = grow(ctx, ctx->ws_prepare, prepare_workspace_bytes(g->n, g->H, g->W), s);
  if (st != HGF_OK) return st;
  cudaError_t e = launch_prepare(g, img, ctx->ws_prepare.ptr, ctx->ws_prepare.size, s,
                                 &ctx->prof);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_prepare");
  return HGF_OK;
}

hgf_status check_outputs(hgf_ctx *ctx, const hgf_guidance *g, const void *cost, int cost_dtype,
                         int L, const void *filtered, int filtered_dtype, const void *labels,
                         const void *best) {
  if (!g) return set_err(ctx, HGF_EINVAL, "guidance is NULL");
  if (g->ctx != ctx) return set_err(ctx, HGF_EINVAL, "guidance belongs to another context");
  if (!cost) return set_err(ctx, HGF_EINVAL, "cost is NULL");
  if (!valid_dtype_cost(cost_dtype))
    return set_err(ctx, HGF_EINVAL, "cost dtype must be HGF_F32, HGF_BF16 or HGF_F16");
  if (L < 1) return set_err(ctx, HGF_EINVAL, "L must be >= 1 (got %d)", L);
  if ((long long)L * g->H * g->W > (1ll << 40))
    return set_err(ctx, HGF_EUNSUPPORTED, "cost volume too large");
  if (!filtered && !labels && !best) return set_err(ctx, HGF_EINVAL, "no output requested");
  if (filtered && filtered_dtype != HGF_F32)
    return set_err(ctx, HGF_EINVAL, "filtered dtype must be HGF_F32");
  return HGF_OK;
}

hgf_status aggregate_locked(hgf_ctx *ctx, const hgf_guidance *g, const void *cost,
                            int cost_dtype, int L, void *filtered, int32_t *labels, float *best,
                            cudaStream_t s, float *margin = nullptr) {
  if (!aggregate_fits(g)) {
    if (g->form != HGF_FORM_CENTRED)
      return set_err(ctx, HGF_EUNSUPPORTED, "the paper form needs 2r+1 < %d", kStripThreads);
    // windows too wide for the streaming kernels' shared-memory rings: the plain kernels
    // compute the same result for any radius
    int chunk = 1;
    size_t need = plain_workspace_bytes(g, L, &chunk);
    const size_t qbytes = filtered ? 0 : (size_t)L * g->H * g->W * sizeof(float);
    hgf_status st = grow(ctx, ctx->ws_plain, need + qbytes, s);
    if (st != HGF_OK) return st;
    float *q = filtered ? (float *)filtered : (float *)((char *)ctx->ws_plain.ptr + need);
    cudaError_t e = launch_aggregate_plain(g, cost, cost_dtype, L, q, labels, best,
                                           ctx->ws_plain.ptr, chunk, s, &ctx->prof, margin);
    if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_aggregate (wide window)");
    return HGF_OK;
  }
  AggregatePlan plan = plan_aggregate(g, L, ctx->tuning, ctx->num_sms);
  hgf_status st = grow(ctx, ctx->ws_coef, aggregate_coef_bytes(g, plan), s);
  if (st == HGF_OK)
    st = grow(ctx, ctx->ws_keys,
              (size_t)g->H * g->W * (margin ? 2 : 1) * sizeof(unsigned long long), s);
  if (st != HGF_OK) return st;
  cudaError_t e = launch_aggregate(g, cost, cost_dtype, L, (float *)filtered, labels, best,
                                   (float *)ctx->ws_coef.ptr,
                                   (unsigned long long *)ctx->ws_keys.ptr, plan, s, &ctx->prof,
                                   nullptr, margin);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_aggregate");
  return HGF_OK;
}

// hgf_guidance_update + hgf_aggregate with ctx->mu held and arguments checked; the aggregation
// waits for `before_aggregate` when given (hgf_filter_host: the cost upload, which then overlaps
// the guidance precompute).
hgf_status filter_locked(hgf_ctx *ctx, hgf_guidance *g, const float *img, const void *cost,
                         int cost_dtype, int L, void *filtered, int32_t *labels, float *best,
                         cudaStream_t s, cudaEvent_t before_aggregate = nullptr) {
  hgf_status st = prepare_locked(ctx, g, img, s);
  if (st != HGF_OK) return st;
  if (before_aggregate) {
    cudaError_t e = cudaStreamWaitEvent(s, before_aggregate, 0);
    if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_filter wait");
  }
  return aggregate_locked(ctx, g, cost, cost_dtype, L, filtered, labels, best, s);
}

}  // namespace

namespace hgf {
hgf_status alloc_guidance_checked(hgf_ctx *ctx, int C, int H, int W, const hgf_params *p,
                                  hgf_guidance **out) {
  int n = 0;
  hgf_status st = check_params(ctx, C, H, W, p, &n);
  if (st != HGF_OK) return st;
  return alloc_guidance(ctx, C, H, W, n, p, out);
}
void free_guidance(hgf_guidance *g) {
  if (!g) return;
  cudaFree(g->rec);
  delete g;
}
}  // namespace hgf

extern "C" {

int hgf_num_channels(int C, int degree, int basis) {
  BasisTable t;
  if (!make_basis_table(C, degree, basis, &t)) return 0;
  return t.n;
}

hgf_status hgf_create(int device, hgf_ctx **out) {
  if (!out) return HGF_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return HGF_EINVAL;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return HGF_ECUDA;
  }
  hgf_ctx *ctx = new (std::nothrow) hgf_ctx;
  if (!ctx) return HGF_ENOMEM;
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  // commit hgf_aggregate_static's fixed scratch now, while the caller expects allocations; if it
  // fails (no memory left), that entry point retries and reports HGF_ENOMEM
  if (static_scratch_init(device) != cudaSuccess) cudaGetLastError();
  *out = ctx;
  return HGF_OK;
}

hgf_status hgf_destroy(hgf_ctx *ctx) {
  if (!ctx) return HGF_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->host_guidance_right) {
    cudaFree(ctx->host_guidance_right->rec);
    delete ctx->host_guidance_right;
  }
  if (ctx->host_guidance) {
    cudaFree(ctx->host_guidance->rec);
    delete ctx->host_guidance;
  }
  for (auto &rec : ctx->prof.recs) {
    cudaEventDestroy(rec.a);
    cudaEventDestroy(rec.b);
  }
  for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
  for (Workspace *w : {&ctx->ws_prepare, &ctx->ws_coef, &ctx->ws_keys, &ctx->ws_plain,
                       &ctx->ws_io, &ctx->ws_grad})
    if (w->ptr) cudaFree(w->ptr);
  if (ctx->io_fork) cudaEventDestroy(ctx->io_fork);
  if (ctx->io_done) cudaEventDestroy(ctx->io_done);
  if (ctx->io_stream) cudaStreamDestroy(ctx->io_stream);
  delete ctx;
  return HGF_OK;
}

const char *hgf_last_error(const hgf_ctx *ctx) {
  if (!ctx) return "context is NULL";
  return ctx->err.c_str();
}

hgf_status hgf_make_guidance(hgf_ctx *ctx, const float *img, int C, int H, int W, int degree,
                             int basis, float *G_out, int *n_out, void *stream) {
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!img || !G_out) return set_err(ctx, HGF_EINVAL, "img and G_out must be non-NULL");
  if (H < 1 || W < 1 || (C != 1 && C != 3)) return set_err(ctx, HGF_EINVAL, "bad image shape");
  BasisTable bt;
  if (!make_basis_table(C, degree, basis, &bt))
    return set_err(ctx, HGF_EUNSUPPORTED, "unsupported degree/basis");
  if (n_out) *n_out = bt.n;
  cudaError_t e = launch_make_guidance(img, C, H, W, bt, G_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "hgf_make_guidance");
  return HGF_OK;
}

hgf_status hgf_prepare(hgf_ctx *ctx, const float *img, int C, int H, int W,
                       const hgf_params *params, void *stream, hgf_guidance **out) {
  NvtxRange nvtx_range("hgf_prepare");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!out) return set_err(ctx, HGF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!img) return set_err(ctx, HGF_EINVAL, "img is NULL");
  int n = 0;
  st = check_params(ctx, C, H, W, params, &n);
  if (st != HGF_OK) return st;
  hgf_guidance *g = nullptr;
  st = alloc_guidance(ctx, C, H, W, n, params, &g);
  if (st != HGF_OK) return st;
  {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    st = prepare_locked(ctx, g, img, (cudaStream_t)stream);
  }
  if (st != HGF_OK) {
    cudaFree(g->rec);
    delete g;
    return st;
  }
  *out = g;
  return HGF_OK;
}

hgf_status hgf_guidance_release(hgf_guidance *g) {
  if (!g) return HGF_OK;
  cudaSetDevice(g->ctx->device);
  cudaFree(g->rec);
  delete g;
  return HGF_OK;
}

hgf_status hgf_guidance_info(const hgf_guidance *g, int *C, int *H, int *W, int *n, int *r,
                             double *eps) {
  if (!g) return HGF_EINVAL;
  if (C) *C = g->C;
  if (H) *H = g->H;
  if (W) *W = g->W;
  if (n) *n = g->n;
  if (r) *r = g->r;
  if (eps) *eps = g->eps;
  return HGF_OK;
}

hgf_status hgf_guidance_export(hgf_ctx *ctx, const hgf_guidance *g, float *minv_out,
                               float *mu_out, void *stream) {
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!g || g->ctx != ctx) return set_err(ctx, HGF_EINVAL, "bad guidance handle");
  if (g->form != HGF_FORM_CENTRED)
    return set_err(ctx, HGF_EUNSUPPORTED, "export holds the centred form's inverse only");
  cudaError_t e = launch_export(g, minv_out, mu_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "hgf_guidance_export");
  return HGF_OK;
}

hgf_status hgf_set_tuning(hgf_ctx *ctx, const hgf_tuning *t) {
  if (!ctx || !t) return HGF_EINVAL;
  if (t->labels_per_pass != 0 && t->labels_per_pass != 1 && t->labels_per_pass != 2 &&
      t->labels_per_pass != 4 && t->labels_per_pass != 8)
    return set_err(ctx, HGF_EINVAL, "labels_per_pass must be 0, 1, 2, 4 or 8");
  if (t->band_rows < 0 || t->chunk_labels < 0)
    return set_err(ctx, HGF_EINVAL, "band_rows and chunk_labels must be >= 0");
  if (t->apply_mode < 0 || t->apply_mode > 2)
    return set_err(ctx, HGF_EINVAL, "apply_mode must be 0, 1 or 2");
  if (t->kernel < 0 || t->kernel > 2) return set_err(ctx, HGF_EINVAL, "kernel must be 0, 1 or 2");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  ctx->tuning = *t;
  return HGF_OK;
}

hgf_status hgf_autotune(hgf_ctx *ctx, const hgf_guidance *g, const void *cost, int cost_dtype,
                        int L, int32_t *labels, int reps, hgf_tuning *best, int *ncand,
                        void *stream) {
  NvtxRange nvtx_range("hgf_autotune");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  st = check_outputs(ctx, g, cost, cost_dtype, L, nullptr, HGF_F32, labels, nullptr);
  if (st != HGF_OK) return st;
  if (!labels || reps < 1) return set_err(ctx, HGF_EINVAL, "labels is NULL or reps < 1");
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  // first round: the kernel path and the two-kernel path's labels per pass, chunk and ring
  // mode, all with the automatic row bands
  std::vector<hgf_tuning> cands;
  for (int K : {2, 4, 8}) {
    if (K != 2 && coef_smem(g->n, g->C, K, g->r) > 227 * 1024) continue;
    for (int chunk : {0, 64, 16}) {
      if (chunk != 0 && chunk >= L) continue;
      for (int apply : {2, 1}) cands.push_back(hgf_tuning{K, 0, chunk, apply, 2});
    }
  }
  if (onepass_fits(g)) cands.push_back(hgf_tuning{0, 0, 0, 0, 1});
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const hgf_tuning saved = ctx->tuning;
  float best_ms = 0.f;
  hgf_tuning pick = cands.front();
  int timed = 0;
  auto time_all = [&](const std::vector<hgf_tuning> &list) {
    for (size_t i = 0; i < list.size() && e == cudaSuccess && st == HGF_OK; ++i) {
      ctx->tuning = list[i];
      st = aggregate_locked(ctx, g, cost, cost_dtype, L, nullptr, labels, nullptr, s);
      if (st != HGF_OK) break;
      e = cudaEventRecord(a, s);
      for (int k = 0; k < reps && e == cudaSuccess && st == HGF_OK; ++k)
        st = aggregate_locked(ctx, g, cost, cost_dtype, L, nullptr, labels, nullptr, s);
      if (e == cudaSuccess) e = cudaEventRecord(b, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e == cudaSuccess && (timed == 0 || ms < best_ms)) {
        best_ms = ms;
        pick = list[i];
      }
      ++timed;
    }
  };
  time_all(cands);
  // second round: row-band heights (tile shape along y) for the winner: a half, a quarter and an
  // eighth of the image height, at least 4r + 8 rows (bands shorter than their warm-up waste it)
  std::vector<hgf_tuning> bands;
  for (int div : {2, 4, 8}) {
    const int rows = (g->H + div - 1) / div;
    if (rows < 4 * g->r + 8 || rows >= g->H) continue;
    hgf_tuning t = pick;
    t.band_rows = rows;
    bands.push_back(t);
  }
  time_all(bands);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st != HGF_OK || e != cudaSuccess) {
    ctx->tuning = saved;
    return st != HGF_OK ? st : cuda_fail_locked(ctx, e, "hgf_autotune");
  }
  ctx->tuning = pick;
  if (best) *best = pick;
  if (ncand) *ncand = timed;
  return HGF_OK;
}

hgf_status hgf_aggregate(hgf_ctx *ctx, const hgf_guidance *g, const void *cost, int cost_dtype,
                         int L, void *filtered, int filtered_dtype, int32_t *labels, float *best,
                         void *stream) {
  NvtxRange nvtx_range("hgf_aggregate");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  st = check_outputs(ctx, g, cost, cost_dtype, L, filtered, filtered_dtype, labels, best);
  if (st != HGF_OK) return st;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  return aggregate_locked(ctx, g, cost, cost_dtype, L, filtered, labels, best,
                          (cudaStream_t)stream);
}

hgf_status hgf_filter(hgf_ctx *ctx, hgf_guidance *g, const float *img, const void *cost,
                      int cost_dtype, int L, void *filtered, int filtered_dtype, int32_t *labels,
                      float *best, void *stream) {
  NvtxRange nvtx_range("hgf_filter");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!img) return set_err(ctx, HGF_EINVAL, "img is NULL");
  st = check_outputs(ctx, g, cost, cost_dtype, L, filtered, filtered_dtype, labels, best);
  if (st != HGF_OK) return st;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  return filter_locked(ctx, g, img, cost, cost_dtype, L, filtered, labels, best,
                       (cudaStream_t)stream);
}

hgf_status hgf_aggregate_margin(hgf_ctx *ctx, const hgf_guidance *g, const void *cost,
                                int cost_dtype, int L, int32_t *labels, float *best,
                                float *margin, void *stream) {
  NvtxRange nvtx_range("hgf_aggregate_margin");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!margin) return set_err(ctx, HGF_EINVAL, "margin is NULL");
  st = check_outputs(ctx, g, cost, cost_dtype, L, nullptr, HGF_F32, labels, best ? best : margin);
  if (st != HGF_OK) return st;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  return aggregate_locked(ctx, g, cost, cost_dtype, L, nullptr, labels, best,
                          (cudaStream_t)stream, margin);
}

hgf_status hgf_aggregate_plain(hgf_ctx *ctx, const hgf_guidance *g, const void *cost,
                               int cost_dtype, int L, void *filtered, int filtered_dtype,
                               int32_t *labels, float *best, void *stream) {
  NvtxRange nvtx_range("hgf_aggregate_plain");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  st = check_outputs(ctx, g, cost, cost_dtype, L, filtered, filtered_dtype, labels, best);
  if (st != HGF_OK) return st;
  if (g->form != HGF_FORM_CENTRED)
    return set_err(ctx, HGF_EUNSUPPORTED, "the plain kernels compute the centred form only");
  cudaStream_t s = (cudaStream_t)stream;
  int chunk = 1;
  size_t need = plain_workspace_bytes(g, L, &chunk);
  const size_t qbytes = filtered ? 0 : (size_t)L * g->H * g->W * sizeof(float);
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  st = grow(ctx, ctx->ws_plain, need + qbytes, s);
  if (st != HGF_OK) return st;
  float *q = filtered ? (float *)filtered : (float *)((char *)ctx->ws_plain.ptr + need);
  cudaError_t e = launch_aggregate_plain(g, cost, cost_dtype, L, q, labels, best,
                                         ctx->ws_plain.ptr, chunk, s, &ctx->prof);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_aggregate_plain");
  return HGF_OK;
}

hgf_status hgf_wta(hgf_ctx *ctx, const void *filtered, int dtype, int L, int H, int W,
                   int32_t *labels, float *best, void *stream) {
  NvtxRange nvtx_range("hgf_wta");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!filtered || (!labels && !best)) return set_err(ctx, HGF_EINVAL, "NULL argument");
  if (dtype != HGF_F32) return set_err(ctx, HGF_EINVAL, "hgf_wta takes HGF_F32 volumes");
  if (L < 1 || H < 1 || W < 1) return set_err(ctx, HGF_EINVAL, "bad shape");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = launch_wta((const float *)filtered, L, H, W, labels, best,
                             (cudaStream_t)stream, &ctx->prof);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "hgf_wta");
  return HGF_OK;
}

hgf_status hgf_wta_margin(hgf_ctx *ctx, const void *filtered, int dtype, int L, int H, int W,
                          int32_t *labels, float *best, float *margin, void *stream) {
  NvtxRange nvtx_range("hgf_wta_margin");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!filtered || !margin) return set_err(ctx, HGF_EINVAL, "NULL argument");
  if (dtype != HGF_F32) return set_err(ctx, HGF_EINVAL, "hgf_wta_margin takes HGF_F32 volumes");
  if (L < 1 || H < 1 || W < 1) return set_err(ctx, HGF_EINVAL, "bad shape");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = launch_wta((const float *)filtered, L, H, W, labels, best,
                             (cudaStream_t)stream, &ctx->prof, margin);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "hgf_wta_margin");
  return HGF_OK;
}

hgf_status hgf_filter_host(hgf_ctx *ctx, const float *img, int C, int H, int W,
                           const hgf_params *params, const void *cost, int cost_dtype, int L,
                           int32_t *labels, float *best, void *stream) {
  NvtxRange nvtx_range("hgf_filter_host");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!img || !cost || (!labels && !best)) return set_err(ctx, HGF_EINVAL, "NULL argument");
  if (!valid_dtype_cost(cost_dtype)) return set_err(ctx, HGF_EINVAL, "bad cost dtype");
  if (L < 1) return set_err(ctx, HGF_EINVAL, "L must be >= 1");
  int n = 0;
  st = check_params(ctx, C, H, W, params, &n);
  if (st != HGF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t HW = (size_t)H * W;
  const size_t img_b = ((size_t)C * HW * 4 + 255) / 256 * 256;
  const size_t cost_b = ((size_t)L * HW * dtype_size(cost_dtype) + 255) / 256 * 256;
  const size_t out_b = (HW * 4 + 255) / 256 * 256;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  st = grow(ctx, ctx->ws_io, img_b + cost_b + 2 * out_b, s);
  if (st != HGF_OK) return st;
  char *base = (char *)ctx->ws_io.ptr;
  float *img_d = (float *)base;
  void *cost_d = base + img_b;
  int32_t *labels_d = (int32_t *)(base + img_b + cost_b);
  float *best_d = (float *)(base + img_b + cost_b + out_b);
  // the image goes first (the guidance precompute needs only it); the cost volume, the bulk of
  // the upload, follows on a second stream while the precompute runs, and the aggregation waits
  // for it (queued after the image, so that copy engines serving the streams in order never make
  // the precompute wait for the volume)
  cudaError_t e = cudaSuccess;
  if (!ctx->io_stream) e = cudaStreamCreateWithFlags(&ctx->io_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !ctx->io_fork)
    e = cudaEventCreateWithFlags(&ctx->io_fork, cudaEventDisableTiming);
  if (e == cudaSuccess && !ctx->io_done)
    e = cudaEventCreateWithFlags(&ctx->io_done, cudaEventDisableTiming);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(img_d, img, (size_t)C * HW * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->io_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->io_stream, ctx->io_fork, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cost_d, cost, (size_t)L * HW * dtype_size(cost_dtype),
                        cudaMemcpyHostToDevice, ctx->io_stream);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->io_done, ctx->io_stream);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_filter_host upload");
  if (!same_shape(ctx->host_guidance, C, H, W, params)) {
    if (ctx->host_guidance) {
      cudaStreamSynchronize(s);
      cudaFree(ctx->host_guidance->rec);
      delete ctx->host_guidance;
      ctx->host_guidance = nullptr;
    }
    hgf_guidance *g = nullptr;
    st = alloc_guidance(ctx, C, H, W, n, params, &g);
    if (st != HGF_OK) return st;
    ctx->host_guidance = g;
  }
  st = filter_locked(ctx, ctx->host_guidance, img_d, cost_d, cost_dtype, L, nullptr,
                     labels ? labels_d : nullptr, best ? best_d : nullptr, s, ctx->io_done);
  if (st != HGF_OK) return st;
  if (labels) e = cudaMemcpyAsync(labels, labels_d, HW * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && best) e = cudaMemcpyAsync(best, best_d, HW * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_filter_host download");
  int status = 0;
  e = read_device_status(&status, true);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_filter_host status");
  if (status != 0) return set_err(ctx, HGF_ETIMEOUT, "a bounded wait in a kernel ran out");
  return HGF_OK;
}

namespace {

hgf_status check_cost_params(hgf_ctx *ctx, const hgf_cost_params *p) {
  if (!(p->alpha >= 0.0 && p->alpha <= 1.0) || !(p->tau_color >= 0.0) || !(p->tau_grad >= 0.0))
    return set_err(ctx, HGF_EINVAL, "alpha must be in [0, 1] and thresholds >= 0");
  if (p->direction != 1 && p->direction != -1)
    return set_err(ctx, HGF_EINVAL, "direction must be +1 or -1");
  return HGF_OK;
}

// Stereo aggregation with ctx->mu held and arguments checked.
hgf_status aggregate_stereo_locked(hgf_ctx *ctx, const hgf_guidance *g, const float *other, int L,
                                   const hgf_cost_params *p, void *filtered, int32_t *labels,
                                   float *best, cudaStream_t s) {
  if (!aggregate_fits(g))
    return set_err(ctx, HGF_EUNSUPPORTED, "stereo aggregation needs 2r+1 < %d", kStripThreads);
  const size_t HW = (size_t)g->H * g->W;
  AggregatePlan plan = plan_aggregate(g, L, ctx->tuning, ctx->num_sms);
  hgf_status st = grow(ctx, ctx->ws_coef, aggregate_coef_bytes(g, plan), s);
  if (st == HGF_OK) st = grow(ctx, ctx->ws_keys, HW * sizeof(unsigned long long), s);
  if (st == HGF_OK) st = grow(ctx, ctx->ws_grad, 2 * HW * sizeof(float), s);
  if (st != HGF_OK) return st;
  StereoSource src;
  src.other = other;
  src.grad = (const float *)ctx->ws_grad.ptr;
  src.direction = p->direction;
  src.alpha = (float)p->alpha;
  src.tau_c = (float)p->tau_color;
  src.tau_g = (float)p->tau_grad;
  cudaError_t e = launch_grad_planes(g->img, other, g->C, g->H, g->W, (float *)ctx->ws_grad.ptr,
                                     s, &ctx->prof);
  if (e == cudaSuccess)
    e = launch_aggregate(g, nullptr, kCostStereo, L, (float *)filtered, labels, best,
                         (float *)ctx->ws_coef.ptr, (unsigned long long *)ctx->ws_keys.ptr, plan,
                         s, &ctx->prof, &src);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "stereo aggregation");
  return HGF_OK;
}

// A host-path guidance handle of this shape, reallocated when the shape or parameters change.
hgf_status host_guidance_for(hgf_ctx *ctx, hgf_guidance **slot, int C, int H, int W, int n,
                             const hgf_params *params, cudaStream_t s) {
  if (same_shape(*slot, C, H, W, params)) return HGF_OK;
  if (*slot) {
    cudaStreamSynchronize(s);
    cudaFree((*slot)->rec);
    delete *slot;
    *slot = nullptr;
  }
  return alloc_guidance(ctx, C, H, W, n, params, slot);
}

}  // namespace

hgf_status hgf_aggregate_stereo(hgf_ctx *ctx, const hgf_guidance *g, const float *other, int L,
                                const hgf_cost_params *p, void *filtered, int filtered_dtype,
                                int32_t *labels, float *best, void *stream) {
  NvtxRange nvtx_range("hgf_aggregate_stereo");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!other || !p) return set_err(ctx, HGF_EINVAL, "NULL argument");
  // the cost is made here, not read: check the outputs with a stand-in cost pointer
  st = check_outputs(ctx, g, other, HGF_F32, L, filtered, filtered_dtype, labels, best);
  if (st != HGF_OK) return st;
  st = check_cost_params(ctx, p);
  if (st != HGF_OK) return st;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  return aggregate_stereo_locked(ctx, g, other, L, p, filtered, labels, best,
                                 (cudaStream_t)stream);
}

hgf_status hgf_stereo_host(hgf_ctx *ctx, const float *left, const float *right, int C, int H,
                           int W, int L, const hgf_params *params, const hgf_cost_params *cost,
                           int refine, int threshold, int32_t *disparity, void *stream) {
  NvtxRange nvtx_range("hgf_stereo_host");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!left || !right || !cost || !disparity) return set_err(ctx, HGF_EINVAL, "NULL argument");
  if (L < 1) return set_err(ctx, HGF_EINVAL, "L must be >= 1");
  if (refine != 0 && refine != 1) return set_err(ctx, HGF_EINVAL, "refine must be 0 or 1");
  if (threshold < 0) return set_err(ctx, HGF_EINVAL, "threshold must be >= 0");
  int n = 0;
  st = check_params(ctx, C, H, W, params, &n);
  if (st != HGF_OK) return st;
  hgf_cost_params cp = *cost;
  cp.direction = 1;
  st = check_cost_params(ctx, &cp);
  if (st != HGF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t HW = (size_t)H * W;
  const size_t img_b = ((size_t)C * HW * 4 + 255) / 256 * 256;
  const size_t out_b = (HW * 4 + 255) / 256 * 256;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  st = grow(ctx, ctx->ws_io, 2 * img_b + 3 * out_b + out_b, s);
  if (st != HGF_OK) return st;
  char *base = (char *)ctx->ws_io.ptr;
  float *left_d = (float *)base;
  float *right_d = (float *)(base + img_b);
  int32_t *lab_l = (int32_t *)(base + 2 * img_b);
  int32_t *lab_r = (int32_t *)(base + 2 * img_b + out_b);
  int32_t *refined = (int32_t *)(base + 2 * img_b + 2 * out_b);
  uint8_t *keep = (uint8_t *)(base + 2 * img_b + 3 * out_b);
  // the left view first; the right view follows on the library's second stream while the left
  // guidance is prepared
  cudaError_t e = cudaSuccess;
  if (!ctx->io_stream) e = cudaStreamCreateWithFlags(&ctx->io_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !ctx->io_fork)
    e = cudaEventCreateWithFlags(&ctx->io_fork, cudaEventDisableTiming);
  if (e == cudaSuccess && !ctx->io_done)
    e = cudaEventCreateWithFlags(&ctx->io_done, cudaEventDisableTiming);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(left_d, left, (size_t)C * HW * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->io_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->io_stream, ctx->io_fork, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(right_d, right, (size_t)C * HW * 4, cudaMemcpyHostToDevice,
                        ctx->io_stream);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->io_done, ctx->io_stream);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_stereo_host upload");
  st = host_guidance_for(ctx, &ctx->host_guidance, C, H, W, n, params, s);
  if (st == HGF_OK && refine)
    st = host_guidance_for(ctx, &ctx->host_guidance_right, C, H, W, n, params, s);
  if (st != HGF_OK) return st;
  st = prepare_locked(ctx, ctx->host_guidance, left_d, s);
  if (st != HGF_OK) return st;
  e = cudaStreamWaitEvent(s, ctx->io_done, 0);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_stereo_host upload wait");
  st = aggregate_stereo_locked(ctx, ctx->host_guidance, right_d, L, &cp, nullptr, lab_l, nullptr,
                               s);
  if (st != HGF_OK) return st;
  const int32_t *result = lab_l;
  if (refine) {
    st = prepare_locked(ctx, ctx->host_guidance_right, right_d, s);
    if (st != HGF_OK) return st;
    hgf_cost_params cr = cp;
    cr.direction = -1;
    st = aggregate_stereo_locked(ctx, ctx->host_guidance_right, left_d, L, &cr, nullptr, lab_r,
                                 nullptr, s);
    if (st != HGF_OK) return st;
    e = launch_refine_lr(lab_l, lab_r, H, W, threshold, refined, keep, s, &ctx->prof);
    if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_stereo_host refine");
    result = refined;
  }
  e = cudaMemcpyAsync(disparity, result, HW * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_stereo_host download");
  int status = 0;
  e = read_device_status(&status, true);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_stereo_host status");
  if (status != 0) return set_err(ctx, HGF_ETIMEOUT, "a bounded wait in a kernel ran out");
  return HGF_OK;
}

hgf_status hgf_refine_lr(hgf_ctx *ctx, const int32_t *disp_left, const int32_t *disp_right, int H,
                         int W, int threshold, int32_t *out, uint8_t *keep, void *stream) {
  NvtxRange nvtx_range("hgf_refine_lr");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!disp_left || !disp_right || !out || !keep) return set_err(ctx, HGF_EINVAL, "NULL argument");
  if (H < 1 || W < 1 || (long long)H * W > (1ll << 31))
    return set_err(ctx, HGF_EINVAL, "bad size %d x %d", H, W);
  if (threshold < 0) return set_err(ctx, HGF_EINVAL, "threshold must be >= 0");
  if (out == disp_left || out == disp_right) return set_err(ctx, HGF_EINVAL, "out aliases an input");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = launch_refine_lr(disp_left, disp_right, H, W, threshold, out, keep,
                                   (cudaStream_t)stream, &ctx->prof);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_refine_lr");
  return HGF_OK;
}

hgf_status hgf_cost_volume(hgf_ctx *ctx, const float *ref, const float *other, int C, int H, int W,
                           int L, const hgf_cost_params *p, int dtype, void *out, void *stream) {
  NvtxRange nvtx_range("hgf_cost_volume");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!ref || !other || !p || !out) return set_err(ctx, HGF_EINVAL, "NULL argument");
  if ((C != 1 && C != 3) || H < 1 || W < 1 || L < 1)
    return set_err(ctx, HGF_EINVAL, "bad sizes C=%d H=%d W=%d L=%d", C, H, W, L);
  if ((long long)L * H * W > (1ll << 40)) return set_err(ctx, HGF_EINVAL, "volume too large");
  if (!(p->alpha >= 0.0 && p->alpha <= 1.0) || !(p->tau_color >= 0.0) || !(p->tau_grad >= 0.0))
    return set_err(ctx, HGF_EINVAL, "alpha must be in [0, 1] and thresholds >= 0");
  if (p->direction != 1 && p->direction != -1)
    return set_err(ctx, HGF_EINVAL, "direction must be +1 or -1");
  if (dtype != HGF_F32 && dtype != HGF_BF16 && dtype != HGF_F16)
    return set_err(ctx, HGF_EINVAL, "dtype must be HGF_F32, HGF_BF16 or HGF_F16");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = launch_cost_volume(ref, other, C, H, W, L, *p, dtype, out,
                                     (cudaStream_t)stream, &ctx->prof);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_cost_volume");
  return HGF_OK;
}

hgf_status hgf_batched_inverse(hgf_ctx *ctx, const double *S, int count, int n, double lambda,
                               int method, int precision, double *out, void *stream) {
  NvtxRange nvtx_range("hgf_batched_inverse");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!S || !out) return set_err(ctx, HGF_EINVAL, "NULL argument");
  if (count < 1) return set_err(ctx, HGF_EINVAL, "count must be >= 1");
  if (!(lambda > 0.0)) return set_err(ctx, HGF_EINVAL, "lambda must be > 0");
  if (method != HGF_INV_PROP1 && method != HGF_INV_CHOLESKY)
    return set_err(ctx, HGF_EINVAL, "unknown method %d", method);
  if (precision != HGF_F64 && precision != HGF_F32 && precision != HGF_DF64)
    return set_err(ctx, HGF_EINVAL, "precision must be HGF_F64, HGF_DF64 or HGF_F32");
  if (!aggregate_supported(n)) return set_err(ctx, HGF_EUNSUPPORTED, "n = %d is not built", n);
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = launch_batched_inverse(S, count, n, lambda, method, precision, out,
                                         (cudaStream_t)stream, &ctx->prof);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_batched_inverse");
  return HGF_OK;
}

hgf_status hgf_watchdog_probe(hgf_ctx *ctx, int limit_us, void *stream) {
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (limit_us < 1 || limit_us > 10000000)
    return set_err(ctx, HGF_EINVAL, "limit_us must be in 1 .. 10^7");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = launch_watchdog_probe((unsigned long long)limit_us * 1000ull,
                                        (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_watchdog_probe");
  return HGF_OK;
}

hgf_status hgf_device_status(hgf_ctx *ctx, int *status, int clear) {
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!status) return set_err(ctx, HGF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = read_device_status(status, clear != 0);
  if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_device_status");
  return HGF_OK;
}


hgf_status hgf_guidance_update(hgf_ctx *ctx, hgf_guidance *g, const float *img, void *stream) {
  NvtxRange nvtx_range("hgf_guidance_update");
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!g || g->ctx != ctx) return set_err(ctx, HGF_EINVAL, "bad guidance handle");
  if (!img) return set_err(ctx, HGF_EINVAL, "img is NULL");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  return prepare_locked(ctx, g, img, (cudaStream_t)stream);
}

hgf_status hgf_profile_enable(hgf_ctx *ctx, int enable) {
  if (!ctx) return HGF_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  ctx->prof.enabled = enable != 0;
  return HGF_OK;
}

hgf_status hgf_last_plan(hgf_ctx *ctx, int *out, int n) {
  if (!ctx || !out || n < 1) return HGF_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  for (int i = 0; i < n; ++i) out[i] = i < 8 ? ctx->prof.plan[i] : 0;
  return HGF_OK;
}

hgf_status hgf_launch_count(hgf_ctx *ctx, unsigned long long *out) {
  if (!ctx || !out) return HGF_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  *out = ctx->prof.launches;
  return HGF_OK;
}

hgf_status hgf_profile_report(hgf_ctx *ctx, char *buf, size_t cap) {
  hgf_status st = enter(ctx);
  if (st != HGF_OK) return st;
  if (!buf || cap == 0) return set_err(ctx, HGF_EINVAL, "NULL buffer");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  struct Acc {
    std::string name;
    int launches;
    double ms;
  };
  std::vector<Acc> acc;
  for (auto &rec : ctx->prof.recs) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(rec.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, rec.a, rec.b);
    if (e != cudaSuccess) return cuda_fail_locked(ctx, e, "hgf_profile_report");
    auto it = std::find_if(acc.begin(), acc.end(), [&](const Acc &a) { return a.name == rec.name; });
    if (it == acc.end()) {
      acc.push_back({rec.name, 1, (double)ms});
    } else {
      it->launches += 1;
      it->ms += ms;
    }
    ctx->prof.pool.push_back(rec.a);
    ctx->prof.pool.push_back(rec.b);
  }
  ctx->prof.recs.clear();
  std::string js = "{";
  for (size_t i = 0; i < acc.size(); ++i) {
    char item[160];
    snprintf(item, sizeof item, "%s\"%s\": {\"launches\": %d, \"ms\": %.6f}", i ? ", " : "",
             acc[i].name.c_str(), acc[i].launches, acc[i].ms);
    js += item;
  }
  js += "}";
  if (js.size() + 1 > cap) return set_err(ctx, HGF_EINVAL, "buffer too small (%zu)", js.size() + 1);
  memcpy(buf, js.c_str(), js.size() + 1);
  return HGF_OK;
}

}  // extern "C"
