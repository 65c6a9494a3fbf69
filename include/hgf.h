/*
 * hgf.h - C ABI of libhgf: multichannel guided aggregation of a cost volume with the
 * Hardware-efficient Guided Filter (HGF, arXiv 1803.00005) followed by winner-takes-all (WTA)
 * label selection, on one NVIDIA GB300 (sm_103a).
 *
 * Problem statement (Sec. 1): a multi-label system records the cost c of label l at pixel (x, y)
 * in a cost volume V(x, y, l); every label slice is smoothed by a guided filter and each pixel
 * then takes the label of lowest filtered cost (WTA). The guidance is a polynomial synthesis of
 * an input image (Sec. 4.2); the per-pixel n x n regularised covariance is inverted once per
 * guidance with the Sherman-Morrison recursion of Prop. 1 (Sec. 3) and kept resident on the GPU.
 *
 * Conventions for every entry point:
 *   - Images and volumes are planar, row-major, x fastest: an image is C x H x W floats, a cost
 *     volume is L x H x W elements, label-major (one contiguous H x W slice per label).
 *   - Pointers documented as "device" must point to memory on the context's device; the caller
 *     owns them and must keep them valid until the work queued on `stream` has completed.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Calls only
 *     enqueue work; nothing is synchronised unless stated.
 *   - Every call returns an hgf_status; nothing aborts, traps or throws across this ABI.
 *     HGF_EINVAL: bad argument (nothing enqueued). HGF_ECUDA: a CUDA call failed; the context
 *     records it (hgf_last_error) and refuses further work with HGF_ECUDA (sticky).
 *   - Windows are (2r+1) x (2r+1) boxes clipped at the image border (no padding); means divide
 *     by the number of in-image pixels N(x, y) (the paper's A(X) = B(X) / B(G0), Eq. HGF_z2).
 */
#ifndef HGF_H_
#define HGF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HGF_OK = 0,
  HGF_EINVAL = 1,        /* invalid argument */
  HGF_ENOMEM = 2,        /* device allocation failed, or a request exceeds the memory budget */
  HGF_ECUDA = 3,         /* CUDA runtime error (sticky per context) */
  HGF_ETIMEOUT = 4,      /* a bounded wait ran out */
  HGF_EBUSY = 5,         /* queue full */
  HGF_EAGAIN = 6,        /* not finished yet */
  HGF_EUNSUPPORTED = 7   /* valid but not supported (e.g. n > 19) */
} hgf_status;

/* HGF_DF64 is an arithmetic precision only (hgf_params.inv_precision, hgf_batched_inverse):
 * double-float, the unevaluated sum of two float32 numbers (about 48 significant bits), built from
 * float32 operations that GB300 runs at 64 times its float64 rate. */
typedef enum { HGF_F32 = 0, HGF_BF16 = 1, HGF_F16 = 2, HGF_F64 = 3, HGF_DF64 = 4 } hgf_dtype;

/* Guidance basis (Sec. 4.2). MONOMIAL: every monomial of degree 1..d of the C input channels,
 * degree-major then lexicographic (R, G, B, RR, RG, RB, GG, GB, BB, RRR, ...), n = C(C+d,d) - 1.
 * POWERS: the paper's G_{(i-1)d+j} = I_i^j, channel-major, n = C d. */
typedef enum { HGF_BASIS_MONOMIAL = 0, HGF_BASIS_POWERS = 1 } hgf_basis;

/* How the per-pixel inverse is read off Prop. 1's alpha (Sec. 3). Both run the recursion in the
 * precision `inv_precision`. W3: lambda^-1 E + S alpha, Eq. HGF_w3 as printed. ALPHA: -lambda alpha,
 * the same matrix (Prop. 1 gives alpha = -lambda^-1 (lambda E + S)^-1); it skips the n^3/2
 * multiply-adds of S alpha and the cancellation of lambda^-1 against it. */
typedef enum { HGF_COMBINE_ALPHA = 0, HGF_COMBINE_W3 = 1 } hgf_combine;

/* Which filter (the two are different filters, not rounding variants of one another).
 * CENTRED (default, Sec. 5.1): mu = A(G), Sigma = A(G G^T) - mu mu^T, a = (Sigma + eps E)^-1 cov,
 *   b = A(p) - a^T mu, q = sum_i A(a_i) G_i + A(b); eps is in units of window means.
 * PAPER (Sec. 3 and 4, Eqs. HGF_Iij, HGF_w3, HGF_z2): G_0 = 1 joins the guidance, the
 *   (n+1) x (n+1) Gram matrix of window sums B(G_i G_j) (i, j = 0..n) and b_k = B(G_k p) are
 *   uncentred, w = (lambda E + Gram)^-1 b penalises all n+1 weights with lambda = eps in units of
 *   window sums, and Z = sum_{i>=1} A(w_i) G_i + A(w_0). Served by the fused path only
 *   (hgf_aggregate_plain, hgf_guidance_export and windows with 2r+1 >= 128 give HGF_EUNSUPPORTED). */
typedef enum { HGF_FORM_CENTRED = 0, HGF_FORM_PAPER = 1 } hgf_form;

typedef struct {
  int degree;         /* polynomial degree d >= 1 (Sec. 4.2); n <= 19 */
  int basis;          /* hgf_basis */
  int r;              /* window radius r >= 0: (2r+1)^2 box (Sec. 6 uses r = 7) */
  double eps;         /* regulariser eps > 0 (lambda); units depend on `form` */
  int inv_precision;  /* precision of the covariance assembly + recursion: HGF_F64 (default,
                       * native float64), HGF_DF64 (double-float) or HGF_F32 */
  int combine;        /* hgf_combine */
  int form;           /* hgf_form (0 = CENTRED) */
  int compensated;    /* 1: Kahan-compensated vertical running sums in the guidance-moment and
                       * aggregation kernels (two labels per pass; slower, smaller rounding
                       * error); 0: plain float32 running sums (default) */
} hgf_params;

typedef struct hgf_ctx hgf_ctx;
typedef struct hgf_guidance hgf_guidance;

/* Create a context on CUDA device `device` (makes it current for the calling thread). */
hgf_status hgf_create(int device, hgf_ctx **out);
/* Destroy a context: synchronises its device, frees its workspace. Guidance handles created from
 * it must be released first. NULL is accepted. */
hgf_status hgf_destroy(hgf_ctx *ctx);
/* Last error message of this context (empty string if none). Valid until the next call. */
const char *hgf_last_error(const hgf_ctx *ctx);
/* Number of guidance channels n for (C, degree, basis); 0 if unsupported. */
int hgf_num_channels(int C, int degree, int basis);

/* Polynomial guidance synthesis (Sec. 4.2, Eqs. HGF_input_output_polynomial_model[_color]).
 * img: device, C x H x W float32 (C = 1 or 3). G_out: device, n x H x W float32, channel order
 * as in hgf_basis. *n_out receives n. */
hgf_status hgf_make_guidance(hgf_ctx *ctx, const float *img, int C, int H, int W, int degree,
                             int basis, float *G_out, int *n_out, void *stream);

/* Guidance precompute (Sec. 5.3: guidance-only box filtering is done once per guidance):
 * polynomial guidance G, means mu = A(G), covariance Sigma = A(G G^T) - mu mu^T plus eps E
 * (Sec. 5.1) and its inverse by Prop. 1 (Sec. 3), kept resident in a handle the library owns.
 * With params->form = HGF_FORM_PAPER, the (n+1) x (n+1) inverse of lambda E + Gram (window sums,
 * G_0 = 1) instead.
 * img: device, C x H x W float32, may be freed once the call's work has completed (the handle
 * keeps a copy). The handle's memory is allocated here (HGF_ENOMEM on failure) and freed by
 * hgf_guidance_release. Bounds: C in {1,3}, 1 <= n <= 19, H, W >= 1, r >= 0, eps > 0. */
hgf_status hgf_prepare(hgf_ctx *ctx, const float *img, int C, int H, int W,
                       const hgf_params *params, void *stream, hgf_guidance **out);
/* Recompute an existing guidance handle from a new image of the same shape and parameters
 * (same precompute as hgf_prepare, Sec. 5.3), reusing its device memory: no allocation once the
 * context's prepare workspace has grown to this shape. img: device, C x H x W float32. */
hgf_status hgf_guidance_update(hgf_ctx *ctx, hgf_guidance *g, const float *img, void *stream);
/* Release a guidance handle (waits for the device work that uses it). NULL is accepted. */
hgf_status hgf_guidance_release(hgf_guidance *g);
/* Shape of a guidance: any pointer may be NULL. */
hgf_status hgf_guidance_info(const hgf_guidance *g, int *C, int *H, int *W, int *n, int *r,
                             double *eps);
/* Copy out the resident inverse for inspection: minv_out (device, n(n+1)/2 x H x W float32,
 * packed upper triangle row by row: (0,0),(0,1)..(0,n-1),(1,1),..), mu_out (device, n x H x W:
 * the window means A(G_i)). Either may be NULL. */
hgf_status hgf_guidance_export(hgf_ctx *ctx, const hgf_guidance *g, float *minv_out,
                               float *mu_out, void *stream);

/* Fused aggregation + WTA (Sec. 1 pipeline; Eqs. GF_w / HGF_z1): for every label slice p of the
 * cost volume, pbar = A(p), cov_i = A(G_i p) - mu_i pbar, a = (Sigma + eps E)^-1 cov,
 * b = pbar - a.mu, q = sum_i A(a_i) G_i + A(b); then labels = argmin_l q_l (lowest l on ties,
 * NaN counted as +inf) and best = min_l q_l. Either one kernel does all of it, WTA included, in a
 * single pass over the slices (n <= 9, r <= 24), or two kernels per chunk of labels with a
 * coefficient workspace in between (see hgf_tuning.kernel for which the plan takes). For a guidance prepared with HGF_FORM_PAPER the
 * coefficients are those of the paper's form instead: w = (lambda E + Gram)^-1 B([1, G] p) and
 * q = sum_i A(w_i) G_i + A(w_0) (see hgf_form).
 * cost: device, L x H x W of cost_dtype (HGF_F32, HGF_BF16 or HGF_F16), H, W of the guidance.
 * filtered: device L x H x W of filtered_dtype (HGF_F32) or NULL; labels: device int32 H x W or
 * NULL; best: device float32 H x W or NULL. At least one output must be non-NULL.
 * Uses the context's workspace (grown on demand; HGF_ENOMEM if that fails). */
hgf_status hgf_aggregate(hgf_ctx *ctx, const hgf_guidance *g, const void *cost, int cost_dtype,
                         int L, void *filtered, int filtered_dtype, int32_t *labels, float *best,
                         void *stream);

/* One frame in one call: hgf_guidance_update(g, img) (Secs. 5.1 and 3: guidance, moments,
 * inverse) followed by hgf_aggregate(g, cost) (aggregation and WTA) on the same stream, with the
 * results of those two calls; g is updated in place and stays usable after it. img: device,
 * C x H x W float32 of the guidance's shape; the other arguments as for hgf_aggregate. Errors as
 * for the two calls. */
hgf_status hgf_filter(hgf_ctx *ctx, hgf_guidance *g, const float *img, const void *cost,
                      int cost_dtype, int L, void *filtered, int filtered_dtype, int32_t *labels,
                      float *best, void *stream);

/* hgf_aggregate for callers that cannot allocate device memory while they run: fixed-latency loops
 * (cudaMalloc/cudaFree can synchronise the device and block), or plugins in a program that hands
 * out all device memory from its own allocator at start-up, where a late cudaMalloc fails or
 * fragments that pool. The same kernels and results, but the scratch - per-pixel WTA keys and
 * either per-chunk coefficient planes (two-kernel path, the default) or the single-pass kernel's
 * ring slots (hgf_tuning.kernel = 1) - comes from one fixed 64 MiB file-scope device array
 * instead of the context's growable workspace. No cudaMalloc/cudaFree or allocating library call
 * is made.
 * The paper has no counterpart; it is a property of this library only.
 * The array is held by every GPU that loads the library until the process exits. hgf_create
 * commits it on the context's device and looks up its address (cudaGetSymbolAddress) with that
 * device current; if that failed (no memory left), the first call here tries again, returns
 * HGF_ENOMEM while it fails (the context stays usable), and should then come before any stream
 * capture. All calls share the array and it keeps the last call's contents (the keys are reset by
 * every call, every coefficient plane is written before it is read); calls that overlap on the
 * GPU race and must be serialised. Returns HGF_EUNSUPPORTED when the keys (8 bytes a pixel) plus
 * one label's coefficient planes (two-kernel path: about 1.4 Mpixel at n = 9) or plus one ring
 * slot (single pass: 140 KB at n = 9, r = 9; about 8 Mpixel) exceed 64 MiB, or when the window is
 * too wide for the fused kernels.
 * Same arguments as hgf_aggregate. */
hgf_status hgf_aggregate_static(hgf_ctx *ctx, const hgf_guidance *g, const void *cost,
                                int cost_dtype, int L, void *filtered, int filtered_dtype,
                                int32_t *labels, float *best, void *stream);

/* The same computation as hgf_aggregate by the plain form: one kernel per step (products, row
 * sums, column sums, coefficients, row sums, column sums, output, WTA) with every intermediate
 * plane in device memory. Comparison baseline for the fused path. Same arguments. */
hgf_status hgf_aggregate_plain(hgf_ctx *ctx, const hgf_guidance *g, const void *cost,
                               int cost_dtype, int L, void *filtered, int filtered_dtype,
                               int32_t *labels, float *best, void *stream);

/* Standalone WTA (Sec. 1) over an already-filtered volume: filtered device L x H x W (HGF_F32),
 * labels device int32 H x W (or NULL), best device float32 H x W (or NULL). */
hgf_status hgf_wta(hgf_ctx *ctx, const void *filtered, int dtype, int L, int H, int W,
                   int32_t *labels, float *best, void *stream);

/* hgf_aggregate with the WTA margin (Sec. 1 WTA, with a confidence output the paper does not
 * have): margin = (second-smallest filtered cost) - (smallest), per pixel, in float32; +inf when
 * L = 1; 0 when two labels tie for the minimum; NaN when the two smallest are both +inf (NaN
 * filtered costs count as +inf, as for the labels). labels, best: as for hgf_aggregate (either may
 * be NULL); margin: device float32 H x W, required. The fused path keeps a second 64-bit key per
 * pixel (the keys workspace doubles) and returns the old key from its atomic minimum; windows too
 * wide for the fused kernels take the plain path and hgf_wta_margin. Same errors as hgf_aggregate,
 * plus HGF_EINVAL for a NULL margin. */
hgf_status hgf_aggregate_margin(hgf_ctx *ctx, const hgf_guidance *g, const void *cost,
                                int cost_dtype, int L, int32_t *labels, float *best,
                                float *margin, void *stream);

/* hgf_wta with the margin (as for hgf_aggregate_margin) over an already-filtered volume: filtered
 * device L x H x W (HGF_F32); labels, best may be NULL; margin device float32 H x W, required. */
hgf_status hgf_wta_margin(hgf_ctx *ctx, const void *filtered, int dtype, int L, int H, int W,
                          int32_t *labels, float *best, float *margin, void *stream);

/* End to end from host memory: copies img (host, C x H x W float32) and cost (host, L x H x W of
 * cost_dtype) to the device, prepares the guidance, aggregates with WTA and copies labels (host
 * int32 H x W, may be NULL) and best (host float32 H x W, may be NULL) back; returns after the
 * results are in host memory. Host buffers may be pageable or pinned (pinned is faster). The cost
 * volume is uploaded on a second, library-owned stream while the guidance precompute runs on
 * `stream`; the aggregation waits for the upload. */
hgf_status hgf_filter_host(hgf_ctx *ctx, const float *img, int C, int H, int W,
                           const hgf_params *params, const void *cost, int cost_dtype, int L,
                           int32_t *labels, float *best, void *stream);

/* Tuning of the fused kernels (0 = automatic): labels per pass of the coefficient kernel (2, 4, 8),
 * row-band height, labels per chunk of the coefficient workspace, how the output kernel gets
 * the row leaving its vertical window (1 = shared-memory ring, 2 = reload from device memory),
 * and which kernels run: kernel = 1 the single-pass kernel (slice moments, coefficients, their
 * box filter, output and WTA of two labels at a time in one pass over the slices, with a small
 * L2-resident ring of coefficient window sums instead of a coefficient workspace; n <= 9 and
 * r <= 24), 2 the two-kernel path (coefficients to a workspace, then output + WTA: the only one
 * for n = 19), 0 automatic: the single pass where it applies and either n <= 3 or its output
 * strips (128 - 4r columns) need no more strips than the two-kernel path's (128 - 2r) and
 * H * W * L is at least 8e6, the two-kernel path otherwise. labels_per_pass, chunk_labels and apply_mode apply to
 * the two-kernel path only. Returns HGF_EINVAL for values the kernels cannot take. */
typedef struct {
  int labels_per_pass;
  int band_rows;
  int chunk_labels;
  int apply_mode;
  int kernel;
} hgf_tuning;
hgf_status hgf_set_tuning(hgf_ctx *ctx, const hgf_tuning *t);
/* Autotuner (no counterpart in the paper): times hgf_aggregate on (g, cost) under every candidate
 * tuning - first the kernel path (single pass where it applies, two kernels with labels per pass
 * 2, 4 or 8 where shared memory allows, labels per chunk all / 64 / 16 and the output kernel's
 * outgoing-row source), with the automatic row bands; then, for the fastest of those, row-band
 * heights of a half, a quarter and an eighth of the image - and makes the fastest ctx's tuning.
 * Candidates of the two-kernel family with the same bands give bit-identical results; the
 * path and the band height change only the order of the sums' rounding (every candidate is
 * within the filter's tolerance). Keep one tuning per shape class (bench.py and hgf.py's
 * autotune_cached key it by GPU, n, r, cost dtype and size class), so that alone, batched and
 * served runs of a shape use one plan. Each candidate runs once untimed, then `reps` times
 * between CUDA events on `stream`; *best (may be NULL) receives the pick, *ncand (may be NULL)
 * the number of candidates timed. labels: device int32 H x W, scratch output. Blocks until done.
 * HGF_EINVAL on bad arguments or reps < 1; errors of hgf_aggregate otherwise. */
hgf_status hgf_autotune(hgf_ctx *ctx, const hgf_guidance *g, const void *cost, int cost_dtype,
                        int L, int32_t *labels, int reps, hgf_tuning *best, int *ncand,
                        void *stream);

/* ---------------------------------------------------------------------------------------------
 * Batches (no counterpart in the paper): many images of different sizes, label counts and
 * guidance degrees processed together. hgf_batch_create allocates, once, every job's guidance
 * handle and the workspaces of `streams` internal CUDA streams (jobs are spread over them,
 * largest first, to balance the work). hgf_batch_run enqueues every job (guidance precompute +
 * fused aggregation + WTA) on those streams, forked from and joined back into `stream` by events:
 * it allocates nothing, so it can be captured into a CUDA graph; hgf_batch_launch_graph captures
 * it once into a graph (instantiated on the first call) and launches that graph. When ctx is
 * tuned to the single-pass kernel (hgf_tuning.kernel = 1) at hgf_batch_create, the jobs that
 * kernel takes here (RGB guidance of degree 1 or 2, not compensated, r <= 24) are aggregated by
 * one persistent launch per 40 jobs on `stream` after every precompute, the CTAs taking the
 * jobs' (labels, strip, band) work items from one device counter; the other jobs take their
 * streams. Job results are the same as hgf_prepare + hgf_aggregate on each job alone under the
 * same tuning.
 * ------------------------------------------------------------------------------------------- */
typedef struct hgf_batch hgf_batch;
typedef struct {
  const float *img;   /* device C x H x W float32 */
  int C, H, W;
  hgf_params params;
  const void *cost;   /* device L x H x W of cost_dtype */
  int cost_dtype;
  int L;
  int32_t *labels;    /* device int32 H x W or NULL */
  float *best;        /* device float32 H x W or NULL */
  float *filtered;    /* device float32 L x H x W or NULL (one output at least) */
} hgf_job;
hgf_status hgf_batch_create(hgf_ctx *ctx, const hgf_job *jobs, int njobs, int streams,
                            hgf_batch **out);
hgf_status hgf_batch_run(hgf_batch *b, void *stream);
hgf_status hgf_batch_launch_graph(hgf_batch *b, void *stream);
hgf_status hgf_batch_destroy(hgf_batch *b);

/* ---------------------------------------------------------------------------------------------
 * Serving (no counterpart in the paper): a request loop in a background thread that admits
 * multi-label jobs of different sizes, label counts and guidance degrees against a device-memory
 * budget, keeps each guidance's resident inverse (hgf_prepare) in an LRU cache shared by
 * requests with equal guidance_key and parameters, and runs admitted requests concurrently on
 * `slots` CUDA streams, each with its own workspace (continuous batching: a request is admitted as
 * soon as a slot and memory are free). Results are bit-identical to hgf_aggregate on the same
 * inputs, whatever else is in flight. Device memory for cached guidances is allocated stream-
 * ordered (cudaMallocAsync) so that admission never synchronises the device.
 * ------------------------------------------------------------------------------------------- */
typedef struct hgf_server hgf_server;

typedef struct {
  uint64_t guidance_key;  /* requests with equal keys, shapes and params share one guidance */
  const float *img;       /* device, C x H x W float32; read only when the guidance is prepared */
  int C, H, W;
  hgf_params params;
  const void *cost;       /* device, L x H x W of cost_dtype */
  int cost_dtype;
  int L;
  int32_t *labels;        /* device int32 H x W (required) */
  float *best;            /* device float32 H x W or NULL */
} hgf_request;

typedef struct {
  uint64_t submitted, completed, failed, rejected_busy, rejected_nomem;
  uint64_t cache_hits, cache_misses, evictions;
  double p50_ms, p99_ms, mean_ms, max_ms;  /* submit -> results written, completed requests */
  double mpixel_labels_per_s;              /* completed H*W*L / (last completion - first submit) */
  size_t budget_bytes, resident_bytes, peak_bytes;
  int slots, max_concurrent;               /* slots, most requests seen running at once */
  /* where a completed request's time went: waiting in the queue (submit -> admission, mean and
   * p99), and device time on its slot's stream, split by guidance size (index 0: n <= 3, 1:
   * n <= 9, 2: n = 19): totals of the precompute (cache misses only) and of the aggregation +
   * WTA in ms, and the completed requests of each class */
  double queue_mean_ms, queue_p99_ms;
  double prepare_ms_total[3], aggregate_ms_total[3];
  uint64_t completed_by_class[3];
} hgf_serve_stats_t;

/* Create a server on `device` with a device-memory budget (slot workspaces + cached guidances),
 * `slots` concurrent streams (1..16) and a queue of at most `max_queue` waiting requests. Each
 * slot's workspace is allocated here for images up to max_pixels pixels and n <= max_n.
 * Admission is in arrival order with one exception, by guidance degree: with two or more slots,
 * requests with n = 19 (the longest, their float64 precompute alone taking several times that of
 * n = 9) hold at most slots - 1 slots at once, and while the request at the head of the queue
 * waits for that reason, a later request with n <= 9 (among the next 16) may start first. */
hgf_status hgf_serve_create(int device, size_t budget_bytes, int slots, int max_queue,
                            int max_pixels, int max_n, hgf_server **out);
/* Queue a request (the structure is copied; the buffers it points to must stay valid until the
 * request completes). HGF_EBUSY: queue full. HGF_ENOMEM: the request alone exceeds the budget.
 * HGF_EINVAL / HGF_EUNSUPPORTED: invalid request. *id receives the request id. */
hgf_status hgf_serve_submit(hgf_server *s, const hgf_request *req, uint64_t *id);
/* HGF_OK: results written; HGF_EAGAIN: queued or running; HGF_ECUDA: the request failed;
 * HGF_EINVAL: unknown id. */
hgf_status hgf_serve_poll(hgf_server *s, uint64_t id);
/* Waits at most timeout_ms (< 0: no limit) for the request: HGF_OK, HGF_ETIMEOUT or as poll. */
hgf_status hgf_serve_wait(hgf_server *s, uint64_t id, int timeout_ms);
/* Statistics since creation (or the last reset when reset != 0, after reading them). */
hgf_status hgf_serve_stats(hgf_server *s, hgf_serve_stats_t *out, int reset);
/* Test hook: make the next `count` guidance allocations fail as if the device were out of memory
 * (the affected requests complete with HGF_ENOMEM). */
hgf_status hgf_serve_inject_alloc_failures(hgf_server *s, int count);
/* Drain the queue, wait for running requests, free everything. NULL is accepted. */
hgf_status hgf_serve_destroy(hgf_server *s);

/* ---------------------------------------------------------------------------------------------
 * Cost volume of a stereo pair: the cost computation that precedes aggregation in the
 * multi-label pipeline (Sec. 1; the cost-volume filtering framework of the stereo experiment,
 * Sec. 6). The paper prints no formula; the library's reading is a truncated colour + gradient
 * difference, for l = 0..L-1:
 *   V(x, y, l) = alpha min(mean_c |I_c(x,y) - J_c(x',y)|, tau_color)
 *              + (1 - alpha) min(|dI(x,y) - dJ(x',y)|, tau_grad),
 *   x' = clamp(x - direction * l, 0, W - 1),
 * I = ref, J = other, dI = 0.5 (g(x+1) - g(x-1)) of the channel mean g with neighbours clamped
 * at the border. direction = +1 when ref is the left view, -1 when it is the right view.
 * ref, other: device float32, C x H x W (C = 1 or 3). out: device, L x H x W of `dtype`
 * (HGF_F32, HGF_BF16 or HGF_F16; computed in float32, rounded to nearest even). Enqueued on
 * `stream`; HGF_EINVAL on NULL pointers, bad sizes, alpha outside [0, 1], negative thresholds,
 * direction not +-1 or a bad dtype. */
typedef struct {
  double alpha;      /* colour weight (the gradient term gets 1 - alpha); 0.9 in the inputs here */
  double tau_color;  /* truncation of the colour term (0.028) */
  double tau_grad;   /* truncation of the gradient term (0.008) */
  int direction;     /* +1: ref is the left view; -1: ref is the right view */
} hgf_cost_params;
hgf_status hgf_cost_volume(hgf_ctx *ctx, const float *ref, const float *other, int C, int H, int W,
                           int L, const hgf_cost_params *p, int dtype, void *out, void *stream);

/* Aggregation + WTA of the stereo cost volume of (guidance image, other), without storing the
 * volume: the guidance handle's image is the reference view I, `other` (device float32,
 * C x H x W, same shape as the guidance image) is J, and the coefficient kernel computes
 * V(x, y, l) of hgf_cost_volume for labels l = 0..L-1 as it reads them (bit-identical to
 * hgf_cost_volume with HGF_F32 storage followed by hgf_aggregate). Outputs as hgf_aggregate.
 * Needs the fused path (2r+1 < 128; HGF_EUNSUPPORTED otherwise); errors as hgf_cost_volume and
 * hgf_aggregate. */
hgf_status hgf_aggregate_stereo(hgf_ctx *ctx, const hgf_guidance *g, const float *other, int L,
                                const hgf_cost_params *p, void *filtered, int filtered_dtype,
                                int32_t *labels, float *best, void *stream);

/* The stereo pipeline of the cost-volume filtering framework (Sec. 6: cost computation,
 * aggregation, WTA, post processing) in one call from host memory: uploads the left and right
 * views (host float32 C x H x W; the right one on a library stream while the left guidance is
 * prepared), prepares the left view's guidance, aggregates the cost of hgf_cost_volume for
 * disparities 0..L-1 with WTA computing the cost on the fly (hgf_aggregate_stereo, direction +1;
 * cost->direction is ignored), and with refine = 1 also the right view's (direction -1) followed
 * by hgf_refine_lr(threshold). Writes the disparity map to `disparity` (host int32 H x W) and
 * returns once it is there. Guidance handles and workspace are kept in ctx between calls (no
 * allocation when shapes repeat). Errors as hgf_prepare, hgf_aggregate_stereo and hgf_refine_lr;
 * HGF_EINVAL for refine not 0 or 1; HGF_ETIMEOUT if a bounded wait in a kernel ran out. */
hgf_status hgf_stereo_host(hgf_ctx *ctx, const float *left, const float *right, int C, int H,
                           int W, int L, const hgf_params *params, const hgf_cost_params *cost,
                           int refine, int threshold, int32_t *disparity, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Post-WTA refinement of a stereo disparity map: the post-processing step that follows WTA in
 * the cost-volume filtering framework of the stereo experiment (Sec. 6). The paper only names the
 * step; the library's reading:
 *  1. left-right consistency: left-view pixel (x, y) with d = disp_left(x, y) is kept when
 *     d >= 0, x - d >= 0 and |d - disp_right(x - d, y)| <= threshold;
 *  2. hole filling: every other pixel takes min(nearest kept disparity to its left, nearest kept
 *     disparity to its right) on its row; with a kept pixel on one side only, that one; with none
 *     on the row, its own disp_left.
 * disp_left, disp_right: device int32 H x W (the labels of hgf_aggregate_stereo with direction
 * +1 and -1, or of hgf_aggregate). out: device int32 H x W (must not alias the inputs). keep:
 * device uint8 H x W scratch, receives 1 for kept pixels, 0 otherwise (caller-owned, required).
 * Enqueued on `stream`; HGF_EINVAL on NULL pointers, H or W < 1, threshold < 0. */
hgf_status hgf_refine_lr(hgf_ctx *ctx, const int32_t *disp_left, const int32_t *disp_right, int H,
                         int W, int threshold, int32_t *out, uint8_t *keep, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Batched inverse of regularised Gram matrices: the paper's comparison of its recursion against a
 * per-matrix factorisation for many small matrices (Sec. 3, Fig. 1b). out_i = (lambda E + S_i)^-1
 * for `count` symmetric n x n matrices S_i (n in 1..9 or 19), one GPU thread per matrix.
 *   S, out: device float64, packed upper triangles row by row (n(n+1)/2 entries: (0,0), (0,1), ..,
 *           (0,n-1), (1,1), ..), element-major over the batch: entry e of matrix i at
 *           [e * count + i]. The caller owns both; they must not overlap.
 *   method: HGF_INV_PROP1 (Prop. 1 recursion with lambda, inverse = -lambda alpha) or
 *           HGF_INV_CHOLESKY (Cholesky factor of lambda E + S, inverse from the factor).
 *   precision: HGF_F64, HGF_DF64 or HGF_F32 arithmetic (input and output stay float64).
 * Enqueued on `stream`. HGF_EINVAL: NULL pointers, count < 1, lambda <= 0, unknown method or
 * precision; HGF_EUNSUPPORTED: n not built. S_i must be positive semidefinite (Gram matrices);
 * otherwise the result is unspecified (no error is detected). */
typedef enum { HGF_INV_PROP1 = 0, HGF_INV_CHOLESKY = 1 } hgf_inverse_method;
hgf_status hgf_batched_inverse(hgf_ctx *ctx, const double *S, int count, int n, double lambda,
                               int method, int precision, double *out, void *stream);

/* Instrumentation (no counterpart in the paper). hgf_launch_count: number of kernels this context
 * has launched since creation. hgf_profile_enable: when on, every kernel launch is bracketed by a
 * CUDA event pair on its stream. hgf_profile_report: waits for the recorded events, writes
 * {"kernel": {"launches": n, "ms": total}, ...} as JSON into buf (cap bytes) and clears them. */
hgf_status hgf_launch_count(hgf_ctx *ctx, unsigned long long *out);
/* The plan of ctx's last aggregation (no counterpart in the paper), for tests and tuning: writes
 * n ints (n >= 1; entries past the eighth are 0) to out: [0] path (1 single-pass kernel, 2 two
 * kernels, 3 plain form, 0 none yet), [1] output columns per strip (strip s covers columns
 * [s * out[1], (s + 1) * out[1])), [2] coefficient columns per strip, [3] rows per band of the
 * coefficient (or single-pass) kernel, [4] rows per band of the output kernel (bands start at
 * multiples of these), [5] labels per pass, [6] labels per chunk (of the last chunk launched),
 * [7] CTAs of the last launch. HGF_EINVAL for NULL arguments or n < 1. */
hgf_status hgf_last_plan(hgf_ctx *ctx, int *out, int n);
/* Kernel watchdog (no counterpart in the paper). Every wait inside a kernel (for a bulk copy into
 * shared memory) is bounded; a wait that runs out sets a per-device status word, the kernel stops
 * its CTA early and that call's results are incomplete. hgf_device_status waits for all work on
 * ctx's device, writes the word to *status (0: no wait ran out) and, when clear is nonzero,
 * resets it. hgf_filter_host checks it itself and returns HGF_ETIMEOUT when it is set. */
hgf_status hgf_device_status(hgf_ctx *ctx, int *status, int clear);
/* Watchdog test hook (no counterpart in the paper): enqueues one CTA that waits, bounded, on an
 * mbarrier nothing arrives on - the same wait k_coef uses for its record copies - so that the
 * wait runs out after limit_us microseconds (1 .. 10^7), sets the device status word and returns.
 * Nothing faults, traps or spins unbounded; the context stays usable. HGF_EINVAL on a bad limit. */
hgf_status hgf_watchdog_probe(hgf_ctx *ctx, int limit_us, void *stream);
hgf_status hgf_profile_enable(hgf_ctx *ctx, int enable);
hgf_status hgf_profile_report(hgf_ctx *ctx, char *buf, size_t cap);

#ifdef __cplusplus
}
#endif
#endif /* HGF_H_ */
