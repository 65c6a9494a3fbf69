// Internal declarations of libhgf (CUDA side). Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>
#include <nvtx3/nvToolsExt.h>

#include "../../include/hgf.h"

namespace hgf {

constexpr int kMaxChannels = 19;        // n <= 19 (degree-3 monomials of RGB)
constexpr int kMaxMonomialDegree = 9;   // gray powers up to I^9 (Table 3 shapes)
constexpr int kStripThreads = 128;      // threads per CTA of the strip kernels

// Channel multiset table: G_i = prod over chan[i][0..deg[i]-1] of I_chan.
struct BasisTable {
  int n;
  int deg[kMaxChannels];
  int chan[kMaxChannels][kMaxMonomialDegree];
};

bool make_basis_table(int C, int degree, int basis, BasisTable *t);

inline int packed_size(int n) { return n * (n + 1) / 2; }

// Per-pixel record of the resident inverse used by the fused kernels, a multiple of 4 floats so
// that records are 16-byte aligned. Centred form: [mu_0..mu_{n-1} | packed n x n Minv | pad];
// paper form: [packed (n+1) x (n+1) inverse | pad], one float more, hence the + 1.
__host__ __device__ constexpr int record_floats(int n) {
  return (n + n * (n + 1) / 2 + 1 + 3) / 4 * 4;
}
// Records are stored plane-major, element e of pixel (x, y) at (e * H + y) * P + x with the row
// pitch P = record_pitch(W) (W rounded up to 4 floats, so that every row starts 16-byte aligned, as
// a tensor copy needs). Consecutive threads of a row read and write consecutive addresses. The
// strip kernels stage the records of one row of their coefficient columns in shared memory with
// one tensor copy (TMA) of a record_box_width(r) x 1 x REC box whose x origin is rounded down to
// a multiple of 4 floats (the tensor copy's alignment rule); columns past the image edge arrive
// as zeros. Records of up to 68 floats (n <= 9) are staged; larger ones (n = 19) are read
// directly from device memory, one coalesced row segment per element.
__host__ __device__ constexpr bool records_staged(int n) { return record_floats(n) <= 68; }
__host__ __device__ constexpr int record_pitch(int W) { return (W + 3) / 4 * 4; }
// Width of the staged box: the kernels' TW = kStripThreads - 2r coefficient columns plus up to
// three columns of alignment offset, rounded up to a multiple of 4.
__host__ __device__ constexpr int record_box_width(int r) {
  return (kStripThreads - 2 * r + 3 + 3) / 4 * 4;
}
// The single-pass kernel stages a box of the widest width (r = 0) whatever r is, so that every
// record element sits at a compile-time offset of the box.
constexpr int kFusedBoxWidth = record_box_width(0);
inline size_t record_total_floats(int H, int W, int n) {
  return (size_t)record_floats(n) * H * record_pitch(W);
}

#ifndef HGF_RECORD_BUFFERS
#define HGF_RECORD_BUFFERS 1
#endif
// Record blocks staged per CTA: 2 = the next row's block arrives while the current row is
// processed; 1 (default) = the next row's copy starts once every thread is done with the current
// row's records and is hidden by that row's vertical update and scans. One buffer halves the
// shared memory of the records, so four CTAs fit on an SM instead of three: k_coef 0.39 -> 0.33 ms
// (450x375, L = 60) and 13.8 -> 11.0 ms (1400x1100, L = 256), n = 9, r = 9.
constexpr int kRecordBuffers = HGF_RECORD_BUFFERS;

#ifndef HGF_COEF_RELOAD
#define HGF_COEF_RELOAD -1
#endif
// k_coef gets the input row leaving its vertical window either from a per-thread shared-memory
// ring or by re-reading it from device memory, where it is still cached in L2, prefetched two
// rows ahead like the new rows. Reload where the records are staged (their buffers take the
// ring's shared memory), the ring otherwise; HGF_COEF_RELOAD = 0 or 1 forces one of them.
__host__ __device__ constexpr bool coef_reload(int n) {
  return HGF_COEF_RELOAD < 0 ? records_staged(n) : HGF_COEF_RELOAD != 0;
}
// Per-pixel coefficient record of the fused kernels' workspace: [b, a_1..a_n | padding] rounded
// up to an even count so that it is read and written as float2 pairs.
__host__ __device__ constexpr int coef_floats(int n) { return (n + 1 + 1) / 2 * 2; }
// The workspace holds one plane per label of the chunk. A plane is tiled by 32 consecutive pixels
// of the flattened index p = y * W + x: tile p / 32 is coef_floats(n) / 2 runs of 32 float2, run q
// holding pair q of the tile's 32 records (coef_pair_index). A warp's 32 consecutive pixels then
// touch at most two tiles, so each float2 access of the warp is one or two contiguous runs
// instead of 32 records 4 * coef_floats(n) bytes apart, and a strip's row stays one contiguous
// block as in a pixel-major layout. The plane is padded to a whole number of tiles.
__host__ __device__ constexpr size_t coef_plane_floats(int n, size_t HW) {
  return (HW + 31) / 32 * 32 * (size_t)coef_floats(n);
}
// Index, in float2 units from the start of a plane, of pair q of pixel p's record.
__host__ __device__ __forceinline__ size_t coef_pair_index(int n, size_t p, int q) {
  return (p >> 5) * (size_t)(coef_floats(n) / 2) * 32 + (size_t)q * 32 + (p & 31);
}

// Packed upper-triangle index of (i, j), i <= j, row by row.
__host__ __device__ constexpr int tri_index(int n, int i, int j) {
  return i * n - (i * (i - 1)) / 2 + (j - i);
}

// Number of in-image samples of the clipped window along one axis.
__device__ __forceinline__ int clipped_count(int x, int r, int W) {
  int lo = x - r < 0 ? 0 : x - r;
  int hi = x + r > W - 1 ? W - 1 : x + r;
  return hi - lo + 1;
}

// Cost element loads (storage dtype -> float32).
__device__ __forceinline__ float load_cost(const float *p, size_t i) { return __ldg(p + i); }
__device__ __forceinline__ float load_cost(const __nv_bfloat16 *p, size_t i) {
  return __bfloat162float(p[i]);
}
__device__ __forceinline__ float load_cost(const __half *p, size_t i) { return __half2float(p[i]); }

// WTA key: orderable float bits in the high word, label in the low word, so that an unsigned
// 64-bit minimum picks the lowest cost and, among equal costs, the lowest label. NaN is counted as
// +inf and -0 as +0 so that equal values compare equal.
__device__ __forceinline__ unsigned long long wta_key(float q, int label) {
  if (q != q) q = __int_as_float(0x7f800000);
  q = q + 0.0f;
  unsigned int u = __float_as_uint(q);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)u << 32) | (unsigned int)label;
}
__device__ __forceinline__ float wta_key_value(unsigned long long key) {
  unsigned int o = (unsigned int)(key >> 32);
  unsigned int u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
  return __uint_as_float(u);
}

// ------------------------------------------------------------------------------------------
// Host-side state
// ------------------------------------------------------------------------------------------
struct Workspace {
  void *ptr = nullptr;
  size_t size = 0;
};

// Per-context kernel instrumentation: a launch counter (always on) and, when enabled, a CUDA
// event pair recorded on the launching stream around every kernel launch.
// NVTX range around an API call (visible in Nsight Systems timelines; a no-op without a tool).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

struct Profiler {
  bool enabled = false;
  unsigned long long launches = 0;
  // the last aggregation's plan (hgf_last_plan): path (1 single pass, 2 two kernels, 3 plain),
  // output columns per strip, coefficient columns per strip, rows per band of the coefficient (or
  // single-pass) kernel and of the output kernel, labels per pass, labels per chunk, CTAs
  int plan[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  struct Rec {
    const char *name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    cudaEvent_t e = nullptr;
    if (!pool.empty()) {
      e = pool.back();
      pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      e = nullptr;
    }
    return e;
  }
};

// Name of the first launch or set-up call that failed on this thread since the last error was
// reported (the API's error message names it), or NULL.
inline const char *&failed_step() {
  static thread_local const char *step = nullptr;
  return step;
}
inline void note_failed(const char *what) {
  if (!failed_step()) failed_step() = what;
}

// Brackets one kernel launch: counts it and, if profiling is on, records events around it; a
// launch that fails is noted by name (failed_step).
class LaunchScope {
 public:
  LaunchScope(Profiler *p, const char *name, cudaStream_t s) : p_(p), name_(name), s_(s) {
    if (!p_) return;
    ++p_->launches;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    // no event pairs inside a graph capture (the capture check only when profiling)
    if (p_->enabled && cudaStreamIsCapturing(s_, &cs) == cudaSuccess &&
        cs == cudaStreamCaptureStatusNone) {
      a_ = p_->get();
      if (a_) cudaEventRecord(a_, s_);
    }
  }
  ~LaunchScope() {
    if (cudaPeekAtLastError() != cudaSuccess) note_failed(name_);
    if (!p_ || !p_->enabled || !a_) return;
    cudaEvent_t b = p_->get();
    if (!b) return;
    cudaEventRecord(b, s_);
    p_->recs.push_back({name_, a_, b});
  }

 private:
  Profiler *p_;
  const char *name_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr;
};

}  // namespace hgf

struct hgf_ctx {
  int device = 0;
  std::atomic<int> sticky{HGF_OK};
  std::string err;
  std::recursive_mutex mu;                // guards the workspaces and err
  hgf::Workspace ws_prepare;     // moment row sums + reduction partials
  hgf::Workspace ws_coef;        // per-chunk coefficient planes (fused path)
  hgf::Workspace ws_keys;        // per-pixel WTA keys
  hgf::Workspace ws_plain;       // plain-form intermediates
  hgf::Workspace ws_io;          // device copies for hgf_filter_host
  hgf::Workspace ws_grad;        // gradient planes of hgf_aggregate_stereo
  // hgf_filter_host uploads the cost volume on io_stream while the guidance precompute runs
  cudaStream_t io_stream = nullptr;
  cudaEvent_t io_fork = nullptr, io_done = nullptr;
  hgf_guidance *host_guidance = nullptr;        // reused by hgf_filter_host, hgf_stereo_host
  hgf_guidance *host_guidance_right = nullptr;  // right view of hgf_stereo_host (refinement)
  hgf_tuning tuning{0, 0, 0, 0, 0};
  int num_sms = 0;
  hgf::Profiler prof;
};

struct hgf_guidance {
  hgf_ctx *ctx = nullptr;
  int C = 0, H = 0, W = 0, n = 0, degree = 0, basis = 0, r = 0;
  double eps = 0.0;
  int inv_precision = HGF_F64, combine = HGF_COMBINE_ALPHA, form = HGF_FORM_CENTRED;
  int compensated = 0;     // Kahan-compensated running sums in the strip kernels
  float *img = nullptr;    // C x H x W, copy of the input image
  float *G = nullptr;      // n x H x W, shifted guidance G_i - c_i
  float *minv = nullptr;   // n(n+1)/2 x H x W, packed (Sigma + eps E)^-1 (centred form only)
  float *mu = nullptr;     // n x H x W, shifted means A(G_i) - c_i (centred form only)
  float *rec = nullptr;    // [mu | packed Minv] per pixel, plane-major (record_pitch)
  float *shift = nullptr;  // n, device: c_i (image mean of G_i)
};

namespace hgf {

// Kernel launchers (each returns cudaGetLastError() of its launches).
cudaError_t launch_make_guidance(const float *img, int C, int H, int W, const BasisTable &bt,
                                 float *G, cudaStream_t s);
cudaError_t launch_prepare(hgf_guidance *g, const float *img, void *ws, size_t ws_size,
                           cudaStream_t s, Profiler *prof);
size_t prepare_workspace_bytes(int n, int H, int W);
cudaError_t launch_export(const hgf_guidance *g, float *minv_out, float *mu_out, cudaStream_t s);

// Cost computed on the fly from a stereo pair (hgf_aggregate_stereo): the reference view is the
// guidance image; `other` is the second view and grad holds both views' gradient planes
// (reference first, H x W each). Passed by value to the coefficient kernel.
struct StereoSource {
  const float *other = nullptr;
  const float *grad = nullptr;
  int direction = 1;
  float alpha = 0.f, tau_c = 0.f, tau_g = 0.f;
};
constexpr int kCostStereo = 100;  // cost_dtype of launch_aggregate for an on-the-fly stereo cost
struct AggregatePlan {
  int K;            // labels per pass
  int band_rows;    // coefficient/output rows per CTA band (0: chosen per kernel from occupancy)
  int chunk;        // labels per workspace chunk
  bool apply_ring;  // output kernel keeps the outgoing rows in a shared-memory ring
  int nominal;      // label count the band heights are planned for: min(64, L rounded up to
                    // even), the same for every chunk of a call so chunking never changes a result
  bool second = false;  // WTA also keeps each pixel's second-smallest key, at keys + H*W
  bool onepass = false;  // single-pass kernel k_fused (a ring buffer instead of the coefficient
                         // workspace, one launch)
  int onepass_ctas = 0;  // its persistent grid
};
AggregatePlan plan_aggregate(const hgf_guidance *g, int L, const hgf_tuning &t, int num_sms);
size_t aggregate_coef_bytes(const hgf_guidance *g, const AggregatePlan &p);
cudaError_t launch_aggregate(const hgf_guidance *g, const void *cost, int cost_dtype, int L,
                             float *filtered, int32_t *labels, float *best, float *coef_ws,
                             unsigned long long *keys, const AggregatePlan &p, cudaStream_t s,
                             Profiler *prof, const StereoSource *stereo = nullptr,
                             float *margin = nullptr);
size_t plain_workspace_bytes(const hgf_guidance *g, int L, int *chunk_out);
cudaError_t launch_aggregate_plain(const hgf_guidance *g, const void *cost, int cost_dtype,
                                   int L, float *filtered, int32_t *labels, float *best,
                                   void *ws, int chunk, cudaStream_t s, Profiler *prof,
                                   float *margin = nullptr);
cudaError_t launch_wta(const float *filtered, int L, int H, int W, int32_t *labels, float *best,
                       cudaStream_t s, Profiler *prof, float *margin = nullptr);
bool aggregate_supported(int n);
// Guidance handle allocation (cudaMalloc) after argument checks; free_guidance releases it.
hgf_status alloc_guidance_checked(hgf_ctx *ctx, int C, int H, int W, const hgf_params *p,
                                  hgf_guidance **out);
void free_guidance(hgf_guidance *g);
bool aggregate_fits(const hgf_guidance *g);
cudaError_t launch_grad_planes(const float *ref, const float *other, int C, int H, int W,
                               float *out, cudaStream_t s, Profiler *prof);
// Left-right consistency + hole filling (hgf_refine_lr).
cudaError_t launch_refine_lr(const int32_t *dl, const int32_t *dr, int H, int W, int threshold,
                             int32_t *out, uint8_t *keep, cudaStream_t s, Profiler *prof);
// Stereo cost volume (hgf_cost_volume).
cudaError_t launch_cost_volume(const float *ref, const float *other, int C, int H, int W, int L,
                               const hgf_cost_params &p, int dtype, void *out, cudaStream_t s,
                               Profiler *prof);
// Batched (lambda E + S_i)^-1, packed, element-major over the batch (hgf_batched_inverse).
cudaError_t launch_batched_inverse(const double *S, int count, int n, double lambda, int method,
                                   int precision, double *out, cudaStream_t s, Profiler *prof);
// Dynamic shared memory of k_coef for n guidance channels, C input channels, K labels, radius r.
size_t coef_smem(int n, int C, int K, int r);
// Device address of the current device's watchdog word (hgf_device_status).
int *device_status_ptr();
// One CTA whose bounded wait cannot complete: it times out after limit_ns and sets the word.
cudaError_t launch_watchdog_probe(unsigned long long limit_ns, cudaStream_t s);
template <int B>
cudaError_t launch_basis(const hgf_guidance *g, const void *cost, int cost_dtype, int L,
                         float *filtered, float *coef_ws, unsigned long long *keys,
                         const AggregatePlan &p, int *status, const StereoSource &stereo,
                         const CUtensorMap &map, cudaStream_t s, Profiler *prof);
// The single-pass kernel of hgf_onepass.cuh (built for the bases with n <= 9: onepass_built in
// hgf_basis.cuh).
template <int B>
cudaError_t launch_onepass(const hgf_guidance *g, const void *cost, int cost_dtype, int L,
                           float *filtered, unsigned long long *keys, unsigned long long *keys2,
                           const AggregatePlan &p, int *status, const StereoSource &stereo,
                           const CUtensorMap &map, float *ring_ws, int grid_ctas, cudaStream_t s,
                           Profiler *prof);
constexpr int kFusedLabels = 2;     // labels per work item of the single-pass kernel
constexpr int kFusedCtasPerSm = 3;  // resident CTAs per SM its persistent grid is sized for
// ... for n guidance channels: up to n = 3 its state fits 128 registers a thread and four CTAs
// share an SM; larger n take 168 registers, three CTAs
__host__ __device__ constexpr int fused_ctas_per_sm(int n) { return n <= 3 ? 4 : kFusedCtasPerSm; }
// Shared memory of the single-pass kernel, whether the plan may select it for g, and the bytes
// of its ring buffer for a persistent grid of `ctas` CTAs.
size_t onepass_smem(int n, int r);
bool onepass_fits(const hgf_guidance *g);
size_t onepass_ring_bytes(int n, int r, int ctas);
// A job of a persistent batch launch of the single-pass kernel (hgf_onepass_batch.cu): its
// guidance, cost, label count, filtered output (or NULL), its own WTA keys (H x W, reset by the
// caller) and the nominal label count its bands are planned for.
struct OnepassBatchJob {
  const hgf_guidance *g;
  const void *cost;
  int cost_dtype, L;
  float *filtered;
  unsigned long long *keys;
  int nominal;
};
// Whether g can join a batch launch (RGB monomials of degree 1 or 2, not compensated, within the
// single-pass kernel's range), the ring floats one CTA needs for g, and the launch itself: one
// persistent launch per 40 jobs on `s` (counters: one zeroed 64-bit work counter per launch).
bool onepass_batch_eligible(const hgf_guidance *g);
size_t onepass_batch_ring_floats(const hgf_guidance *g);
cudaError_t launch_onepass_batch(const OnepassBatchJob *jobs, int n, float *ring_ws,
                                 size_t ring_stride, int grid_ctas, int band_rows_tuned,
                                 unsigned long long *counters, int *status, cudaStream_t s,
                                 Profiler *prof);
constexpr int kOnepassBatchJobsPerLaunch = 40;
// Unpacks per-pixel WTA keys into labels / best (either may be NULL).
cudaError_t launch_wta_finalize(const unsigned long long *keys, int HW, int32_t *labels,
                                float *best, cudaStream_t s, Profiler *prof);
// Tensor map of g's plane-major records: a box_w x 1 x record_floats(n) box (box_w = 0:
// record_box_width(r)).
cudaError_t make_record_map(const hgf_guidance *g, CUtensorMap *out, int box_w = 0);
// Commits the allocation-free entry point's static scratch array on `device` (current) and caches
// its address (hgf_static.cu); hgf_create calls it, and a failure there is not an error.
cudaError_t static_scratch_init(int device);
// Reads (and, with clear, resets) the current device's watchdog word set by bounded waits.
cudaError_t read_device_status(int *status, bool clear);  // fused kernels take this shape

}  // namespace hgf
