// Host side of the fused multi-label aggregation + WTA (Sec. 1 pipeline): planning (labels per
// pass, bands, chunks), dispatch to the per-basis kernels of hgf_fused.cuh (compiled in the
// hgf_fused_*.cu translation units), the kernel watchdog word, and the WTA kernels.
#include "hgf_basis.cuh"
#include "hgf_mbarrier.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

namespace hgf {

namespace {

constexpr int NT = kStripThreads;
constexpr int kRowStride = NT + 4;  // shared row stride of the fused kernels' scan buffers
__device__ int g_device_status = 0;  // nonzero after a bounded wait in a kernel ran out

// Unpacks the per-pixel WTA keys. With `second` (the smallest key other than the winner's, all
// ones while a pixel has seen one label only), margin = second-best cost - best cost, +inf for a
// single label.
__global__ void k_wta_finalize(const unsigned long long *__restrict__ keys,
                               const unsigned long long *__restrict__ second, int HW,
                               int32_t *__restrict__ labels, float *__restrict__ best,
                               float *__restrict__ margin) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW) return;
  unsigned long long key = keys[p];
  if (labels) labels[p] = (int32_t)(unsigned int)(key & 0xffffffffull);
  if (best) best[p] = wta_key_value(key);
  if (margin) {
    const unsigned long long k2 = second[p];
    margin[p] = k2 == ~0ull ? __int_as_float(0x7f800000) : wta_key_value(k2) - wta_key_value(key);
  }
}

// Standalone WTA over a filtered volume: one thread per pixel scanning the labels in order,
// keeping the best and second-best values (a tie with the best gives margin 0).
__global__ void k_wta_volume(const float *__restrict__ q, int L, int HW,
                             int32_t *__restrict__ labels, float *__restrict__ best,
                             float *__restrict__ margin) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW) return;
  const float inf = __int_as_float(0x7f800000);
  float b = 0.f, b2 = inf;
  int lb = 0;
  for (int l = 0; l < L; ++l) {
    float v = q[(size_t)l * HW + p];
    if (v != v) v = inf;
    if (l == 0) {
      b = v;
    } else if (v < b) {
      b2 = b;
      b = v;
      lb = l;
    } else if (v < b2) {
      b2 = v;
    }
  }
  if (labels) labels[p] = lb;
  if (best) best[p] = b;
  if (margin) margin[p] = L == 1 ? inf : b2 - b;
}

// Watchdog probe: one CTA waits, bounded, on an mbarrier that nothing arrives on (it expects one
// arrival that never comes), exactly as k_coef waits for a record copy; when the limit runs out
// it records the timeout in the status word and returns. No copy is in flight, so the CTA exits
// cleanly.
__global__ void k_watchdog_probe(int *status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit_ns)) atomicExch(status, 1);
}

}  // namespace

// Dynamic shared memory of k_coef for n guidance channels, C input channels, K labels, radius r:
// 128 bytes of alignment slack, the staged record boxes, two mbarriers, two scan buffers, the
// raw-row ring (ring mode only).
size_t coef_smem(int n, int C, int K, int r) {
  const bool stage = records_staged(n);
  const size_t rbuf = ((size_t)record_floats(n) * record_box_width(r) + 31) / 32 * 32;
  return 128 + 16 +
         sizeof(float) * ((size_t)2 * K * (n + 1) * kRowStride +
                          (stage ? (size_t)kRecordBuffers * rbuf : 0) +
                          (coef_reload(n) ? 0 : (size_t)(2 * r + 1) * (C + K) * NT));
}

// Dynamic shared memory of the single-pass kernel k_fused (hgf_onepass.cuh): 128 bytes of
// alignment slack, the record box, an mbarrier and the scan rows of both stages for its labels.
size_t onepass_smem(int n, int r) {
  (void)r;
  return 128 + sizeof(float) * (size_t)record_floats(n) * kFusedBoxWidth + 16 +
         sizeof(float) * (size_t)2 * kFusedLabels * (n + 1) * kRowStride;
}

// Its ring buffer: per CTA, (2r+1) rows x labels x (n + 1) channels x (128 - 4r) output columns.
size_t onepass_ring_bytes(int n, int r, int ctas) {
  return sizeof(float) * (size_t)ctas * (2 * r + 1) * kFusedLabels * (n + 1) * (NT - 4 * r);
}

// The single-pass kernel serves n <= 9 (records staged) while its strip keeps at least 32 output
// columns (r <= 24) and its shared memory fits one CTA.
bool onepass_fits(const hgf_guidance *g) {
  return records_staged(g->n) && NT - 4 * g->r >= 32 && onepass_smem(g->n, g->r) <= 227 * 1024;
}

// Tensor map of the plane-major records of g: dims (W, H, REC) with row pitch record_pitch(W),
// box (record_box_width(r), 1, REC); columns outside [0, W) load as zeros. The encoder is the
// driver's cuTensorMapEncodeTiled, looked up once through the runtime.
cudaError_t make_record_map(const hgf_guidance *g, CUtensorMap *out, int box_w) {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  std::call_once(once, [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    else
      cudaGetLastError();
  });
  if (!encode) {
    note_failed("cuTensorMapEncodeTiled lookup");
    return cudaErrorNotSupported;
  }
  const int REC = record_floats(g->n);
  const cuuint64_t P = (cuuint64_t)record_pitch(g->W);
  const cuuint64_t dims[3] = {(cuuint64_t)g->W, (cuuint64_t)g->H, (cuuint64_t)REC};
  const cuuint64_t strides[2] = {P * sizeof(float), P * g->H * sizeof(float)};
  const int bw = box_w > 0 ? box_w : record_box_width(g->r);
  const cuuint32_t box[3] = {(cuuint32_t)bw, 1u, (cuuint32_t)REC};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  if (REC > 256 || bw > 256 || bw % 4) return cudaErrorInvalidValue;
  CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)g->rec, dims, strides, box,
                      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) note_failed("cuTensorMapEncodeTiled");
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Device address of the watchdog word on the current device (looked up once per device).
int *device_status_ptr() {
  static std::mutex mu;
  static int *ptr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return nullptr;
    ptr[dev] = (int *)p;
  }
  return ptr[dev];
}

bool aggregate_supported(int n) {
  switch (n) {
    case 1: case 2: case 3: case 4: case 5: case 6: case 7: case 8: case 9: case 19:
      return true;
    default:
      return false;
  }
}

cudaError_t read_device_status(int *status, bool clear) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_device_status, sizeof(int));
  if (e == cudaSuccess && clear && v != 0) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int));
  }
  *status = v;
  return e;
}

cudaError_t launch_watchdog_probe(unsigned long long limit_ns, cudaStream_t s) {
  int *status = device_status_ptr();
  if (!status) return cudaErrorInvalidValue;
  k_watchdog_probe<<<1, 32, 0, s>>>(status, limit_ns);
  return cudaGetLastError();
}

bool aggregate_fits(const hgf_guidance *g) {
  return 2 * g->r + 1 < NT && coef_smem(g->n, g->C, 2, g->r) <= 227 * 1024;
}

AggregatePlan plan_aggregate(const hgf_guidance *g, int L, const hgf_tuning &t, int num_sms) {
  AggregatePlan p;
  // two labels per pass unless tuned: with the records staged in shared memory, two beat four
  // and eight on both measured sizes (k_coef, n = 9, r = 9: 450x375 0.44 / 0.54 / 0.78 ms,
  // 1400x1100 13.3 / 16.4 / 26.9 ms). K never changes a result (each label's arithmetic is the
  // same for any K).
  p.K = 2;
  p.nominal = std::max(2, std::min(64, (L + 1) / 2 * 2));
  if (t.labels_per_pass == 2 ||
      ((t.labels_per_pass == 4 || t.labels_per_pass == 8) &&
       coef_smem(g->n, g->C, t.labels_per_pass, g->r) <= 227 * 1024) ||
      (t.labels_per_pass == 1 && !records_staged(g->n)))
    p.K = t.labels_per_pass;
  const size_t plane = coef_plane_floats(g->n, (size_t)g->H * g->W) * sizeof(float);
  // labels per chunk: all labels while the coefficient workspace stays under 4 GiB
  size_t cap = std::max<size_t>(1, ((size_t)4 << 30) / plane);
  p.chunk = t.chunk_labels > 0 ? t.chunk_labels : (int)std::min<size_t>((size_t)L, cap);
  p.chunk = std::max(1, std::min(p.chunk, L));
  const int TW = NT - 2 * g->r;
  const int strips = (g->W + TW - 1) / TW;
  const int passes = (p.chunk + p.K - 1) / p.K;
  // the outgoing coefficient rows of the output kernel are reloaded by default: they were read
  // 2r+1 steps earlier and are still in L2, and without the ring more CTAs fit on an SM
  const size_t ring = sizeof(float) * (size_t)(g->n + 1) * ((2 * g->r + 1) * NT + 2 * kRowStride);
  p.apply_ring = t.apply_mode == 1 && ring <= 227 * 1024;
  (void)strips;
  (void)passes;
  (void)num_sms;
  p.band_rows = t.band_rows;  // 0: each kernel picks its bands from its occupancy at launch
  // kernel path: as tuned, else for n <= 3 the single pass (four CTAs an SM), and for larger n
  // the single pass when its narrower output strips (128 - 4r columns against the two-kernel
  // path's 128 - 2r) cost no extra strips and the job fills the GPU. On GB300 (warm aggregation,
  // 15 shapes): at n = 3 the single pass was 1-17 % faster on all five shapes, also with more
  // strips (450x375/L=60/r=4: 0.253 vs 0.263 ms with 5 against 4 strips; 640x480/L=64/r=4:
  // 0.409 vs 0.519 ms; 320x240/L=32: 0.082 vs 0.085 ms); at n = 9 with equal strip counts it
  // was 1-5 % faster from 8 Mpixel*labels up (450x375/L=60/r=9: 0.531 vs 0.541 ms) and with more
  // strips 3-40 % slower (1400x1100/L=256/r=9: 16 vs 13 strips, 20.4 vs 17.9 ms)
  const int strips_single = (g->W + NT - 4 * g->r - 1) / std::max(1, NT - 4 * g->r);
  const int strips_two = (g->W + NT - 2 * g->r - 1) / std::max(1, NT - 2 * g->r);
  const bool auto_single = g->n <= 3 || (strips_single == strips_two &&
                                         (double)g->H * g->W * L >= 8.0e6);
  p.onepass = onepass_fits(g) && (t.kernel == 1 || (t.kernel == 0 && auto_single));
  p.onepass_ctas = std::max(1, num_sms) * fused_ctas_per_sm(g->n);
  return p;
}

size_t aggregate_coef_bytes(const hgf_guidance *g, const AggregatePlan &p) {
  if (p.onepass) return onepass_ring_bytes(g->n, g->r, p.onepass_ctas);
  return (size_t)p.chunk * coef_plane_floats(g->n, (size_t)g->H * g->W) * sizeof(float);
}

cudaError_t launch_aggregate(const hgf_guidance *g, const void *cost, int cost_dtype, int L,
                             float *filtered, int32_t *labels, float *best, float *coef_ws,
                             unsigned long long *keys, const AggregatePlan &plan,
                             cudaStream_t s, Profiler *prof, const StereoSource *stereo,
                             float *margin) {
  const int HW = g->H * g->W;
  const bool want_wta = labels || best || margin;
  unsigned long long *k = want_wta ? keys : nullptr;
  AggregatePlan p = plan;
  p.second = margin != nullptr;  // the keys workspace then holds 2 x H x W keys
  if (k) {
    cudaError_t e = cudaMemsetAsync(k, 0xff, (size_t)HW * (p.second ? 2 : 1) *
                                                 sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  if (cost_dtype == kCostStereo && !stereo) return cudaErrorInvalidValue;
  const int b = basis_id(g->C, g->degree, g->basis);
  int *status = device_status_ptr();
  if (!status) return cudaErrorInvalidValue;
  CUtensorMap map;
  cudaError_t e = make_record_map(g, &map, p.onepass ? kFusedBoxWidth : 0);
  if (e != cudaSuccess) return e;
  e = cudaErrorInvalidValue;
  bool ok = dispatch_basis(b, [&](auto bc) {
    constexpr int B = decltype(bc)::value;
    e = launch_basis<B>(g, cost, cost_dtype, L, filtered, coef_ws, k, p, status,
                        stereo ? *stereo : StereoSource{}, map, s, prof);
  });
  if (!ok) return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  if (k) {
    LaunchScope ls(prof, "k_wta_finalize", s);
    k_wta_finalize<<<(HW + 255) / 256, 256, 0, s>>>(k, p.second ? k + HW : nullptr, HW, labels,
                                                    best, margin);
  }
  return cudaGetLastError();
}

cudaError_t launch_wta_finalize(const unsigned long long *keys, int HW, int32_t *labels,
                                float *best, cudaStream_t s, Profiler *prof) {
  LaunchScope ls(prof, "k_wta_finalize", s);
  k_wta_finalize<<<(HW + 255) / 256, 256, 0, s>>>(keys, nullptr, HW, labels, best, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_wta(const float *filtered, int L, int H, int W, int32_t *labels, float *best,
                       cudaStream_t s, Profiler *prof, float *margin) {
  int HW = H * W;
  LaunchScope ls(prof, "k_wta_volume", s);
  k_wta_volume<<<(HW + 255) / 256, 256, 0, s>>>(filtered, L, HW, labels, best, margin);
  return cudaGetLastError();
}

}  // namespace hgf
