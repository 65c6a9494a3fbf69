// hgf_aggregate_static: the fused aggregation + WTA of hgf_aggregate for callers that must not
// allocate device memory once they are running - for example a fixed-latency loop (cudaMalloc and
// cudaFree can synchronise the device and block for an unbounded time), or a plugin inside a host
// program that hands out all device memory from its own allocator at start-up, so that a late
// cudaMalloc fails or fragments the host's pool. Instead of
// the context's growable workspace, this entry point takes its scratch (the per-pixel WTA keys and,
// on the two-kernel path, the per-chunk coefficient planes) from one file-scope device array of
// fixed size, which every GPU that loads this library holds until the process exits.
//
// Set-up: hgf_create looks up the array's device address with cudaGetSymbolAddress, with the
// context's device current. That lookup loads this file's device module, which is when the array
// is committed on that device (under lazy module loading it would otherwise be committed by the
// first call of this entry point). If it failed there (no memory left), the entry point tries
// again on its first call and returns HGF_ENOMEM, without marking the context failed, while it
// keeps failing; make the first call before any stream capture in that case. Once the address is
// known a call allocates nothing and only enqueues a memset and kernels on `stream`.
//
// Every call shares the one array, and it keeps the previous call's contents: the WTA keys are
// reset at the start of each call and every coefficient plane is written before it is read.
// Calls whose work overlaps on the GPU (different streams, or different contexts on one device)
// race on the array and must be serialised by the caller.
#include "hgf_internal.cuh"

#include <algorithm>
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {};

// Device address of the array on `device` (current), looked up once per device.
cudaError_t static_scratch(int device, void **out) {
  if (!out) return cudaErrorInvalidValue;
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[device] = p;
  }
  *out = g_static_ptr[device];
  return cudaSuccess;
}

}  // namespace

namespace hgf {
// Commits the array on `device` (current) and caches its address; called by hgf_create.
cudaError_t static_scratch_init(int device) {
  void *p = nullptr;
  return static_scratch(device, &p);
}
}  // namespace hgf

extern "C" hgf_status hgf_aggregate_static(hgf_ctx *ctx, const hgf_guidance *g, const void *cost,
                                           int cost_dtype, int L, void *filtered,
                                           int filtered_dtype, int32_t *labels, float *best,
                                           void *stream) {
  if (!ctx) return HGF_EINVAL;
  if (ctx->sticky.load() != HGF_OK) return HGF_ECUDA;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  auto fail = [&](hgf_status st, const std::string &msg) {
    ctx->err = "hgf_aggregate_static: " + msg;
    return st;
  };
  auto cuda_fail = [&](cudaError_t e, const char *where) {
    ctx->sticky.store(HGF_ECUDA);
    ctx->err = std::string("hgf_aggregate_static: ") + where + ": " + cudaGetErrorString(e);
    return HGF_ECUDA;
  };
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  if (!g || g->ctx != ctx) return fail(HGF_EINVAL, "bad guidance handle");
  if (!cost) return fail(HGF_EINVAL, "cost is NULL");
  if (cost_dtype != HGF_F32 && cost_dtype != HGF_BF16 && cost_dtype != HGF_F16)
    return fail(HGF_EINVAL, "cost dtype must be HGF_F32, HGF_BF16 or HGF_F16");
  if (L < 1) return fail(HGF_EINVAL, "L must be >= 1");
  if (!filtered && !labels && !best) return fail(HGF_EINVAL, "no output requested");
  if (filtered && filtered_dtype != HGF_F32) return fail(HGF_EINVAL, "filtered must be HGF_F32");
  if (!hgf::aggregate_fits(g)) return fail(HGF_EUNSUPPORTED, "window too wide for this path");

  hgf::AggregatePlan plan = hgf::plan_aggregate(g, L, ctx->tuning, ctx->num_sms);
  const size_t HW = (size_t)g->H * g->W;
  const size_t keys_bytes = (HW * sizeof(unsigned long long) + 255) / 256 * 256;
  // the single-pass kernel needs the keys and one ring slot per CTA of its persistent grid (the
  // grid shrinks to what fits); the two-kernel path one coefficient plane per label of a chunk
  const size_t per_unit = plan.onepass
                              ? hgf::onepass_ring_bytes(g->n, g->r, 1)
                              : hgf::coef_plane_floats(g->n, HW) * sizeof(float);
  if (keys_bytes + per_unit > kStaticScratchBytes)
    return fail(HGF_EUNSUPPORTED,
                "image too large for the " + std::to_string(kStaticScratchBytes >> 20) +
                    " MiB static scratch: needs " + std::to_string(keys_bytes + per_unit) +
                    " bytes; use hgf_aggregate");
  const int fit = (int)((kStaticScratchBytes - keys_bytes) / per_unit);
  if (plan.onepass)
    plan.onepass_ctas = std::max(1, std::min(plan.onepass_ctas, fit));
  else
    plan.chunk = std::max(1, std::min(plan.chunk, fit));

  void *base = nullptr;
  e = static_scratch(ctx->device, &base);
  if (e != cudaSuccess) {
    cudaGetLastError();  // not sticky: the context stays usable
    return fail(HGF_ENOMEM, std::string("the static scratch array is not available on this "
                                        "device: ") + cudaGetErrorString(e));
  }
  hgf::Profiler count_only;  // counts launches, records no events
  e = hgf::launch_aggregate(g, cost, cost_dtype, L, (float *)filtered, labels, best,
                            (float *)((char *)base + keys_bytes), (unsigned long long *)base,
                            plan, (cudaStream_t)stream, &count_only);
  ctx->prof.launches += count_only.launches;
  for (int i = 0; i < 8; ++i) ctx->prof.plan[i] = count_only.plan[i];
  if (e != cudaSuccess) return cuda_fail(e, "launch");
  return HGF_OK;
}
