// Cost volume of a stereo pair (hgf_cost_volume in include/hgf.h): the cost computation step that
// precedes aggregation in the multi-label pipeline of Sec. 1 (the cost-volume filtering framework
// the paper's stereo experiment uses, Sec. 6). The paper prints no formula; this is the library's
// reading, a truncated colour + gradient difference:
//   V(x, y, l) = alpha min(mean_c |I_c(x, y) - J_c(x', y)|, tau_c)
//              + (1 - alpha) min(|dI(x, y) - dJ(x', y)|, tau_g),   x' = clamp(x - dir l, 0, W-1)
// with dI the central difference along x of the channel mean, neighbours clamped at the border.
// One thread per pixel and 16 labels: the reference pixel and its gradient are loaded once; the
// matching pixels of neighbouring threads are neighbours in memory (coalesced, L1-shared), and
// each label slice is written as one coalesced row per warp. Bound by the HBM write of V.
#include "hgf_stereo.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace hgf {

namespace {

constexpr int kCostThreads = 128;
constexpr int kCostLabels = 16;

__device__ __forceinline__ void store_cost(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_cost(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void store_cost(__half *p, float v) { *p = __float2half_rn(v); }

template <typename OT>
__global__ void __launch_bounds__(kCostThreads) k_cost_volume(
    const float *__restrict__ ref, const float *__restrict__ other, int C, int H, int W, int L,
    int direction, float alpha, float tau_c, float tau_g, OT *__restrict__ out) {
  const int x = blockIdx.x * kCostThreads + threadIdx.x;
  const int y = blockIdx.y;
  const int l0 = blockIdx.z * kCostLabels;
  if (x >= W) return;
  const size_t HW = (size_t)H * W, row = (size_t)y * W;
  float I[3];
  for (int c = 0; c < C; ++c) I[c] = __ldg(ref + c * HW + row + x);
  const float dI = grad_x(ref, C, HW, row, x, W);
  const int l1 = min(L, l0 + kCostLabels);
  for (int l = l0; l < l1; ++l) {
    const int xs = min(max(x - direction * l, 0), W - 1);
    float col = 0.f;
    for (int c = 0; c < C; ++c) col += fabsf(I[c] - __ldg(other + c * HW + row + xs));
    const float v = stereo_cost(col, C, dI, grad_x(other, C, HW, row, xs, W), alpha, tau_c, tau_g);
    store_cost(out + (size_t)l * HW + row + x, v);
  }
}

// gradient planes dI of both views for the fused stereo aggregation: out[v][y][x]
__global__ void __launch_bounds__(kCostThreads) k_grad_planes(const float *__restrict__ ref,
                                                              const float *__restrict__ other,
                                                              int C, int H, int W,
                                                              float *__restrict__ out) {
  const int x = blockIdx.x * kCostThreads + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= W) return;
  const size_t HW = (size_t)H * W, row = (size_t)y * W;
  const float *img = blockIdx.z == 0 ? ref : other;
  out[blockIdx.z * HW + row + x] = grad_x(img, C, HW, row, x, W);
}

template <typename OT>
cudaError_t launch_t(const float *ref, const float *other, int C, int H, int W, int L,
                     int direction, const hgf_cost_params &p, void *out, cudaStream_t s,
                     Profiler *prof) {
  dim3 grid((W + kCostThreads - 1) / kCostThreads, H, (L + kCostLabels - 1) / kCostLabels);
  LaunchScope ls(prof, "k_cost_volume", s);
  k_cost_volume<OT><<<grid, kCostThreads, 0, s>>>(ref, other, C, H, W, L, direction,
                                                  (float)p.alpha, (float)p.tau_color,
                                                  (float)p.tau_grad, (OT *)out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grad_planes(const float *ref, const float *other, int C, int H, int W,
                               float *out, cudaStream_t s, Profiler *prof) {
  dim3 grid((W + kCostThreads - 1) / kCostThreads, H, 2);
  LaunchScope ls(prof, "k_grad_planes", s);
  k_grad_planes<<<grid, kCostThreads, 0, s>>>(ref, other, C, H, W, out);
  return cudaGetLastError();
}

cudaError_t launch_cost_volume(const float *ref, const float *other, int C, int H, int W, int L,
                               const hgf_cost_params &p, int dtype, void *out, cudaStream_t s,
                               Profiler *prof) {
  switch (dtype) {
    case HGF_F32:
      return launch_t<float>(ref, other, C, H, W, L, p.direction, p, out, s, prof);
    case HGF_BF16:
      return launch_t<__nv_bfloat16>(ref, other, C, H, W, L, p.direction, p, out, s, prof);
    case HGF_F16:
      return launch_t<__half>(ref, other, C, H, W, L, p.direction, p, out, s, prof);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace hgf
