// Post-WTA refinement of a stereo disparity map (hgf_refine_lr in include/hgf.h): the "post
// processing" step that follows WTA in the cost-volume filtering framework of the stereo
// experiment (Sec. 6). The paper names the step only; this is the library's reading:
//  1. left-right consistency: a left-view pixel (x, y) with disparity d = D_L(x, y) is kept when
//     x - d >= 0 and |d - D_R(x - d, y)| <= threshold, where D_R is the right-view map;
//  2. hole filling: every other pixel takes the smaller of the nearest kept disparities to its
//     left and to its right on the same row (the background side of an occlusion); with a kept
//     pixel on one side only, that one; with none on the row, its own D_L.
// k_lr_check is one thread per pixel; k_fill is one CTA per row that finds, for every x, the
// nearest kept index on each side with block-wide max / min scans over the row in chunks.
#include "hgf_internal.cuh"

namespace hgf {

namespace {

constexpr int kFillThreads = 256;

__global__ void k_lr_check(const int32_t *__restrict__ dl, const int32_t *__restrict__ dr, int H,
                           int W, int threshold, uint8_t *__restrict__ keep) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= W) return;
  const size_t p = (size_t)y * W + x;
  const int d = dl[p];
  const int xr = x - d;
  bool ok = d >= 0 && xr >= 0 && xr < W;
  if (ok) {
    const int e = dr[(size_t)y * W + xr] - d;
    ok = (e < 0 ? -e : e) <= threshold;
  }
  keep[p] = ok ? 1 : 0;
}

// block-wide inclusive scan (max when MAX, min otherwise) of one value per thread
template <bool MAX>
__device__ __forceinline__ int block_scan(int v, int *warp_tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = MAX ? max(v, u) : min(v, u);
  }
  if (lane == 31) warp_tot[wid] = v;
  __syncthreads();
  if (wid > 0) {
    int pre = warp_tot[0];
    for (int w = 1; w < wid; ++w) pre = MAX ? max(pre, warp_tot[w]) : min(pre, warp_tot[w]);
    v = MAX ? max(v, pre) : min(v, pre);
  }
  __syncthreads();
  return v;
}

__global__ void __launch_bounds__(kFillThreads) k_fill(const int32_t *__restrict__ dl,
                                                       const uint8_t *__restrict__ keep, int W,
                                                       int32_t *__restrict__ out) {
  __shared__ int warp_tot[kFillThreads / 32];
  __shared__ int carry;
  const int y = blockIdx.x;
  const size_t row = (size_t)y * W;
  const int t = threadIdx.x;
  const int chunks = (W + kFillThreads - 1) / kFillThreads;
  // pass 1, left to right: last kept index <= x (-1 if none), written to out as a scratch index
  if (t == 0) carry = -1;
  __syncthreads();
  for (int c = 0; c < chunks; ++c) {
    const int x = c * kFillThreads + t;
    int v = (x < W && keep[row + x]) ? x : -1;
    v = block_scan<true>(v, warp_tot);
    v = max(v, carry);
    if (x < W) out[row + x] = v;
    __syncthreads();
    if (t == kFillThreads - 1) carry = v;
    __syncthreads();
  }
  // pass 2, right to left: first kept index >= x (W if none); resolve every pixel
  if (t == 0) carry = W;
  __syncthreads();
  for (int c = chunks - 1; c >= 0; --c) {
    const int x = c * kFillThreads + (kFillThreads - 1 - t);  // thread t scans from the right
    int v = (x < W && keep[row + x]) ? x : W;
    v = block_scan<false>(v, warp_tot);
    v = min(v, carry);
    if (x < W) {
      const int lo = out[row + x];
      int d;
      if (keep[row + x]) {
        d = dl[row + x];
      } else if (lo >= 0 && v < W) {
        d = min(dl[row + lo], dl[row + v]);
      } else if (lo >= 0) {
        d = dl[row + lo];
      } else if (v < W) {
        d = dl[row + v];
      } else {
        d = dl[row + x];
      }
      out[row + x] = d;
    }
    __syncthreads();
    if (t == kFillThreads - 1) carry = v;
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_refine_lr(const int32_t *dl, const int32_t *dr, int H, int W, int threshold,
                             int32_t *out, uint8_t *keep, cudaStream_t s, Profiler *prof) {
  {
    LaunchScope ls(prof, "k_lr_check", s);
    k_lr_check<<<dim3((W + 127) / 128, H), 128, 0, s>>>(dl, dr, H, W, threshold, keep);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  LaunchScope ls(prof, "k_fill", s);
  k_fill<<<H, kFillThreads, 0, s>>>(dl, keep, W, out);
  return cudaGetLastError();
}

}  // namespace hgf
