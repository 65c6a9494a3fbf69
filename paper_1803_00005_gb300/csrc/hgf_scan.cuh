// Shared-memory row scans of the strip kernels (hgf_fused.cuh, hgf_prepare.cu): a CTA of
// kStripThreads threads owns one column each; per image row it writes one value per channel into
// a shared row, scans the rows, and reads window sums as differences of inclusive prefix sums.
#pragma once
#include "hgf_internal.cuh"

namespace hgf {
namespace strip {

constexpr int NT = kStripThreads;
constexpr int kRowStride = NT + 4;  // [0..3] padding (index 3 holds the zero prefix), 4+t values

// Inclusive prefix sums along each shared row (values at [4 .. 4+NT)), one warp per row.
// All rows of a warp are loaded first and their shuffle chains advance together, so the chain
// latency is paid once per warp rather than once per row. Warp w scans rows w, w+4, w+8, ..
// (RPW of them at most) among the first `rows`.
template <int RPW>
__device__ __forceinline__ void scan_rows(float *sA, int rows) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  float4 v[RPW];
  float tot[RPW];
#pragma unroll
  for (int j = 0; j < RPW; ++j) {
    const int row = warp + j * NW;
    v[j] = row < rows ? *(reinterpret_cast<float4 *>(sA + row * kRowStride + 4) + lane)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    v[j].y += v[j].x;
    v[j].z += v[j].y;
    v[j].w += v[j].z;
    tot[j] = v[j].w;
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
    for (int j = 0; j < RPW; ++j) {
      const float o = __shfl_up_sync(0xffffffffu, tot[j], off);
      if (lane >= off) tot[j] += o;
    }
  }
#pragma unroll
  for (int j = 0; j < RPW; ++j) {
    const int row = warp + j * NW;
    const float ex = tot[j] - v[j].w;
    v[j].x += ex;
    v[j].y += ex;
    v[j].z += ex;
    v[j].w += ex;
    if (row < rows) *(reinterpret_cast<float4 *>(sA + row * kRowStride + 4) + lane) = v[j];
  }
}

// Window sum [t, t + 2r] of a scanned shared row.
__device__ __forceinline__ float window(const float *row, int t, int r) {
  return row[4 + t + 2 * r] - row[3 + t];
}

}  // namespace strip
}  // namespace hgf
