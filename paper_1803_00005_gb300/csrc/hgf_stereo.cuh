// The stereo matching cost of hgf_cost_volume (include/hgf.h), as device functions shared by the
// standalone cost-volume kernel (hgf_cost.cu) and the aggregation kernels that compute the cost
// on the fly (hgf_fused.cuh), so that both give bit-identical costs:
//   V(x, y, l) = alpha min(mean_c |I_c(x, y) - J_c(x', y)|, tau_c)
//              + (1 - alpha) min(|dI(x, y) - dJ(x', y)|, tau_g),   x' = clamp(x - dir l, 0, W-1)
// with dI = 0.5 (g(x+1) - g(x-1)) of the channel mean g, neighbours clamped at the border.
#pragma once
#include "hgf_internal.cuh"

namespace hgf {

// channel mean of img at (row offset `row`, column x)
__device__ __forceinline__ float channel_mean(const float *img, int C, size_t HW, size_t row,
                                              int x) {
  float s = 0.f;
  for (int c = 0; c < C; ++c) s += __ldg(img + c * HW + row + x);
  return s / (float)C;
}

// central difference along x of the channel mean, neighbours clamped at the border
__device__ __forceinline__ float grad_x(const float *img, int C, size_t HW, size_t row, int x,
                                        int W) {
  const int xp = min(x + 1, W - 1), xm = max(x - 1, 0);
  return 0.5f * (channel_mean(img, C, HW, row, xp) - channel_mean(img, C, HW, row, xm));
}

// cost from the summed absolute colour difference over C channels and the two gradients
__device__ __forceinline__ float stereo_cost(float colsum, int C, float dI, float dJ, float alpha,
                                             float tau_c, float tau_g) {
  const float col = colsum / (float)C;
  const float grd = fabsf(dI - dJ);
  return alpha * fminf(col, tau_c) + (1.f - alpha) * fminf(grd, tau_g);
}

}  // namespace hgf
