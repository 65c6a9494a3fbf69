// Prop. 1 (Sec. 3) in registers: the Sherman-Morrison recursion that builds alpha with
// (lambda E + S)^-1 = lambda^-1 E + S alpha one channel at a time, and the inverse read off alpha.
// Shared by the guidance precompute (hgf_prepare.cu) and the batched inverse (hgf_inverse.cu).
#pragma once
#include "hgf_internal.cuh"

namespace hgf {

// Prop. 1 with lambda on an m x m symmetric S (packed upper triangle), starting from an empty
// alpha: for kappa = 0..m-1
//   u_i   = sum_{j<kappa} alpha_ij S_{j kappa}
//   gamma = -1 / (1 + S_{kappa kappa} / lambda + sum_{i<kappa} S_{kappa i} u_i)
//   alpha_ij += gamma u_i u_j (i, j < kappa);  alpha_{i kappa} = gamma u_i / lambda;
//   alpha_{kappa kappa} = gamma / lambda^2
// which yields (lambda E + S)^-1 = lambda^-1 E + S alpha (Eq. HGF_w3) = -lambda alpha.
// -1 / d. For float64, the Newton-Raphson iteration for the reciprocal, r <- r + r (1 - d r), from
// the float32 reciprocal of d: each step doubles the correct bits (24 -> 48 -> 53), two steps
// give the float64 result to within an ulp with four fused multiply-adds. d > 0 here (the
// recursion's denominators are >= 1 for positive semidefinite S), and |d| stays far inside the
// float32 range.
template <typename T>
__device__ __forceinline__ T neg_recip(T d) { return T(-1) / d; }
template <>
__device__ __forceinline__ double neg_recip<double>(double d) {
  double r = (double)__frcp_rn((float)d);
  r = fma(r, fma(-d, r, 1.0), r);
  r = fma(r, fma(-d, r, 1.0), r);
  return -r;
}

template <int M, typename T>
__device__ __forceinline__ void prop1_alpha(const T *S, T inv_lam, T *al) {
#pragma unroll
  for (int e = 0; e < M * (M + 1) / 2; ++e) al[e] = T(0);
#pragma unroll
  for (int k = 0; k < M; ++k) {
    T u[M > 1 ? M - 1 : 1];
#pragma unroll
    for (int i = 0; i < k; ++i) {
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < k; ++j)
        acc = fma(al[tri_index(M, i < j ? i : j, i < j ? j : i)], S[tri_index(M, j, k)], acc);
      u[i] = acc;
    }
    T den = T(1) + S[tri_index(M, k, k)] * inv_lam;
#pragma unroll
    for (int i = 0; i < k; ++i) den = fma(S[tri_index(M, i, k)], u[i], den);
    const T gam = neg_recip(den);
#pragma unroll
    for (int i = 0; i < k; ++i) {
      const T v = gam * u[i];
#pragma unroll
      for (int j = i; j < k; ++j) al[tri_index(M, i, j)] = fma(v, u[j], al[tri_index(M, i, j)]);
      al[tri_index(M, i, k)] = v * inv_lam;
    }
    al[tri_index(M, k, k)] = gam * inv_lam * inv_lam;
  }
}

// (lambda E + S)^-1 from alpha, packed: lambda^-1 E + S alpha (HGF_COMBINE_W3, Eq. HGF_w3 as
// printed) or -lambda alpha (HGF_COMBINE_ALPHA).
template <int M, typename T>
__device__ __forceinline__ T inverse_entry(const T *S, const T *al, T lam, T inv_lam,
                                           int combine, int i, int j) {
  if (combine != HGF_COMBINE_W3) return -lam * al[tri_index(M, i, j)];
  T acc = (i == j) ? inv_lam : T(0);
#pragma unroll
  for (int k = 0; k < M; ++k)
    acc = fma(S[tri_index(M, i < k ? i : k, i < k ? k : i)],
              al[tri_index(M, k < j ? k : j, k < j ? j : k)], acc);
  return acc;
}

}  // namespace hgf
