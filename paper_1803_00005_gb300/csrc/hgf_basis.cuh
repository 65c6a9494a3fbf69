// Compile-time polynomial guidance bases (Sec. 4.2) for the hot kernels: each basis id fixes the
// input channel count C, the basis kind and the degree d, hence n and every monomial's factors, so
// that the kernels evaluate G_1..G_n from the C input values with constant register indices.
#pragma once

#include "hgf_internal.cuh"

namespace hgf {

enum BasisId : int {
  B_RGB_MONO1 = 0,  // R, G, B                                             n = 3
  B_RGB_MONO2,      // + RR RG RB GG GB BB                                 n = 9
  B_RGB_MONO3,      // + RRR RRG RRB RGG RGB RBB GGG GGB GBB BBB           n = 19
  B_RGB_POW2,       // R R^2 G G^2 B B^2 (the paper's colour powers, d=2)  n = 6
  B_RGB_POW3,       // R R^2 R^3 G G^2 G^3 B B^2 B^3                       n = 9
  B_GRAY1, B_GRAY2, B_GRAY3, B_GRAY4, B_GRAY5, B_GRAY6, B_GRAY7, B_GRAY8, B_GRAY9,  // I..I^d
  B_COUNT
};

__host__ __device__ constexpr int basis_channels_in(int b) { return b >= B_GRAY1 ? 1 : 3; }

__host__ __device__ constexpr int basis_n(int b) {
  return b == B_RGB_MONO1 ? 3 : b == B_RGB_MONO2 ? 9 : b == B_RGB_MONO3 ? 19
       : b == B_RGB_POW2 ? 6 : b == B_RGB_POW3 ? 9 : (b - B_GRAY1 + 1);
}

// Number of factors (degree) of monomial i.
__host__ __device__ constexpr int basis_deg(int b, int i) {
  if (b >= B_GRAY1) return i + 1;
  if (b == B_RGB_POW2) return i % 2 + 1;
  if (b == B_RGB_POW3) return i % 3 + 1;
  return i < 3 ? 1 : i < 9 ? 2 : 3;  // monomials, degree-major
}

// Input channel of factor k of monomial i.
__host__ __device__ constexpr int basis_factor(int b, int i, int k) {
  if (b >= B_GRAY1) return 0;
  if (b == B_RGB_POW2) return i / 2;
  if (b == B_RGB_POW3) return i / 3;
  if (i < 3) return i;
  // degree 2: (0,0) (0,1) (0,2) (1,1) (1,2) (2,2); degree 3: lexicographic multisets
  int e = i < 9 ? i - 3 : i - 9;
  if (i < 9) {
    int a = e < 3 ? 0 : e < 5 ? 1 : 2;
    int c = a == 0 ? e : a == 1 ? e - 2 : 2;
    return k == 0 ? a : c;
  }
  // degree 3: 000 001 002 011 012 022 111 112 122 222
  const int f0 = e < 6 ? 0 : e < 9 ? 1 : 2;
  const int f1 = e < 3 ? 0 : e < 5 ? 1 : e < 6 ? 2 : e < 8 ? 1 : 2;
  const int f2 = e == 0 ? 0 : e == 1 || e == 3 || e == 6 ? 1 : 2;
  return k == 0 ? f0 : k == 1 ? f1 : f2;
}

// G_i(x) - c_i for every i, from the C input values x (fully unrolled; constant indices).
template <int B>
__device__ __forceinline__ void eval_basis(const float *x, const float *shift, float *g) {
  constexpr int N = basis_n(B);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float v = x[basis_factor(B, i, 0)];
#pragma unroll
    for (int k = 1; k < basis_deg(B, i); ++k) v *= x[basis_factor(B, i, k)];
    g[i] = v - shift[i];
  }
}

// Bases for which the single-pass kernel (hgf_onepass.cuh) is built: n <= 9, whose records are
// staged in shared memory.
__host__ __device__ constexpr bool onepass_built(int b) { return basis_n(b) <= 9; }

// Maps (C, degree, basis) to a basis id, -1 if not built.
inline int basis_id(int C, int degree, int basis) {
  if (C == 1) return degree >= 1 && degree <= 9 ? B_GRAY1 + degree - 1 : -1;
  if (C != 3) return -1;
  if (basis == HGF_BASIS_MONOMIAL || degree == 1)
    return degree == 1 ? B_RGB_MONO1 : degree == 2 ? B_RGB_MONO2 : degree == 3 ? B_RGB_MONO3 : -1;
  return degree == 2 ? B_RGB_POW2 : degree == 3 ? B_RGB_POW3 : -1;
}

// Calls f(std::integral_constant<int, B>) for the runtime basis id b.
template <typename F>
inline bool dispatch_basis(int b, F &&f) {
  switch (b) {
#define HGF_BCASE(X) \
  case X:            \
    f(std::integral_constant<int, X>{}); \
    return true;
    HGF_BCASE(B_RGB_MONO1) HGF_BCASE(B_RGB_MONO2) HGF_BCASE(B_RGB_MONO3) HGF_BCASE(B_RGB_POW2)
    HGF_BCASE(B_RGB_POW3) HGF_BCASE(B_GRAY1) HGF_BCASE(B_GRAY2) HGF_BCASE(B_GRAY3)
    HGF_BCASE(B_GRAY4) HGF_BCASE(B_GRAY5) HGF_BCASE(B_GRAY6) HGF_BCASE(B_GRAY7)
    HGF_BCASE(B_GRAY8) HGF_BCASE(B_GRAY9)
#undef HGF_BCASE
    default:
      return false;
  }
}

}  // namespace hgf
