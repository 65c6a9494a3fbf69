// Batched inverse of regularised Gram matrices, (lambda E + S_i)^-1 for many small symmetric S_i:
// the comparison of Sec. 3 / Fig. 1b between the HGF recursion (Prop. 1) and a per-matrix
// factorisation, one thread per matrix, on the GPU (hgf_batched_inverse in include/hgf.h).
//
// Layout: packed upper triangles (row by row, n(n+1)/2 entries), element-major over the batch:
// entry e of matrix i is at [e * count + i], so consecutive threads touch consecutive addresses.
// Input and output are float64; T is the arithmetic precision.
#include "hgf_internal.cuh"
#include "hgf_df64.cuh"
#include "hgf_prop1.cuh"

namespace hgf {

namespace {

// Prop. 1: alpha by the recursion, then (lambda E + S)^-1 = -lambda alpha.
template <int N, typename T>
__global__ void __launch_bounds__(128) k_inverse_prop1(const double *__restrict__ S, int count,
                                                       double lambda, double *__restrict__ out) {
  constexpr int P = N * (N + 1) / 2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  T s[P], al[P];
#pragma unroll
  for (int e = 0; e < P; ++e) s[e] = T(__ldg(S + (size_t)e * count + i));
  const T lam = T(lambda), inv_lam = T(1) / lam;
  prop1_alpha<N, T>(s, inv_lam, al);
#pragma unroll
  for (int e = 0; e < P; ++e) out[(size_t)e * count + i] = double(-lam * al[e]);
}

// Textbook route: Cholesky factor A = lambda E + S = L L^T (column by column), X = L^-1 by
// forward substitution, A^-1 = X^T X. L and X are lower triangles packed column-free as
// lo(i, j) = i(i+1)/2 + j (j <= i).
__host__ __device__ constexpr int lo_index(int i, int j) { return i * (i + 1) / 2 + j; }

template <int N, typename T>
__global__ void __launch_bounds__(128) k_inverse_cholesky(const double *__restrict__ S, int count,
                                                          double lambda,
                                                          double *__restrict__ out) {
  constexpr int P = N * (N + 1) / 2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  T L[P];
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      T a = T(__ldg(S + (size_t)tri_index(N, c, r) * count + i));
      if (r == c) a += T(lambda);
      L[lo_index(r, c)] = a;
    }
  // in place: L[r][c] for c <= r
#pragma unroll
  for (int c = 0; c < N; ++c) {
    T d = L[lo_index(c, c)];
#pragma unroll
    for (int k = 0; k < c; ++k) d = fma(-L[lo_index(c, k)], L[lo_index(c, k)], d);
    const T lcc = sqrt(d);
    const T inv = T(1) / lcc;
    L[lo_index(c, c)] = lcc;
#pragma unroll
    for (int r = c + 1; r < N; ++r) {
      T v = L[lo_index(r, c)];
#pragma unroll
      for (int k = 0; k < c; ++k) v = fma(-L[lo_index(r, k)], L[lo_index(c, k)], v);
      L[lo_index(r, c)] = v * inv;
    }
  }
  // X = L^-1 (lower), in place column by column from the right
  T X[P];
#pragma unroll
  for (int c = 0; c < N; ++c) {
    X[lo_index(c, c)] = T(1) / L[lo_index(c, c)];
#pragma unroll
    for (int r = c + 1; r < N; ++r) {
      T v = T(0);
#pragma unroll
      for (int k = c; k < r; ++k) v = fma(-L[lo_index(r, k)], X[lo_index(k, c)], v);
      X[lo_index(r, c)] = v / L[lo_index(r, r)];
    }
  }
  // A^-1 = X^T X: (A^-1)_{ab} = sum_{k >= max(a, b)} X_ka X_kb
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int b = a; b < N; ++b) {
      T v = T(0);
#pragma unroll
      for (int k = b; k < N; ++k) v = fma(X[lo_index(k, a)], X[lo_index(k, b)], v);
      out[(size_t)tri_index(N, a, b) * count + i] = double(v);
    }
}

template <int N, typename T>
cudaError_t launch_n(const double *S, int count, double lambda, int method, double *out,
                     cudaStream_t s, Profiler *prof) {
  const int blocks = (count + 127) / 128;
  if (method == HGF_INV_CHOLESKY) {
    LaunchScope ls(prof, "k_inverse_cholesky", s);
    k_inverse_cholesky<N, T><<<blocks, 128, 0, s>>>(S, count, lambda, out);
  } else {
    LaunchScope ls(prof, "k_inverse_prop1", s);
    k_inverse_prop1<N, T><<<blocks, 128, 0, s>>>(S, count, lambda, out);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_t(const double *S, int count, int n, double lambda, int method, double *out,
                     cudaStream_t s, Profiler *prof) {
  switch (n) {
#define HGF_BI_CASE(N) \
  case N:              \
    return launch_n<N, T>(S, count, lambda, method, out, s, prof);
    HGF_BI_CASE(1) HGF_BI_CASE(2) HGF_BI_CASE(3) HGF_BI_CASE(4) HGF_BI_CASE(5) HGF_BI_CASE(6)
    HGF_BI_CASE(7) HGF_BI_CASE(8) HGF_BI_CASE(9) HGF_BI_CASE(19)
#undef HGF_BI_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_batched_inverse(const double *S, int count, int n, double lambda, int method,
                                   int precision, double *out, cudaStream_t s, Profiler *prof) {
  if (precision == HGF_F32) return launch_t<float>(S, count, n, lambda, method, out, s, prof);
  if (precision == HGF_DF64) return launch_t<df64>(S, count, n, lambda, method, out, s, prof);
  return launch_t<double>(S, count, n, lambda, method, out, s, prof);
}

}  // namespace hgf
