// Fused multi-label aggregation + WTA (Sec. 1 pipeline with the centred form of Sec. 5.1 and the
// multipoint aggregation of Sec. 4.1, Eq. HGF_z1).
//
// Two streaming kernels per chunk of labels, both over vertical strips of the image:
//   k_coef : per input row, float32 vertical running sums of (p, G_1 p, .., G_n p) for K labels,
//            horizontal window sums by a prefix scan in shared memory, then per coefficient pixel
//            cov = A(G p) - mu A(p), a = Minv cov, b = A(p) - a.mu. Each cost element is read from
//            device memory once (plus its halo columns) and the resident inverse once per K labels.
//   k_apply: per coefficient row, vertical running sums of (b, a_1..a_n), horizontal window sums,
//            q = sum_i A(a_i) G_i + A(b), minimum over the CTA's labels and one packed 64-bit
//            atomicMin per pixel (cost in the high word, label in the low word: lowest cost, then
//            lowest label).
// Windows are clipped at the image border: samples outside the image never enter a sum and the
// means divide by the in-image count N(x, y).
#include "hgf_internal.cuh"

#include <algorithm>

namespace hgf {

namespace {

constexpr int NT = kStripThreads;
constexpr int kRowStride = NT + 4;  // [0..3] padding (index 3 holds the zero prefix), 4+t values

// Inclusive prefix sums along each shared row (values at [4 .. 4+NT)), one warp per row.
__device__ __forceinline__ void scan_rows(float *sA, int rows) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int row = warp; row < rows; row += NT / 32) {
    float4 *p = reinterpret_cast<float4 *>(sA + row * kRowStride + 4) + lane;
    float4 v = *p;
    v.y += v.x;
    v.z += v.y;
    v.w += v.z;
    float tot = v.w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      float o = __shfl_up_sync(0xffffffffu, tot, off);
      if (lane >= off) tot += o;
    }
    float ex = tot - v.w;
    v.x += ex;
    v.y += ex;
    v.z += ex;
    v.w += ex;
    *p = v;
  }
}

template <int NG, int K, typename CT>
__global__ void __launch_bounds__(NT) k_coef(const CT *__restrict__ cost, int H, int W, int r,
                                             const float *__restrict__ G,
                                             const float *__restrict__ minv,
                                             const float *__restrict__ mu,
                                             float *__restrict__ coef, int l_first, int n_chunk,
                                             int band_rows) {
  constexpr int C1 = NG + 1;
  __shared__ __align__(16) float sA[K * C1 * kRowStride];
  const size_t HW = (size_t)H * W;
  const int t = threadIdx.x;
  const int TW = NT - 2 * r;
  const int x0 = blockIdx.x * TW;
  const int xi = x0 - r + t;
  const bool col_ok = xi >= 0 && xi < W;
  const int Y0 = blockIdx.y * band_rows;
  const int Y1 = min(H, Y0 + band_rows);
  const int k0 = blockIdx.z * K;
  const int nk = min(K, n_chunk - k0);
  const int add_lo = max(0, Y0 - r);

  for (int i = t; i < K * C1; i += NT) sA[i * kRowStride + 3] = 0.f;

  float V[K][C1];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < C1; ++c) V[k][c] = 0.f;

  const CT *cbase = cost + (size_t)(l_first + k0) * HW;

  for (int s = Y0 - r; s < Y1 + r; ++s) {
    // ---- phase A: vertical running sums over input rows [s-2r, s]
    if (col_ok) {
      if (s >= 0 && s < H) {
        const size_t pix = (size_t)s * W + xi;
        float g[NG];
#pragma unroll
        for (int i = 0; i < NG; ++i) g[i] = __ldg(G + (size_t)i * HW + pix);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (k < nk) {
            const float p = load_cost(cbase, (size_t)k * HW + pix);
            V[k][0] += p;
#pragma unroll
            for (int i = 0; i < NG; ++i) V[k][i + 1] = fmaf(g[i], p, V[k][i + 1]);
          }
        }
      }
      const int so = s - 2 * r - 1;
      if (so >= add_lo) {
        const size_t pix = (size_t)so * W + xi;
        float g[NG];
#pragma unroll
        for (int i = 0; i < NG; ++i) g[i] = __ldg(G + (size_t)i * HW + pix);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (k < nk) {
            const float p = load_cost(cbase, (size_t)k * HW + pix);
            V[k][0] -= p;
#pragma unroll
            for (int i = 0; i < NG; ++i) V[k][i + 1] = fmaf(-g[i], p, V[k][i + 1]);
          }
        }
      }
    }
    const int y1 = s - r;
    if (y1 < Y0) continue;  // warm-up rows: no coefficient row complete yet (uniform per CTA)

    // ---- phase B: horizontal window sums via inclusive prefix scans
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < C1; ++c) sA[(k * C1 + c) * kRowStride + 4 + t] = V[k][c];
    __syncthreads();
    scan_rows(sA, nk * C1);
    __syncthreads();

    // ---- phase C: coefficients at (x0 + t, y1)
    const int x = x0 + t;
    if (t < TW && x < W) {
      const size_t pix = (size_t)y1 * W + x;
      const float invN = 1.f / (float)(clipped_count(x, r, W) * clipped_count(y1, r, H));
      float m[NG];
#pragma unroll
      for (int i = 0; i < NG; ++i) m[i] = __ldg(mu + (size_t)i * HW + pix);
      float cov[K][NG], a[K][NG], pbar[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float *row = sA + k * C1 * kRowStride;
        pbar[k] = (row[4 + t + 2 * r] - row[3 + t]) * invN;
#pragma unroll
        for (int i = 0; i < NG; ++i) {
          const float *ri = row + (i + 1) * kRowStride;
          const float mi = (ri[4 + t + 2 * r] - ri[3 + t]) * invN;
          cov[k][i] = fmaf(-m[i], pbar[k], mi);
          a[k][i] = 0.f;
        }
      }
#pragma unroll
      for (int i = 0; i < NG; ++i) {
#pragma unroll
        for (int j = i; j < NG; ++j) {
          const float Mij = __ldg(minv + (size_t)tri_index(NG, i, j) * HW + pix);
#pragma unroll
          for (int k = 0; k < K; ++k) {
            a[k][i] = fmaf(Mij, cov[k][j], a[k][i]);
            if (j != i) a[k][j] = fmaf(Mij, cov[k][i], a[k][j]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (k < nk) {
          float b = pbar[k];
#pragma unroll
          for (int i = 0; i < NG; ++i) b = fmaf(-a[k][i], m[i], b);
          float *dst = coef + (size_t)(k0 + k) * C1 * HW + pix;
          dst[0] = b;
#pragma unroll
          for (int i = 0; i < NG; ++i) dst[(size_t)(i + 1) * HW] = a[k][i];
        }
      }
    }
    __syncthreads();
  }
}

template <int NG, int K>
__global__ void __launch_bounds__(NT) k_apply(const float *__restrict__ coef, int H, int W, int r,
                                              const float *__restrict__ G,
                                              unsigned long long *__restrict__ keys,
                                              float *__restrict__ filtered, int l_first,
                                              int n_chunk, int band_rows) {
  constexpr int C1 = NG + 1;
  __shared__ __align__(16) float sA[K * C1 * kRowStride];
  const size_t HW = (size_t)H * W;
  const int t = threadIdx.x;
  const int TW = NT - 2 * r;
  const int x0 = blockIdx.x * TW;
  const int xc = x0 - r + t;
  const bool col_ok = xc >= 0 && xc < W;
  const int Y0 = blockIdx.y * band_rows;
  const int Y1 = min(H, Y0 + band_rows);
  const int k0 = blockIdx.z * K;
  const int nk = min(K, n_chunk - k0);
  const int add_lo = max(0, Y0 - r);

  for (int i = t; i < K * C1; i += NT) sA[i * kRowStride + 3] = 0.f;

  float V[K][C1];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < C1; ++c) V[k][c] = 0.f;

  const float *cb = coef + (size_t)k0 * C1 * HW;

  for (int s = Y0 - r; s < Y1 + r; ++s) {
    if (col_ok) {
      if (s >= 0 && s < H) {
        const size_t pix = (size_t)s * W + xc;
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (k < nk) {
#pragma unroll
            for (int c = 0; c < C1; ++c) V[k][c] += __ldg(cb + (size_t)(k * C1 + c) * HW + pix);
          }
      }
      const int so = s - 2 * r - 1;
      if (so >= add_lo) {
        const size_t pix = (size_t)so * W + xc;
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (k < nk) {
#pragma unroll
            for (int c = 0; c < C1; ++c) V[k][c] -= __ldg(cb + (size_t)(k * C1 + c) * HW + pix);
          }
      }
    }
    const int y2 = s - r;
    if (y2 < Y0) continue;

#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < C1; ++c) sA[(k * C1 + c) * kRowStride + 4 + t] = V[k][c];
    __syncthreads();
    scan_rows(sA, nk * C1);
    __syncthreads();

    const int x = x0 + t;
    if (t < TW && x < W) {
      const size_t pix = (size_t)y2 * W + x;
      const float invN = 1.f / (float)(clipped_count(x, r, W) * clipped_count(y2, r, H));
      float g[NG];
#pragma unroll
      for (int i = 0; i < NG; ++i) g[i] = __ldg(G + (size_t)i * HW + pix);
      float qbest = 0.f;
      int kbest = -1;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (k < nk) {
          const float *row = sA + k * C1 * kRowStride;
          float q = row[4 + t + 2 * r] - row[3 + t];
#pragma unroll
          for (int i = 0; i < NG; ++i) {
            const float *ri = row + (i + 1) * kRowStride;
            q = fmaf(ri[4 + t + 2 * r] - ri[3 + t], g[i], q);
          }
          q *= invN;
          if (filtered) filtered[(size_t)(l_first + k0 + k) * HW + pix] = q;
          const float qk = (q != q) ? __int_as_float(0x7f800000) : q;
          if (kbest < 0 || qk < qbest) {
            qbest = qk;
            kbest = k;
          }
        }
      }
      if (keys) atomicMin(keys + pix, wta_key(qbest, l_first + k0 + kbest));
    }
    __syncthreads();
  }
}

__global__ void k_wta_finalize(const unsigned long long *__restrict__ keys, int HW,
                               int32_t *__restrict__ labels, float *__restrict__ best) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW) return;
  unsigned long long key = keys[p];
  if (labels) labels[p] = (int32_t)(unsigned int)(key & 0xffffffffull);
  if (best) best[p] = wta_key_value(key);
}

// Standalone WTA over a filtered volume: one thread per pixel scanning the labels in order.
__global__ void k_wta_volume(const float *__restrict__ q, int L, int HW,
                             int32_t *__restrict__ labels, float *__restrict__ best) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW) return;
  float b = 0.f;
  int lb = 0;
  for (int l = 0; l < L; ++l) {
    float v = q[(size_t)l * HW + p];
    if (v != v) v = __int_as_float(0x7f800000);
    if (l == 0 || v < b) {
      b = v;
      lb = l;
    }
  }
  if (labels) labels[p] = lb;
  if (best) best[p] = b;
}

template <int NG, int K>
cudaError_t launch_chunk(const hgf_guidance *g, const void *cost, int cost_dtype, int l_first,
                         int nc, float *filtered, float *coef_ws, unsigned long long *keys,
                         int band_rows, cudaStream_t s, Profiler *prof) {
  const int H = g->H, W = g->W, r = g->r;
  const int TW = NT - 2 * r;
  dim3 grid((W + TW - 1) / TW, (H + band_rows - 1) / band_rows, (nc + K - 1) / K);
  {
  LaunchScope ls(prof, "k_coef", s);
  switch (cost_dtype) {
    case HGF_F32:
      k_coef<NG, K, float><<<grid, NT, 0, s>>>((const float *)cost, H, W, r, g->G, g->minv, g->mu,
                                               coef_ws, l_first, nc, band_rows);
      break;
    case HGF_BF16:
      k_coef<NG, K, __nv_bfloat16><<<grid, NT, 0, s>>>((const __nv_bfloat16 *)cost, H, W, r,
                                                       g->G, g->minv, g->mu, coef_ws, l_first,
                                                       nc, band_rows);
      break;
    case HGF_F16:
      k_coef<NG, K, __half><<<grid, NT, 0, s>>>((const __half *)cost, H, W, r, g->G, g->minv,
                                                g->mu, coef_ws, l_first, nc, band_rows);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  }
  {
    LaunchScope ls(prof, "k_apply", s);
    k_apply<NG, K><<<grid, NT, 0, s>>>(coef_ws, H, W, r, g->G, keys, filtered, l_first, nc,
                                       band_rows);
  }
  return cudaGetLastError();
}

}  // namespace

bool aggregate_supported(int n) {
  switch (n) {
    case 1: case 2: case 3: case 4: case 5: case 6: case 7: case 8: case 9: case 19:
      return true;
    default:
      return false;
  }
}

static int labels_per_pass_for(int n) { return n >= 19 ? 2 : 4; }

AggregatePlan plan_aggregate(const hgf_guidance *g, int L, const hgf_tuning &t, int num_sms) {
  AggregatePlan p;
  p.K = labels_per_pass_for(g->n);
  const size_t plane = (size_t)(g->n + 1) * g->H * g->W * sizeof(float);
  // labels per chunk: all labels while the coefficient workspace stays under 4 GiB
  size_t cap = std::max<size_t>(1, ((size_t)4 << 30) / plane);
  p.chunk = t.chunk_labels > 0 ? t.chunk_labels : (int)std::min<size_t>((size_t)L, cap);
  p.chunk = std::max(1, std::min(p.chunk, L));
  const int TW = NT - 2 * g->r;
  const int strips = (g->W + TW - 1) / TW;
  const int passes = (p.chunk + p.K - 1) / p.K;
  if (t.band_rows > 0) {
    p.band_rows = t.band_rows;
  } else {
    // about 2 CTAs per SM, but bands of at least 4r rows so the warm-up rows stay a fraction
    const int target = 2 * std::max(1, num_sms);
    int bands = std::max(1, (target + strips * passes - 1) / (strips * passes));
    int rows = (g->H + bands - 1) / bands;
    p.band_rows = std::max(rows, std::min(g->H, std::max(16, 4 * g->r)));
  }
  return p;
}

size_t aggregate_coef_bytes(const hgf_guidance *g, const AggregatePlan &p) {
  return (size_t)p.chunk * (g->n + 1) * g->H * g->W * sizeof(float);
}

template <int NG>
static cudaError_t run_chunks(const hgf_guidance *g, const void *cost, int cost_dtype, int L,
                              float *filtered, float *coef_ws, unsigned long long *keys,
                              const AggregatePlan &p, cudaStream_t s, Profiler *prof) {
  for (int l0 = 0; l0 < L; l0 += p.chunk) {
    int nc = std::min(p.chunk, L - l0);
    cudaError_t e;
    if (p.K == 4)
      e = launch_chunk<NG, 4>(g, cost, cost_dtype, l0, nc, filtered, coef_ws, keys, p.band_rows,
                              s, prof);
    else if (p.K == 2)
      e = launch_chunk<NG, 2>(g, cost, cost_dtype, l0, nc, filtered, coef_ws, keys, p.band_rows,
                              s, prof);
    else
      e = launch_chunk<NG, 1>(g, cost, cost_dtype, l0, nc, filtered, coef_ws, keys, p.band_rows,
                              s, prof);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_aggregate(const hgf_guidance *g, const void *cost, int cost_dtype, int L,
                             float *filtered, int32_t *labels, float *best, float *coef_ws,
                             unsigned long long *keys, const AggregatePlan &p, cudaStream_t s,
                             Profiler *prof) {
  const int HW = g->H * g->W;
  const bool want_wta = labels || best;
  unsigned long long *k = want_wta ? keys : nullptr;
  if (k) {
    cudaError_t e = cudaMemsetAsync(k, 0xff, (size_t)HW * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e;
  switch (g->n) {
#define HGF_AGG_CASE(N)                                                                   \
  case N:                                                                                 \
    e = run_chunks<N>(g, cost, cost_dtype, L, filtered, coef_ws, k, p, s, prof);          \
    break;
    HGF_AGG_CASE(1) HGF_AGG_CASE(2) HGF_AGG_CASE(3) HGF_AGG_CASE(4) HGF_AGG_CASE(5)
    HGF_AGG_CASE(6) HGF_AGG_CASE(7) HGF_AGG_CASE(8) HGF_AGG_CASE(9) HGF_AGG_CASE(19)
#undef HGF_AGG_CASE
    default:
      return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  if (k) {
    LaunchScope ls(prof, "k_wta_finalize", s);
    k_wta_finalize<<<(HW + 255) / 256, 256, 0, s>>>(k, HW, labels, best);
  }
  return cudaGetLastError();
}

cudaError_t launch_wta(const float *filtered, int L, int H, int W, int32_t *labels, float *best,
                       cudaStream_t s, Profiler *prof) {
  int HW = H * W;
  LaunchScope ls(prof, "k_wta_volume", s);
  k_wta_volume<<<(HW + 255) / 256, 256, 0, s>>>(filtered, L, HW, labels, best);
  return cudaGetLastError();
}

}  // namespace hgf
