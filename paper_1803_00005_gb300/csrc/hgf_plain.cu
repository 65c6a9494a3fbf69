// Plain form of the aggregation + WTA: one kernel per step of the centred guided filter
// (Sec. 5.1) and the multipoint aggregation (Sec. 4.1), every intermediate plane in device
// memory, direct (2r+1)-term window sums per axis. It computes the same quantities as the fused
// path and serves as its comparison baseline. Labels are processed in chunks so that the two
// intermediate buffers stay bounded.
#include "hgf_internal.cuh"

#include <algorithm>

namespace hgf {

namespace {

template <typename CT>
__global__ void p_products(const CT *__restrict__ cost, const float *__restrict__ G, int n,
                           int HW, int l0, int Lp, float *__restrict__ X) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)Lp * HW) return;
  int k = (int)(idx / HW);
  size_t p = idx - (size_t)k * HW;
  float v = load_cost(cost, (size_t)(l0 + k) * HW + p);
  float *dst = X + (size_t)k * (n + 1) * HW + p;
  dst[0] = v;
  for (int i = 0; i < n; ++i) dst[(size_t)(i + 1) * HW] = G[(size_t)i * HW + p] * v;
}

__global__ void p_rowsum(const float *__restrict__ in, size_t planes, int H, int W, int r,
                         float *__restrict__ out) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t HW = (size_t)H * W;
  if (idx >= planes * HW) return;
  int x = (int)(idx % W);
  const float *row = in + (idx - x);
  int lo = max(0, x - r), hi = min(W - 1, x + r);
  float s = 0.f;
  for (int xx = lo; xx <= hi; ++xx) s += row[xx];
  out[idx] = s;
}

__global__ void p_colsum(const float *__restrict__ in, size_t planes, int H, int W, int r,
                         float *__restrict__ out) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t HW = (size_t)H * W;
  if (idx >= planes * HW) return;
  size_t pl = idx / HW;
  size_t rem = idx - pl * HW;
  int y = (int)(rem / W), x = (int)(rem % W);
  const float *col = in + pl * HW + x;
  int lo = max(0, y - r), hi = min(H - 1, y + r);
  float s = 0.f;
  for (int yy = lo; yy <= hi; ++yy) s += col[(size_t)yy * W];
  out[idx] = s;
}

__global__ void p_coef(const float *__restrict__ S, int n, int H, int W, int r,
                       const float *__restrict__ minv, const float *__restrict__ mu, int Lp,
                       float *__restrict__ out) {
  size_t HW = (size_t)H * W;
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)Lp * HW) return;
  int k = (int)(idx / HW);
  size_t p = idx - (size_t)k * HW;
  int y = (int)(p / W), x = (int)(p % W);
  float invN = 1.f / (float)(clipped_count(x, r, W) * clipped_count(y, r, H));
  const float *src = S + (size_t)k * (n + 1) * HW + p;
  float pbar = src[0] * invN;
  float cov[kMaxChannels], a[kMaxChannels];
  for (int i = 0; i < n; ++i) {
    cov[i] = src[(size_t)(i + 1) * HW] * invN - mu[(size_t)i * HW + p] * pbar;
    a[i] = 0.f;
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      int e = i <= j ? tri_index(n, i, j) : tri_index(n, j, i);
      a[i] += minv[(size_t)e * HW + p] * cov[j];
    }
  float b = pbar;
  for (int i = 0; i < n; ++i) b -= a[i] * mu[(size_t)i * HW + p];
  float *dst = out + (size_t)k * (n + 1) * HW + p;
  dst[0] = b;
  for (int i = 0; i < n; ++i) dst[(size_t)(i + 1) * HW] = a[i];
}

__global__ void p_output(const float *__restrict__ S2, const float *__restrict__ G, int n, int H,
                         int W, int r, int Lp, float *__restrict__ q) {
  size_t HW = (size_t)H * W;
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)Lp * HW) return;
  int k = (int)(idx / HW);
  size_t p = idx - (size_t)k * HW;
  int y = (int)(p / W), x = (int)(p % W);
  float invN = 1.f / (float)(clipped_count(x, r, W) * clipped_count(y, r, H));
  const float *src = S2 + (size_t)k * (n + 1) * HW + p;
  float v = src[0] * invN;
  for (int i = 0; i < n; ++i) v += src[(size_t)(i + 1) * HW] * invN * G[(size_t)i * HW + p];
  q[idx] = v;
}

inline unsigned nblk(size_t work) { return (unsigned)((work + 255) / 256); }

}  // namespace

size_t plain_workspace_bytes(const hgf_guidance *g, int L, int *chunk_out) {
  const size_t plane = (size_t)(g->n + 1) * g->H * g->W * sizeof(float);
  size_t cap = std::max<size_t>(1, ((size_t)2 << 30) / plane);
  int chunk = (int)std::min<size_t>((size_t)L, cap);
  if (chunk_out) *chunk_out = chunk;
  return 2 * plane * chunk;
}

cudaError_t launch_aggregate_plain(const hgf_guidance *g, const void *cost, int cost_dtype, int L,
                                   float *q, int32_t *labels, float *best, void *ws, int chunk,
                                   cudaStream_t s, Profiler *prof, float *margin) {
  const int H = g->H, W = g->W, n = g->n, r = g->r;
  const size_t HW = (size_t)H * W;
  if (prof) {
    const int pl[8] = {3, W, W, H, H, 1, chunk, 0};
    for (int i = 0; i < 8; ++i) prof->plan[i] = pl[i];
  }
  float *A = (float *)ws;
  float *B = A + (size_t)chunk * (n + 1) * HW;
  for (int l0 = 0; l0 < L; l0 += chunk) {
    const int Lp = std::min(chunk, L - l0);
    const size_t planes = (size_t)Lp * (n + 1);
    switch (cost_dtype) {
      case HGF_F32:
        {
          LaunchScope ls(prof, "p_products", s);
          p_products<<<nblk(Lp * HW), 256, 0, s>>>((const float *)cost, g->G, n, (int)HW, l0, Lp, A);
        }
        break;
      case HGF_BF16:
        {
          LaunchScope ls(prof, "p_products", s);
          p_products<<<nblk(Lp * HW), 256, 0, s>>>((const __nv_bfloat16 *)cost, g->G, n, (int)HW,
                                                 l0, Lp, A);
        }
        break;
      case HGF_F16:
        {
          LaunchScope ls(prof, "p_products", s);
          p_products<<<nblk(Lp * HW), 256, 0, s>>>((const __half *)cost, g->G, n, (int)HW, l0, Lp,
                                                 A);
        }
        break;
      default:
        return cudaErrorInvalidValue;
    }
    {
      LaunchScope ls(prof, "p_rowsum", s);
      p_rowsum<<<nblk(planes * HW), 256, 0, s>>>(A, planes, H, W, r, B);
    }
    {
      LaunchScope ls(prof, "p_colsum", s);
      p_colsum<<<nblk(planes * HW), 256, 0, s>>>(B, planes, H, W, r, A);
    }
    {
      LaunchScope ls(prof, "p_coef", s);
      p_coef<<<nblk(Lp * HW), 256, 0, s>>>(A, n, H, W, r, g->minv, g->mu, Lp, B);
    }
    {
      LaunchScope ls(prof, "p_rowsum", s);
      p_rowsum<<<nblk(planes * HW), 256, 0, s>>>(B, planes, H, W, r, A);
    }
    {
      LaunchScope ls(prof, "p_colsum", s);
      p_colsum<<<nblk(planes * HW), 256, 0, s>>>(A, planes, H, W, r, B);
    }
    {
      LaunchScope ls(prof, "p_output", s);
      p_output<<<nblk(Lp * HW), 256, 0, s>>>(B, g->G, n, H, W, r, Lp, q + (size_t)l0 * HW);
    }
  }
  if (labels || best || margin) return launch_wta(q, L, H, W, labels, best, s, prof, margin);
  return cudaGetLastError();
}

}  // namespace hgf
