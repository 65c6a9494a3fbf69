// Fused multi-label aggregation + WTA (Sec. 1 pipeline with the centred form of Sec. 5.1 and the
// multipoint aggregation of Sec. 4.1, Eq. HGF_z1).
//
// Two streaming kernels per chunk of labels, both over vertical strips of the image (128 columns
// per CTA, one thread per column, 2r of them halo) that walk down a band of rows:
//   k_coef : vertical running sums of (p, G_1 p, .., G_n p) for K labels, horizontal window sums
//            by prefix scans in shared memory, then per coefficient pixel
//            cov = A(G p) - mu A(p), a = Minv cov, b = A(p) - a.mu, written to the workspace.
//            The guidance G is recomputed from the input image (constant-index monomials).
//   k_apply: vertical running sums of (b, a_1..a_n), horizontal window sums,
//            q = sum_i A(a_i) G_i + A(b), and one packed 64-bit atomicMin per pixel (cost in the
//            high word, label in the low word: lowest cost, then lowest label).
// Every input row is read from device memory once: each thread keeps its column's last 2r+1 rows
// in a private shared-memory ring (the row leaving the vertical window is subtracted from there)
// and loads rows two steps ahead into registers, so the load latency overlaps two steps of work.
// Windows are clipped at the image border: samples outside the image never enter a sum and the
// means divide by the in-image count N(x, y).
#include "hgf_basis.cuh"

#include <algorithm>

namespace hgf {

namespace {

constexpr int NT = kStripThreads;
constexpr int kRowStride = NT + 4;  // [0..3] padding (index 3 holds the zero prefix), 4+t values

// Inclusive prefix sums along each shared row (values at [4 .. 4+NT)), one warp per row; two
// rows per iteration with both loads issued first so that their shuffle chains overlap.
__device__ __forceinline__ void scan4(float4 &v, int lane) {
  v.y += v.x;
  v.z += v.y;
  v.w += v.z;
  float tot = v.w;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    float o = __shfl_up_sync(0xffffffffu, tot, off);
    if (lane >= off) tot += o;
  }
  const float ex = tot - v.w;
  v.x += ex;
  v.y += ex;
  v.z += ex;
  v.w += ex;
}

__device__ __forceinline__ void scan_rows(float *sA, int rows) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  int row = warp;
  for (; row + NW < rows; row += 2 * NW) {
    float4 *p0 = reinterpret_cast<float4 *>(sA + row * kRowStride + 4) + lane;
    float4 *p1 = reinterpret_cast<float4 *>(sA + (row + NW) * kRowStride + 4) + lane;
    float4 v0 = *p0, v1 = *p1;
    scan4(v0, lane);
    scan4(v1, lane);
    *p0 = v0;
    *p1 = v1;
  }
  if (row < rows) {
    float4 *p0 = reinterpret_cast<float4 *>(sA + row * kRowStride + 4) + lane;
    float4 v0 = *p0;
    scan4(v0, lane);
    *p0 = v0;
  }
}

// Window sum [t, t + 2r] of a scanned shared row.
__device__ __forceinline__ float window(const float *row, int t, int r) {
  return row[4 + t + 2 * r] - row[3 + t];
}

template <int B, int K>
constexpr size_t coef_smem_bytes(int r) {
  return sizeof(float) * ((size_t)2 * K * (basis_n(B) + 1) * kRowStride +
                          (size_t)(2 * r + 1) * (basis_channels_in(B) + K) * NT);
}

template <int B, int K, typename CT>
__global__ void __launch_bounds__(NT) k_coef(const CT *__restrict__ cost, int H, int W, int r,
                                             const float *__restrict__ img,
                                             const float *__restrict__ shift,
                                             const float *__restrict__ rec,
                                             float *__restrict__ coef, int l_first, int n_chunk,
                                             int band_rows) {
  constexpr int NG = basis_n(B), C1 = NG + 1, NC = basis_channels_in(B), RAW = NC + K;
  constexpr int P = NG * (NG + 1) / 2;
  constexpr int REC = record_floats(NG), CP = coef_floats(NG);
#ifndef HGF_EARLY_RECORD_FLOATS
#define HGF_EARLY_RECORD_FLOATS 68
#endif
  constexpr bool EARLY = REC <= HGF_EARLY_RECORD_FLOATS;  // record held in registers over the scans
  extern __shared__ __align__(16) float smem[];
  // two scan buffers used on alternate rows: a warp may start the next row's vertical update
  // while others still read this row's window sums, so no barrier is needed at the end of a row
  float *sA0 = smem;
  float *ring = smem + 2 * K * C1 * kRowStride;  // [2r+1][RAW][NT], thread-private columns
  const int R = 2 * r + 1;
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
  const int s_begin = Y0 - r, s_end = Y1 + r;

  for (int i = t; i < 2 * K * C1; i += NT) sA0[i * kRowStride + 3] = 0.f;
  float sh[NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) sh[i] = __ldg(shift + i);

  const CT *cbase = cost + (size_t)(l_first + k0) * HW;
  auto load_row = [&](int row, float *v) {
    if (col_ok && row >= 0 && row < H) {
      const size_t pix = (size_t)row * W + xi;
#pragma unroll
      for (int c = 0; c < NC; ++c) v[c] = __ldg(img + (size_t)c * HW + pix);
#pragma unroll
      for (int k = 0; k < K; ++k)
        v[NC + k] = k < nk ? load_cost(cbase, (size_t)k * HW + pix) : 0.f;
    }
  };
  float pa[RAW], pb[RAW], pc[RAW];
#pragma unroll
  for (int c = 0; c < RAW; ++c) pa[c] = pb[c] = pc[c] = 0.f;
  load_row(s_begin, pa);
  load_row(s_begin + 1, pb);

  float V[K][C1];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < C1; ++c) V[k][c] = 0.f;

  // One step per input row s: `cur` holds row s (loaded two steps earlier) and row s + 2 is
  // loaded into `nxt`. The loop is unrolled three times so that the three buffers rotate roles
  // without register copies (a copy would wait for the load it copies).
  auto step = [&](const int s, const float *cur, float *nxt) {
    if (s >= s_end) return;
    load_row(s + 2, nxt);
    const int y1 = s - r;
    const int x = x0 + t;
    const bool coef_here = y1 >= Y0 && t < TW && x < W;
    // per-pixel record [mu | packed Minv]: issued now, used after the scans so that the load
    // latency overlaps phases A and B (when it fits in registers)
    float Rg[EARLY ? REC : 4];
    const float4 *rp = reinterpret_cast<const float4 *>(rec + ((size_t)y1 * W + x) * REC);
    if (coef_here && EARLY) {
#pragma unroll
      for (int q = 0; q < (EARLY ? REC : 4) / 4; ++q) {
        const float4 v = __ldg(rp + q);
        Rg[4 * q] = v.x;
        Rg[4 * q + 1] = v.y;
        Rg[4 * q + 2] = v.z;
        Rg[4 * q + 3] = v.w;
      }
    }
    // ---- phase A: vertical running sums over input rows [s-2r, s]
    if (col_ok) {
      float *slot = ring + (size_t)(((s - s_begin) % R) * RAW) * NT + t;
      const int so = s - 2 * r - 1;
      if (so >= add_lo) {  // the outgoing row occupies the slot the new row will take
        float xo[NC], go[NG];
#pragma unroll
        for (int c = 0; c < NC; ++c) xo[c] = slot[c * NT];
        eval_basis<B>(xo, sh, go);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float p = slot[(NC + k) * NT];
          V[k][0] -= p;
#pragma unroll
          for (int i = 0; i < NG; ++i) V[k][i + 1] = fmaf(-go[i], p, V[k][i + 1]);
        }
      }
      if (s >= 0 && s < H) {
        float g[NG];
        eval_basis<B>(cur, sh, g);
#pragma unroll
        for (int c = 0; c < RAW; ++c) slot[c * NT] = cur[c];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float p = cur[NC + k];
          V[k][0] += p;
#pragma unroll
          for (int i = 0; i < NG; ++i) V[k][i + 1] = fmaf(g[i], p, V[k][i + 1]);
        }
      }
    }
    if (y1 < Y0) return;  // warm-up rows: no coefficient row complete yet (uniform per CTA)
    float *sA = sA0 + ((y1 - Y0) & 1) * K * C1 * kRowStride;

    // ---- phase B: horizontal window sums via inclusive prefix scans
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < C1; ++c) sA[(k * C1 + c) * kRowStride + 4 + t] = V[k][c];
    __syncthreads();
    scan_rows(sA, nk * C1);
    __syncthreads();

    // ---- phase C: coefficients at (x, y1)
    if (coef_here) {
      const size_t pix = (size_t)y1 * W + x;
      const float invN = 1.f / (float)(clipped_count(x, r, W) * clipped_count(y1, r, H));
      auto recv = [&](int e) -> float {
        return EARLY ? Rg[EARLY ? e : 0] : __ldg(rec + pix * REC + e);
      };
      float m[NG];
#pragma unroll
      for (int i = 0; i < NG; ++i) m[i] = recv(i);
      float cov[K][NG], a[K][NG], pbar[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float *row = sA + k * C1 * kRowStride;
        pbar[k] = window(row, t, r) * invN;
#pragma unroll
        for (int i = 0; i < NG; ++i) {
          const float mi = window(row + (i + 1) * kRowStride, t, r) * invN;
          cov[k][i] = fmaf(-m[i], pbar[k], mi);
          a[k][i] = 0.f;
        }
      }
#pragma unroll
      for (int i = 0; i < NG; ++i) {
#pragma unroll
        for (int j = i; j < NG; ++j) {
          const float Mij = recv(NG + tri_index(NG, i, j));
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
          float o[CP];
          o[0] = b;
#pragma unroll
          for (int i = 0; i < NG; ++i) o[i + 1] = a[k][i];
#pragma unroll
          for (int i = C1; i < CP; ++i) o[i] = 0.f;
          float2 *dst = reinterpret_cast<float2 *>(coef + ((size_t)(k0 + k) * HW + pix) * CP);
#pragma unroll
          for (int q = 0; q < CP / 2; ++q) dst[q] = make_float2(o[2 * q], o[2 * q + 1]);
        }
      }
    }
  };
  for (int s = s_begin; s < s_end; s += 3) {
    step(s, pa, pc);
    step(s + 1, pb, pa);
    step(s + 2, pc, pb);
  }
}

template <int B, bool RING>
constexpr size_t apply_smem_bytes(int r) {
  return sizeof(float) * ((size_t)2 * (basis_n(B) + 1) * kRowStride +
                          (RING ? (size_t)(2 * r + 1) * (basis_n(B) + 1) * NT : 0));
}

// One label per CTA. RING: the outgoing coefficient row comes from the thread's shared-memory
// ring; otherwise it is reloaded from device memory (used when the ring does not fit).
template <int B, bool RING>
__global__ void __launch_bounds__(NT) k_apply(const float *__restrict__ coef, int H, int W, int r,
                                              const float *__restrict__ img,
                                              const float *__restrict__ shift,
                                              unsigned long long *__restrict__ keys,
                                              float *__restrict__ filtered, int l_first,
                                              int band_rows) {
  constexpr int NG = basis_n(B), C1 = NG + 1, NC = basis_channels_in(B), CP = coef_floats(NG);
  extern __shared__ __align__(16) float smem[];
  float *sA0 = smem;                         // two scan buffers, alternate rows (see k_coef)
  float *ring = smem + 2 * C1 * kRowStride;  // [2r+1][C1][NT]
  const int R = 2 * r + 1;
  const size_t HW = (size_t)H * W;
  const int t = threadIdx.x;
  const int TW = NT - 2 * r;
  const int x0 = blockIdx.x * TW;
  const int xc = x0 - r + t;
  const bool col_ok = xc >= 0 && xc < W;
  const int Y0 = blockIdx.y * band_rows;
  const int Y1 = min(H, Y0 + band_rows);
  const int k = blockIdx.z;
  const int add_lo = max(0, Y0 - r);
  const int s_begin = Y0 - r, s_end = Y1 + r;

  if (t < 2 * C1) sA0[t * kRowStride + 3] = 0.f;
  float sh[NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) sh[i] = __ldg(shift + i);
  const float *cb = coef + (size_t)k * HW * CP;
  auto load_row = [&](int row, float *v) {
    if (col_ok && row >= 0 && row < H) {
      const float2 *src = reinterpret_cast<const float2 *>(cb + ((size_t)row * W + xc) * CP);
#pragma unroll
      for (int q = 0; q < CP / 2; ++q) {
        const float2 u = __ldg(src + q);
        if (2 * q < C1) v[2 * q] = u.x;
        if (2 * q + 1 < C1) v[2 * q + 1] = u.y;
      }
    }
  };
  // outgoing rows (only without the ring): row `row` if it entered this band's window
  auto load_old = [&](int row, float *v) {
    if (!RING && row >= add_lo) load_row(row, v);
  };
  float pa[C1], pb[C1], pc[C1];
  float oa[RING ? 1 : C1], ob[RING ? 1 : C1], oc[RING ? 1 : C1];
#pragma unroll
  for (int c = 0; c < C1; ++c) pa[c] = pb[c] = pc[c] = 0.f;
#pragma unroll
  for (int c = 0; c < (RING ? 1 : C1); ++c) oa[c] = ob[c] = oc[c] = 0.f;
  load_row(s_begin, pa);
  load_row(s_begin + 1, pb);
  load_old(s_begin - 2 * r - 1, oa);
  load_old(s_begin + 1 - 2 * r - 1, ob);
  float V[C1];
#pragma unroll
  for (int c = 0; c < C1; ++c) V[c] = 0.f;

  // Same three-buffer rotation as k_coef; without the ring, the outgoing row (2r+1 rows back,
  // resident in L2) is prefetched two steps ahead as well.
  auto step = [&](const int s, const float *cur, float *nxt, const float *cur_o, float *nxt_o) {
    if (s >= s_end) return;
    load_row(s + 2, nxt);
    if (!RING) load_old(s + 2 - 2 * r - 1, nxt_o);
    const int y2 = s - r;
    const int x = x0 + t;
    const bool out_here = y2 >= Y0 && t < TW && x < W;
    float xin[NC];
    if (out_here) {
      const size_t pix = (size_t)y2 * W + x;
#pragma unroll
      for (int c = 0; c < NC; ++c) xin[c] = __ldg(img + (size_t)c * HW + pix);
    }
    if (col_ok) {
      const int so = s - 2 * r - 1;
      if (RING) {
        float *slot = ring + (size_t)(((s - s_begin) % R) * C1) * NT + t;
        if (so >= add_lo) {
#pragma unroll
          for (int c = 0; c < C1; ++c) V[c] -= slot[c * NT];
        }
        if (s >= 0 && s < H) {
#pragma unroll
          for (int c = 0; c < C1; ++c) {
            V[c] += cur[c];
            slot[c * NT] = cur[c];
          }
        }
      } else {
        if (so >= add_lo) {
#pragma unroll
          for (int c = 0; c < C1; ++c) V[c] -= cur_o[c];
        }
        if (s >= 0 && s < H) {
#pragma unroll
          for (int c = 0; c < C1; ++c) V[c] += cur[c];
        }
      }
    }
    if (y2 < Y0) return;
    float *sA = sA0 + ((y2 - Y0) & 1) * C1 * kRowStride;

#pragma unroll
    for (int c = 0; c < C1; ++c) sA[c * kRowStride + 4 + t] = V[c];
    __syncthreads();
    scan_rows(sA, C1);
    __syncthreads();

    if (out_here) {
      const size_t pix = (size_t)y2 * W + x;
      const float invN = 1.f / (float)(clipped_count(x, r, W) * clipped_count(y2, r, H));
      float g[NG];
      eval_basis<B>(xin, sh, g);
      float q = window(sA, t, r);
#pragma unroll
      for (int i = 0; i < NG; ++i) q = fmaf(window(sA + (i + 1) * kRowStride, t, r), g[i], q);
      q *= invN;
      const int label = l_first + k;
      if (filtered) filtered[(size_t)label * HW + pix] = q;
      if (keys) atomicMin(keys + pix, wta_key(q, label));
    }
  };
  for (int s = s_begin; s < s_end; s += 3) {
    step(s, pa, pc, oa, oc);
    step(s + 1, pb, pa, ob, oa);
    step(s + 2, pc, pb, oc, ob);
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

template <typename Kern>
cudaError_t set_smem(Kern k, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Rows per band for a kernel whose grid is strips x bands x slabs: the band count that minimises
// (waves of resident CTAs) x (rows streamed per CTA, including the 2r warm-up rows). Callers pass
// a nominal slab count that depends on the shape only (not on how many labels a call or chunk
// has): the band boundaries decide the order of the running sums, so results are then identical
// whether an image is aggregated alone, in a batch, in the serving loop or in label chunks.
static int choose_band_rows(int H, int r, long long strips_slabs, int resident) {
  long long best_cost = -1;
  int best = H;
  for (int bands = 1; bands <= std::max(1, H / std::max(8, 2 * r)); ++bands) {
    const int rows = (H + bands - 1) / bands;
    const long long ctas = strips_slabs * ((H + rows - 1) / rows);
    const long long waves = (ctas + resident - 1) / resident;
    const long long cost = waves * (rows + 2 * r);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = rows;
    }
  }
  return best;
}

constexpr int kNominalLabels = 64;  // label count the band heights are planned for

template <typename Kern>
static int resident_ctas(Kern k, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  return std::max(1, per_sm) * std::max(1, sms);
}

template <int B, int K>
cudaError_t launch_chunk(const hgf_guidance *g, const void *cost, int cost_dtype, int l_first,
                         int nc, float *filtered, float *coef_ws, unsigned long long *keys,
                         int band_rows, bool apply_ring, cudaStream_t s, Profiler *prof) {
  const int H = g->H, W = g->W, r = g->r;
  const int TW = NT - 2 * r;
  const unsigned strips = (W + TW - 1) / TW;
  cudaError_t e;
  {
    const size_t sm = coef_smem_bytes<B, K>(r);
    // the shared-memory limit is raised before the occupancy query so that every call (the
    // first included) plans the same bands
    e = set_smem(k_coef<B, K, float>, sm);
    if (e == cudaSuccess) e = set_smem(k_coef<B, K, __nv_bfloat16>, sm);
    if (e == cudaSuccess) e = set_smem(k_coef<B, K, __half>, sm);
    if (e != cudaSuccess) return e;
    const int passes = (nc + K - 1) / K;
    // bands planned for the two-label kernel whatever K is, so that K never changes a result
    const size_t sm2 = coef_smem_bytes<B, 2>(r);
    e = set_smem(k_coef<B, 2, float>, sm2);
    if (e != cudaSuccess) return e;
    const int rows = band_rows > 0 ? band_rows
                                   : choose_band_rows(H, r, (long long)strips * (kNominalLabels / 2),
                                                      resident_ctas(k_coef<B, 2, float>, sm2));
    dim3 grid(strips, (H + rows - 1) / rows, passes);
    LaunchScope ls(prof, "k_coef", s);
#define HGF_COEF(CT)                                                                          \
  k_coef<B, K, CT><<<grid, NT, sm, s>>>((const CT *)cost, H, W, r, g->img, g->shift, g->rec,  \
                                        coef_ws, l_first, nc, rows);
    switch (cost_dtype) {
      case HGF_F32: HGF_COEF(float) break;
      case HGF_BF16: HGF_COEF(__nv_bfloat16) break;
      case HGF_F16: HGF_COEF(__half) break;
      default: return cudaErrorInvalidValue;
    }
#undef HGF_COEF
  }
  {
    LaunchScope ls(prof, "k_apply", s);
    const size_t ring_sm = apply_smem_bytes<B, true>(r);
    if (apply_ring && ring_sm <= 227 * 1024) {
      e = set_smem(k_apply<B, true>, ring_sm);
      if (e != cudaSuccess) return e;
      const int rows = band_rows > 0 ? band_rows
                                     : choose_band_rows(H, r, (long long)strips * kNominalLabels,
                                                        resident_ctas(k_apply<B, true>, ring_sm));
      dim3 grid(strips, (H + rows - 1) / rows, nc);
      k_apply<B, true><<<grid, NT, ring_sm, s>>>(coef_ws, H, W, r, g->img, g->shift, keys,
                                                 filtered, l_first, rows);
    } else {
      const size_t sm = apply_smem_bytes<B, false>(r);
      e = set_smem(k_apply<B, false>, sm);
      if (e != cudaSuccess) return e;
      const int rows = band_rows > 0 ? band_rows
                                     : choose_band_rows(H, r, (long long)strips * kNominalLabels,
                                                        resident_ctas(k_apply<B, false>, sm));
      dim3 grid(strips, (H + rows - 1) / rows, nc);
      k_apply<B, false><<<grid, NT, sm, s>>>(coef_ws, H, W, r, g->img, g->shift, keys, filtered,
                                             l_first, rows);
    }
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

// Dynamic shared memory of k_coef for n guidance channels, C input channels, K labels, radius r.
static size_t coef_smem(int n, int C, int K, int r) {
  return sizeof(float) *
         ((size_t)2 * K * (n + 1) * kRowStride + (size_t)(2 * r + 1) * (C + K) * NT);
}

bool aggregate_fits(const hgf_guidance *g) {
  return 2 * g->r + 1 < NT && coef_smem(g->n, g->C, 2, g->r) <= 227 * 1024;
}

AggregatePlan plan_aggregate(const hgf_guidance *g, int L, const hgf_tuning &t, int num_sms) {
  AggregatePlan p;
  // four labels per pass on large images (1400x1100, n = 9: 18.3 vs 22.5 ms), two on small ones
  // (450x375, n = 9: 0.51 vs 0.54 ms); four only while two CTAs still fit on an SM. The choice
  // does not change results (each label's arithmetic is the same for any K).
  const bool large = (long long)g->H * g->W >= 500000;
  p.K = (large && g->n < 19 && coef_smem(g->n, g->C, 4, g->r) <= 113 * 1024) ? 4 : 2;
  if (t.labels_per_pass == 1 || t.labels_per_pass == 2 ||
      (t.labels_per_pass == 4 && coef_smem(g->n, g->C, 4, g->r) <= 227 * 1024))
    p.K = t.labels_per_pass;
  const size_t plane = (size_t)coef_floats(g->n) * g->H * g->W * sizeof(float);
  // labels per chunk: all labels while the coefficient workspace stays under 4 GiB
  size_t cap = std::max<size_t>(1, ((size_t)4 << 30) / plane);
  p.chunk = t.chunk_labels > 0 ? t.chunk_labels : (int)std::min<size_t>((size_t)L, cap);
  p.chunk = std::max(1, std::min(p.chunk, L));
  const int TW = NT - 2 * g->r;
  const int strips = (g->W + TW - 1) / TW;
  const int passes = (p.chunk + p.K - 1) / p.K;
  // the outgoing coefficient rows of the output kernel are reloaded by default: they were read
  // 2r+1 steps earlier and are still in L2, and without the ring more CTAs fit on an SM
  const size_t ring = sizeof(float) * (size_t)(g->n + 1) * ((2 * g->r + 1) * NT + 2 * kRowStride);
  p.apply_ring = t.apply_mode == 1 && ring <= 227 * 1024;
  (void)strips;
  (void)passes;
  (void)num_sms;
  p.band_rows = t.band_rows;  // 0: each kernel picks its bands from its occupancy at launch
  return p;
}

size_t aggregate_coef_bytes(const hgf_guidance *g, const AggregatePlan &p) {
  return (size_t)p.chunk * coef_floats(g->n) * g->H * g->W * sizeof(float);
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
  const int b = basis_id(g->C, g->degree, g->basis);
  cudaError_t e = cudaErrorInvalidValue;
  bool ok = dispatch_basis(b, [&](auto bc) {
    constexpr int B = decltype(bc)::value;
    e = cudaSuccess;
    for (int l0 = 0; l0 < L && e == cudaSuccess; l0 += p.chunk) {
      const int nc = std::min(p.chunk, L - l0);
      if (p.K == 4)
        e = launch_chunk<B, 4>(g, cost, cost_dtype, l0, nc, filtered, coef_ws, k, p.band_rows,
                               p.apply_ring, s, prof);
      else if (p.K == 1)
        e = launch_chunk<B, 1>(g, cost, cost_dtype, l0, nc, filtered, coef_ws, k, p.band_rows,
                               p.apply_ring, s, prof);
      else
        e = launch_chunk<B, 2>(g, cost, cost_dtype, l0, nc, filtered, coef_ws, k, p.band_rows,
                               p.apply_ring, s, prof);
    }
  });
  if (!ok) return cudaErrorInvalidValue;
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
