// Guidance precompute: polynomial guidance (Sec. 4.2), window moments (Prop. 2: Gram entries are
// box sums), covariance assembly (Sec. 5.1) and the per-pixel inverse by the Sherman-Morrison
// recursion of Prop. 1 (Sec. 3). Runs once per guidance; the result stays resident.
//
// Numerics: every guidance channel is shifted by c_i, its mean over a fixed sample of pixels
// (k_shifted_guidance), before moments are formed.
// The centred form is exactly invariant to G_i -> G_i - c_i (Sigma, cov and q do not change), and
// the shift shrinks the cancellation in A(G_i G_j) - mu_i mu_j. Window sums are float32 direct
// sums of 2r+1 terms per axis; the assembly Sigma = A(GG^T) - mu mu^T and the recursion run in the
// precision chosen by hgf_params.inv_precision (float64 by default).
#include "hgf_basis.cuh"
#include "hgf_df64.cuh"
#include "hgf_prop1.cuh"
#include "hgf_scan.cuh"

#include <algorithm>

namespace hgf {

bool make_basis_table(int C, int degree, int basis, BasisTable *t) {
  if (C < 1 || C > 3 || degree < 1) return false;
  int n = 0;
  if (basis == HGF_BASIS_POWERS || C == 1) {
    if (degree > kMaxMonomialDegree) return false;
    for (int c = 0; c < C; ++c)
      for (int j = 1; j <= degree; ++j) {
        if (n >= kMaxChannels) return false;
        t->deg[n] = j;
        for (int k = 0; k < j; ++k) t->chan[n][k] = c;
        ++n;
      }
  } else if (basis == HGF_BASIS_MONOMIAL) {
    if (degree > 3) return false;
    // degree-major, then lexicographic multisets c0 <= c1 <= ... (combinations with replacement)
    for (int d = 1; d <= degree; ++d) {
      int idx[3] = {0, 0, 0};
      while (true) {
        if (n >= kMaxChannels) return false;
        t->deg[n] = d;
        for (int k = 0; k < d; ++k) t->chan[n][k] = idx[k];
        ++n;
        int k = d - 1;
        while (k >= 0 && idx[k] == C - 1) --k;
        if (k < 0) break;
        ++idx[k];
        for (int m = k + 1; m < d; ++m) idx[m] = idx[k];
      }
    }
  } else {
    return false;
  }
  t->n = n;
  return true;
}

// ---------------------------------------------------------------------------- guidance synthesis
__global__ void k_make_guidance(const float *__restrict__ img, int C, int HW, BasisTable bt,
                                float *__restrict__ G) {
  size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (p >= (size_t)HW) return;
  float x[3];
  for (int c = 0; c < C; ++c) x[c] = img[(size_t)c * HW + p];
  for (int i = 0; i < bt.n; ++i) {
    float v = x[bt.chan[i][0]];
    for (int k = 1; k < bt.deg[i]; ++k) v *= x[bt.chan[i][k]];
    G[(size_t)i * HW + p] = v;
  }
}

cudaError_t launch_make_guidance(const float *img, int C, int H, int W, const BasisTable &bt,
                                 float *G, cudaStream_t s) {
  int HW = H * W;
  k_make_guidance<<<(HW + 255) / 256, 256, 0, s>>>(img, C, HW, bt, G);
  return cudaGetLastError();
}

// ------------------------------------------------------ shifted guidance (deterministic shift)
// The shift c_i only conditions the float32 moment sums (the centred form is exactly invariant to
// G_i -> G_i - c_i, and the paper form undoes it exactly in float64), so any value near the
// image mean of G_i serves: c_i is the mean of G_i over a fixed sample of kShiftSamples pixels
// spread evenly over the image. Every CTA computes it from the same pixels in the same order (a
// fixed per-thread partial, then a fixed tree over the CTA), so all CTAs get identical values,
// and CTA 0 stores them in `shift`. Then G_i - c_i for the CTA's pixels.
constexpr int kShiftSamples = 1024;
constexpr int kShiftThreads = 256;

template <int B>
__global__ void __launch_bounds__(kShiftThreads) k_shifted_guidance(const float *__restrict__ img,
                                                                    int HW,
                                                                    float *__restrict__ shift,
                                                                    float *__restrict__ G) {
  constexpr int N = basis_n(B), C = basis_channels_in(B);
  constexpr int NW = kShiftThreads / 32;
  __shared__ float red[NW][N];
  __shared__ float sh_s[N];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const float zero[N] = {};
  float acc[N];
#pragma unroll
  for (int i = 0; i < N; ++i) acc[i] = 0.f;
  const int ns = min(kShiftSamples, HW);
#pragma unroll 4
  for (int k = t; k < ns; k += kShiftThreads) {  // the loads of all four samples in flight
    const int p = (int)(((long long)k * HW) / ns);
    float x[C], g[N];
#pragma unroll
    for (int c = 0; c < C; ++c) x[c] = __ldg(img + (size_t)c * HW + p);
    eval_basis<B>(x, zero, g);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] += g[i];
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float v = acc[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  if (t < N) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) v += red[w][t];
    const float c = v / (float)ns;
    sh_s[t] = c;
    if (blockIdx.x == 0) shift[t] = c;
  }
  __syncthreads();
  float sh[N];
#pragma unroll
  for (int i = 0; i < N; ++i) sh[i] = sh_s[i];
  const int p = blockIdx.x * kShiftThreads + t;
  if (p < HW) {
    float x[C], g[N];
#pragma unroll
    for (int c = 0; c < C; ++c) x[c] = __ldg(img + (size_t)c * HW + p);
    eval_basis<B>(x, sh, g);
#pragma unroll
    for (int i = 0; i < N; ++i) G[(size_t)i * HW + p] = g[i];
  }
}

// ------------------------------------------------------------------ moment window sums (strips)
// The window sums of the moment channels for n <= 9: a CTA walks down a band of rows over a
// 128-column strip (one thread per column, 2r halo columns), keeps the vertical window sums of its
// channels in registers (adding the entering row's values, subtracting those of the row leaving
// the window, re-read from L2), and forms the horizontal window sums by prefix scans of shared
// rows. Channel m < n is G_m; m >= n is the pair (i, j), i <= j, of the packed upper triangle.
// The M = n + n(n+1)/2 channels are split into groups of at most kMomentGroup (grid z), so that a
// small image still gives enough CTAs and each thread holds fewer sums.
constexpr int kMomentGroup = 18;

template <int NG, bool COMP, int GRP>
__device__ __forceinline__ void moments_group(const float *__restrict__ G, int H, int W, int r,
                                              int band_rows, float *__restrict__ mom,
                                              float *smem) {
  using namespace strip;
  constexpr int M = NG + NG * (NG + 1) / 2;
  constexpr int M0 = GRP * kMomentGroup;
  constexpr int MG = (M - M0) < kMomentGroup ? (M - M0) : kMomentGroup;
  constexpr int RPW = (MG + NT / 32 - 1) / (NT / 32);
  const size_t HW = (size_t)H * W;
  const int t = threadIdx.x;
  const int TW = NT - 2 * r;
  const int x0 = blockIdx.x * TW;
  const int xc = x0 - r + t;
  const bool col_ok = xc >= 0 && xc < W;
  const int Y0 = blockIdx.y * band_rows;
  const int Y1 = min(H, Y0 + band_rows);
  const int add_lo = max(0, Y0 - r);
  const int s_begin = Y0 - r, s_end = Y1 + r;
  for (int i = t; i < 2 * MG; i += NT) smem[i * kRowStride + 3] = 0.f;

  auto ld_new = [&](int row, float *v) {
    if (col_ok && row >= 0 && row < H) {
#pragma unroll
      for (int i = 0; i < NG; ++i) v[i] = __ldg(G + (size_t)i * HW + (size_t)row * W + xc);
    }
  };
  auto ld_old = [&](int row, float *v) {  // rows that entered this band's windows only
    if (col_ok && row >= add_lo && row < H) {
#pragma unroll
      for (int i = 0; i < NG; ++i) v[i] = __ldg(G + (size_t)i * HW + (size_t)row * W + xc);
    }
  };
  float pa[NG], pb[NG], pc[NG], oa[NG], ob[NG], oc[NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) pa[i] = pb[i] = pc[i] = oa[i] = ob[i] = oc[i] = 0.f;
  ld_new(s_begin, pa);
  ld_new(s_begin + 1, pb);
  ld_old(s_begin - 2 * r - 1, oa);
  ld_old(s_begin - 2 * r, ob);
  float V[MG], Vc[COMP ? MG : 1];  // running sums and (COMP) their Kahan compensation terms
#pragma unroll
  for (int m = 0; m < MG; ++m) V[m] = 0.f;
#pragma unroll
  for (int m = 0; m < (COMP ? MG : 1); ++m) Vc[m] = 0.f;
  // V[m] += x for channel M0 + m (compensated in the COMP instantiation)
  auto acc = [&](int m, float x) {
    if constexpr (COMP) {
      const float y = x - Vc[m];
      const float t2 = V[m] + y;
      Vc[m] = (t2 - V[m]) - y;
      V[m] = t2;
    } else {
      V[m] += x;
    }
  };
  // adds sign * (every channel of this group) at a row with guidance values g; the loops unroll
  // completely, so the channel tests and indices are compile-time constants
  auto update = [&](const float *g, float sign) {
#pragma unroll
    for (int i = 0; i < NG; ++i)
      if (i >= M0 && i < M0 + MG) acc(i - M0, sign * g[i]);
#pragma unroll
    for (int i = 0; i < NG; ++i) {
#pragma unroll
      for (int j = i; j < NG; ++j) {
        const int c = NG + tri_index(NG, i, j);
        if (c >= M0 && c < M0 + MG) {
          if constexpr (COMP)
            acc(c - M0, sign * g[i] * g[j]);
          else
            V[c - M0] = fmaf(sign * g[i], g[j], V[c - M0]);
        }
      }
    }
  };

  // three-buffer rotation: row s + 2 (and the row leaving two steps later) load while row s works
  auto step = [&](const int s, const float *cur, float *nxt, const float *cur_o, float *nxt_o) {
    if (s >= s_end) return;
    ld_new(s + 2, nxt);
    ld_old(s + 1 - 2 * r, nxt_o);
    if (col_ok) {
      if (s - 2 * r - 1 >= add_lo) update(cur_o, -1.f);
      if (s >= 0 && s < H) update(cur, 1.f);
    }
    const int y2 = s - r;
    if (y2 < Y0) return;  // warm-up rows (uniform per CTA)
    float *sA = smem + ((y2 - Y0) & 1) * MG * kRowStride;
#pragma unroll
    for (int m = 0; m < MG; ++m)
      sA[m * kRowStride + 4 + t] = COMP ? V[m] - Vc[COMP ? m : 0] : V[m];
    __syncthreads();
    scan_rows<RPW>(sA, MG);
    __syncthreads();
    const int x = x0 + t;
    if (t < TW && x < W) {
      const size_t pix = (size_t)y2 * W + x;
#pragma unroll
      for (int m = 0; m < MG; ++m)
        mom[(size_t)(M0 + m) * HW + pix] = window(sA + m * kRowStride, t, r);
    }
  };
  for (int s = s_begin; s < s_end; s += 3) {
    step(s, pa, pc, oa, oc);
    step(s + 1, pb, pa, ob, oa);
    step(s + 2, pc, pb, oc, ob);
  }
}

template <int NG, bool COMP>
__global__ void __launch_bounds__(kStripThreads) k_moments(const float *__restrict__ G, int H,
                                                           int W, int r, int band_rows,
                                                           float *__restrict__ mom) {
  constexpr int M = NG + NG * (NG + 1) / 2;
  extern __shared__ __align__(16) float smem[];  // two scan buffers of a group's rows
  switch (blockIdx.z) {  // uniform per CTA
    case 0:
      moments_group<NG, COMP, 0>(G, H, W, r, band_rows, mom, smem);
      break;
    case 1:
      if constexpr (M > kMomentGroup) moments_group<NG, COMP, 1>(G, H, W, r, band_rows, mom, smem);
      break;
    case 2:
      if constexpr (M > 2 * kMomentGroup)
        moments_group<NG, COMP, 2>(G, H, W, r, band_rows, mom, smem);
      break;
    default:
      break;
  }
}

template <int NG, bool COMP>
cudaError_t launch_moments_strip(const float *G, int H, int W, int r, int num_sms, float *mom,
                                 cudaStream_t s, Profiler *prof) {
  constexpr int M = NG + NG * (NG + 1) / 2;
  constexpr int groups = (M + kMomentGroup - 1) / kMomentGroup;
  static_assert(groups <= 3, "k_moments dispatches three channel groups at most");
  constexpr int MG = M < kMomentGroup ? M : kMomentGroup;
  const size_t sm = sizeof(float) * 2 * MG * strip::kRowStride;
  cudaError_t e = cudaSuccess;
  if (sm > 48 * 1024) {
    e = cudaFuncSetAttribute(k_moments<NG, COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_moments<NG, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sm);
  }
  if (e != cudaSuccess) return e;
  // bands planned from the uncompensated kernel's occupancy: compensation changes rounding only
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_moments<NG, false>, kStripThreads,
                                                    sm) != cudaSuccess)
    per_sm = 1;
  const long long resident = (long long)std::max(1, per_sm) * std::max(1, num_sms);
  const int TW = kStripThreads - 2 * r;
  const int strips = (W + TW - 1) / TW;
  // band count minimising (waves of resident CTAs) x (rows streamed, with the 2r warm-up rows)
  long long best_cost = -1;
  int rows = H;
  for (int bands = 1; bands <= std::max(1, H / std::max(8, 2 * r)); ++bands) {
    const int rw = (H + bands - 1) / bands;
    const long long ctas = (long long)strips * groups * ((H + rw - 1) / rw);
    const long long cost = ((ctas + resident - 1) / resident) * (rw + 2 * r);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      rows = rw;
    }
  }
  dim3 grid(strips, (H + rows - 1) / rows, groups);
  LaunchScope ls(prof, "k_moments", s);
  k_moments<NG, COMP><<<grid, kStripThreads, sm, s>>>(G, H, W, r, rows, mom);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------- moment row sums
// Direct sums for n = 19 (too many channels for registers) and windows wider than a strip.
// Moment channel m < n is G_m; m >= n enumerates the pairs (i, j), i <= j, of the packed upper
// triangle. rows[m][y][x] = sum over the clipped horizontal window of the channel's values.
__global__ void k_moment_rows(const float *__restrict__ G, int n, int H, int W, int r,
                              float *__restrict__ rows) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y;
  int m = blockIdx.z;
  if (x >= W) return;
  size_t HW = (size_t)H * W;
  int i, j;
  if (m < n) {
    i = m;
    j = -1;
  } else {
    int e = m - n;  // packed index -> (i, j)
    i = 0;
    while (e >= n - i) {
      e -= n - i;
      ++i;
    }
    j = i + e;
  }
  const float *gi = G + (size_t)i * HW + (size_t)y * W;
  const float *gj = j >= 0 ? G + (size_t)j * HW + (size_t)y * W : nullptr;
  int lo = max(0, x - r), hi = min(W - 1, x + r);
  float s = 0.f;
  if (gj) {
    for (int xx = lo; xx <= hi; ++xx) s = fmaf(__ldg(gi + xx), __ldg(gj + xx), s);
  } else {
    for (int xx = lo; xx <= hi; ++xx) s += __ldg(gi + xx);
  }
  rows[(size_t)m * HW + (size_t)y * W + x] = s;
}

// ------------------------------------------------------------------ moment column sums
// mom[m][y][x] = sum over the clipped vertical window of rows[m][.][x]: the full window sums of
// every moment channel (Prop. 2: the Gram entries are box sums).
__global__ void k_moment_cols(const float *__restrict__ rows, int H, int W, int r,
                              float *__restrict__ mom) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int m = blockIdx.z;
  if (x >= W) return;
  const size_t HW = (size_t)H * W;
  const float *src = rows + (size_t)m * HW + x;
  const int y0 = max(0, y - r), y1 = min(H - 1, y + r);
  float s = 0.f;
#pragma unroll 4
  for (int yy = y0; yy <= y1; ++yy) s += __ldg(src + (size_t)yy * W);
  mom[(size_t)m * HW + (size_t)y * W + x] = s;
}

// ------------------------------------------------------------------- assembly + HGF inverse
// Writes one pixel's record, plane-major with the row pitch record_pitch(W) (consecutive threads
// write consecutive addresses).
template <int NG>
__device__ __forceinline__ void store_record(float *rec, const float *out, int x, int y, int H,
                                             int W) {
  constexpr int REC = record_floats(NG);
  const size_t P = (size_t)record_pitch(W);
  float *dst = rec + (size_t)y * P + x;
#pragma unroll
  for (int e = 0; e < REC; ++e) dst[(size_t)e * H * P] = out[e];
}

// Centred form, one thread per pixel, in window-sum units: with the window sums s_i = B(G_i) and
// s_ij = B(G_i G_j) of the (shifted) guidance, N Sigma = T with T_ij = s_ij - (s_i / N) s_j, and
// (Sigma + eps E)^-1 = N (N eps E + T)^-1. Prop. 1 runs on T with lambda' = N eps (Sec. 3; Sec. 5.1
// for the centred moments), which saves the per-entry division by N; the record then holds
// [mu | packed N (lambda' E + T)^-1 | 0] with mu = s / N.
template <int NG, typename T>
__global__ void __launch_bounds__(128) k_inverse(const float *__restrict__ mom, int H, int W,
                                                 int r, double eps, int combine,
                                                 float *__restrict__ minv,
                                                 float *__restrict__ mu,
                                                 float *__restrict__ rec) {
  constexpr int P = NG * (NG + 1) / 2;
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y;
  if (x >= W) return;
  size_t HW = (size_t)H * W;
  size_t pix = (size_t)y * W + x;
  const int Ni = clipped_count(x, r, W) * clipped_count(y, r, H);
  const T Nn = T(Ni);
  const T invN = T(1) / Nn;

  float raw[NG + P];
#pragma unroll
  for (int e = 0; e < NG + P; ++e) raw[e] = __ldg(mom + (size_t)e * HW + pix);
  T m[NG], sd[NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) {
    sd[i] = T(raw[i]);
    m[i] = sd[i] * invN;
  }
  T S[P];  // N x covariance
#pragma unroll
  for (int i = 0; i < NG; ++i) {
#pragma unroll
    for (int j = i; j < NG; ++j) {
      const int e = tri_index(NG, i, j);
      S[e] = fma(-m[i], sd[j], T(raw[NG + e]));
    }
  }

  const T lam = T(eps) * Nn;
  const T inv_lam = T(1) / lam;
  T al[P];
  prop1_alpha<NG, T>(S, inv_lam, al);

  constexpr int REC = record_floats(NG);
  float out[REC];
#pragma unroll
  for (int i = 0; i < NG; ++i) out[i] = (float)m[i];
  if (combine == HGF_COMBINE_W3) {
    const float nf = (float)Ni;  // exact
#pragma unroll
    for (int i = 0; i < NG; ++i)
#pragma unroll
      for (int j = i; j < NG; ++j)
        out[NG + tri_index(NG, i, j)] =
            (float)inverse_entry<NG, T>(S, al, lam, inv_lam, combine, i, j) * nf;
  } else {
    // N (lambda' E + T)^-1 = -N lambda' alpha: one float64 product, then float32 scaling
    const float f = (float)(-(lam * Nn));
#pragma unroll
    for (int e = 0; e < P; ++e) out[NG + e] = (float)al[e] * f;
  }
#pragma unroll
  for (int e = NG + P; e < REC; ++e) out[e] = 0.f;
#pragma unroll
  for (int e = 0; e < P; ++e) minv[(size_t)e * HW + pix] = out[NG + e];
#pragma unroll
  for (int i = 0; i < NG; ++i) mu[(size_t)i * HW + pix] = out[i];
  store_record<NG>(rec, out, x, y, H, W);
}

// Paper form (Secs. 3-4), one thread per pixel: G_0 = 1 joins the guidance and the uncentred
// (n+1) x (n+1) Gram matrix of window sums, Gram_ij = B(G_i G_j), is inverted with lambda = eps
// in sum units by Prop. 1. The moments are window sums of the shifted channels G~_i = G_i - c_i,
// so Gram = T Gram~ T^T with [1, G] = T [1, G~], T = [[1, 0], [c, E]], rebuilt here in FP64. The
// record holds Mt = T^T (lambda E + Gram)^-1 T, packed: the fused kernels multiply it by the
// shifted slice sums b~ = B([1, G~] p) = T^-1 b, which gives v = T^T w, and the output
// sum_i A(w_i) G_i + A(w_0) equals A(v_0) + sum_i A(v_i) G~_i: the same coefficient layout
// [v_0 | v_1..v_n] as the centred form's [b | a].
template <int NG, typename T>
__global__ void __launch_bounds__(128) k_inverse_paper(const float *__restrict__ mom, int H,
                                                       int W, int r, double eps, int combine,
                                                       const float *__restrict__ shift,
                                                       float *__restrict__ rec) {
  constexpr int P = NG * (NG + 1) / 2, M = NG + 1, PM = M * (M + 1) / 2;
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y;
  if (x >= W) return;
  size_t HW = (size_t)H * W;
  size_t pix = (size_t)y * W + x;
  const T N = T(clipped_count(x, r, W) * clipped_count(y, r, H));

  T c[NG], sg[NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) {
    c[i] = T(__ldg(shift + i));
    sg[i] = T(__ldg(mom + (size_t)i * HW + pix));
  }
  T S[PM];
  S[tri_index(M, 0, 0)] = N;
#pragma unroll
  for (int i = 0; i < NG; ++i) S[tri_index(M, 0, i + 1)] = fma(c[i], N, sg[i]);
#pragma unroll
  for (int i = 0; i < NG; ++i) {
#pragma unroll
    for (int j = i; j < NG; ++j) {
      const T sgg = T(__ldg(mom + (size_t)(NG + tri_index(NG, i, j)) * HW + pix));
      S[tri_index(M, i + 1, j + 1)] = sgg + c[i] * sg[j] + c[j] * sg[i] + c[i] * c[j] * N;
    }
  }

  const T lam = T(eps);
  const T inv_lam = T(1) / lam;
  T al[PM];
  prop1_alpha<M, T>(S, inv_lam, al);
  // Q = (lambda E + Gram)^-1 (packed, in al's place), then Mt = T^T Q T
  T Q[PM];
#pragma unroll
  for (int i = 0; i < M; ++i)
#pragma unroll
    for (int j = i; j < M; ++j)
      Q[tri_index(M, i, j)] = inverse_entry<M, T>(S, al, lam, inv_lam, combine, i, j);
  auto q = [&](int i, int j) { return Q[tri_index(M, i < j ? i : j, i < j ? j : i)]; };
  T u[M];  // u_j = (Q T)_{j0} = Q_j0 + sum_{l>=1} Q_jl c_l
#pragma unroll
  for (int j = 0; j < M; ++j) {
    T acc = q(j, 0);
#pragma unroll
    for (int l = 1; l < M; ++l) acc = fma(q(j, l), c[l - 1], acc);
    u[j] = acc;
  }
  constexpr int REC = record_floats(NG);
  float out[REC];
  T m00 = u[0];
#pragma unroll
  for (int j = 1; j < M; ++j) m00 = fma(c[j - 1], u[j], m00);
  out[tri_index(M, 0, 0)] = (float)m00;
#pragma unroll
  for (int k = 1; k < M; ++k) out[tri_index(M, 0, k)] = (float)u[k];  // (T^T Q T)_{0k} = u_k
#pragma unroll
  for (int i = 1; i < M; ++i)
#pragma unroll
    for (int k = i; k < M; ++k) out[tri_index(M, i, k)] = (float)q(i, k);
#pragma unroll
  for (int e = PM; e < REC; ++e) out[e] = 0.f;
  store_record<NG>(rec, out, x, y, H, W);
  (void)P;
}

template <int NG, typename T>
static void launch_inverse_t(const float *mom, const hgf_guidance *g, cudaStream_t s,
                             Profiler *prof) {
  dim3 grid((g->W + 127) / 128, g->H);
  LaunchScope ls(prof, "k_inverse", s);
  if (g->form == HGF_FORM_PAPER)
    k_inverse_paper<NG, T><<<grid, 128, 0, s>>>(mom, g->H, g->W, g->r, g->eps, g->combine,
                                                 g->shift, g->rec);
  else
    k_inverse<NG, T><<<grid, 128, 0, s>>>(mom, g->H, g->W, g->r, g->eps, g->combine, g->minv,
                                           g->mu, g->rec);
}

template <typename T>
static bool launch_inverse_n(const float *mom, const hgf_guidance *g, cudaStream_t s,
                             Profiler *prof) {
  switch (g->n) {
#define HGF_INV_CASE(N) \
  case N:               \
    launch_inverse_t<N, T>(mom, g, s, prof); \
    return true;
    HGF_INV_CASE(1) HGF_INV_CASE(2) HGF_INV_CASE(3) HGF_INV_CASE(4) HGF_INV_CASE(5)
    HGF_INV_CASE(6) HGF_INV_CASE(7) HGF_INV_CASE(8) HGF_INV_CASE(9) HGF_INV_CASE(19)
#undef HGF_INV_CASE
    default:
      return false;
  }
}

size_t prepare_workspace_bytes(int n, int H, int W) {
  size_t M = (size_t)n + (size_t)n * (n + 1) / 2;
  size_t plane = ((M * (size_t)H * W * sizeof(float) + 255) / 256) * 256;
  return 2 * plane;  // row sums, window sums
}

cudaError_t launch_prepare(hgf_guidance *g, const float *img, void *ws, size_t ws_size,
                           cudaStream_t s, Profiler *prof) {
  const int b = basis_id(g->C, g->degree, g->basis);
  if (b < 0 || basis_n(b) != g->n) return cudaErrorInvalidValue;
  const int H = g->H, W = g->W, n = g->n, HW = H * W;
  const size_t M = (size_t)n + (size_t)n * (n + 1) / 2;
  if (ws_size < prepare_workspace_bytes(n, H, W)) return cudaErrorInvalidValue;
  const size_t plane = ((M * HW * sizeof(float) + 255) / 256) * 256;
  float *rows = (float *)ws;
  float *mom = (float *)((char *)ws + plane);

  cudaError_t e = cudaMemcpyAsync(g->img, img, (size_t)g->C * HW * sizeof(float),
                                  cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  dispatch_basis(b, [&](auto bc) {
    constexpr int B = decltype(bc)::value;
    LaunchScope ls(prof, "k_shifted_guidance", s);
    k_shifted_guidance<B><<<(HW + kShiftThreads - 1) / kShiftThreads, kShiftThreads, 0, s>>>(
        g->img, HW, g->shift, g->G);
  });
  if (n <= 9 && 2 * g->r + 1 < kStripThreads) {
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 1;
    switch (n) {
#define HGF_MOM_CASE(N) \
  case N:               \
    e = g->compensated ? launch_moments_strip<N, true>(g->G, H, W, g->r, sms, mom, s, prof)   \
                       : launch_moments_strip<N, false>(g->G, H, W, g->r, sms, mom, s, prof); \
    break;
      HGF_MOM_CASE(1) HGF_MOM_CASE(2) HGF_MOM_CASE(3) HGF_MOM_CASE(4) HGF_MOM_CASE(5)
      HGF_MOM_CASE(6) HGF_MOM_CASE(7) HGF_MOM_CASE(8) HGF_MOM_CASE(9)
#undef HGF_MOM_CASE
      default:
        e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  } else {
    {
      dim3 grid((W + 127) / 128, H, (unsigned)M);
      LaunchScope ls(prof, "k_moment_rows", s);
      k_moment_rows<<<grid, 128, 0, s>>>(g->G, n, H, W, g->r, rows);
    }
    {
      dim3 grid((W + 127) / 128, H, (unsigned)M);
      LaunchScope ls(prof, "k_moment_cols", s);
      k_moment_cols<<<grid, 128, 0, s>>>(rows, H, W, g->r, mom);
    }
  }
  bool ok = g->inv_precision == HGF_F32    ? launch_inverse_n<float>(mom, g, s, prof)
            : g->inv_precision == HGF_DF64 ? launch_inverse_n<df64>(mom, g, s, prof)
                                           : launch_inverse_n<double>(mom, g, s, prof);
  if (!ok) return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ export
__global__ void k_export_mu(const float *__restrict__ mu, const float *__restrict__ shift, int n,
                            int HW, float *__restrict__ out) {
  size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (p >= (size_t)HW) return;
  for (int i = 0; i < n; ++i) out[(size_t)i * HW + p] = mu[(size_t)i * HW + p] + shift[i];
}

cudaError_t launch_export(const hgf_guidance *g, float *minv_out, float *mu_out, cudaStream_t s) {
  size_t HW = (size_t)g->H * g->W;
  if (minv_out) {
    cudaError_t e = cudaMemcpyAsync(minv_out, g->minv, packed_size(g->n) * HW * sizeof(float),
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  if (mu_out) k_export_mu<<<(unsigned)((HW + 255) / 256), 256, 0, s>>>(g->mu, g->shift, g->n,
                                                                       (int)HW, mu_out);
  return cudaGetLastError();
}

}  // namespace hgf
