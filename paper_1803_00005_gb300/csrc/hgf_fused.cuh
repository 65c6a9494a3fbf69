// Fused multi-label aggregation kernels (included by the hgf_fused_*.cu translation units, each
// of which instantiates launch_basis for some guidance bases; the host side is hgf_aggregate.cu).
//
// Multi-label aggregation + WTA (Sec. 1 pipeline with the centred form of Sec. 5.1 and the
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
// Rows are loaded two steps ahead into registers (a three-buffer rotation), so the load latency
// overlaps two steps of work; the row leaving the vertical window is re-read, still in L2 (or,
// in the ring instantiations, kept in a per-thread shared-memory ring). k_coef stages each row's
// block of inverse records in shared memory with one bulk asynchronous copy. The paper's form
// (HGF_FORM_PAPER) changes only k_coef's per-pixel solve; the stereo instantiation computes the
// cost from the two views instead of reading a cost volume.
// Windows are clipped at the image border: samples outside the image never enter a sum and the
// means divide by the in-image count N(x, y).
#pragma once
#include "hgf_basis.cuh"
#include "hgf_stereo.cuh"
#include "hgf_scan.cuh"
#include "hgf_mbarrier.cuh"
#include "hgf_f32x2.cuh"

#include <algorithm>
#include <type_traits>

namespace hgf {

namespace {

struct StereoTag {};  // cost type of k_coef when the cost is computed from a stereo pair

using strip::NT;
using strip::kRowStride;
using strip::scan_rows;
using strip::window;

// bulk asynchronous copies and bounded mbarrier waits: hgf_mbarrier.cuh
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // a bounded wait gives up after 1 s

// Inverse records of up to 68 floats (n <= 9) are staged in shared memory by tensor copies
// (kRecordBuffers boxes per CTA); larger ones (n = 19) are loaded by phase C itself, one coalesced
// row segment per element.
template <int B>
__host__ __device__ constexpr bool stage_records() { return records_staged(basis_n(B)); }


// CTAs per SM that shared memory leaves room for when the records are staged (r = 9: three at two
// labels per pass, two at four), passed to __launch_bounds__ as the register budget
template <int B, int K, bool COMP>
__host__ __device__ constexpr int coef_min_blocks() {
  return !stage_records<B>() ? (K == 1 ? 3 : 1)  // n = 19: one label per pass leaves room for 3
         : (K <= 2 && !COMP) ? (kRecordBuffers == 1 ? 4 : 3)
         : K <= 4 ? 2 : 1;
}

// Compensated (Kahan) update s += x: c carries the low-order part lost so far, and the sum is
// s - c. Used by the kernels' COMP instantiations for the vertical running sums, where each row
// adds one sample and removes another, so rounding errors would otherwise accumulate over a band.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

template <int B, int K, typename CT, bool COMP>
__global__ void __launch_bounds__(NT, (coef_min_blocks<B, K, COMP>())) k_coef(const CT *__restrict__ cost, int H, int W, int r,
                                             const float *__restrict__ img,
                                             const float *__restrict__ shift,
                                             const float *__restrict__ rec,
                                             const __grid_constant__ CUtensorMap rec_map,
                                             float *__restrict__ coef, int l_first, int n_chunk,
                                             int band_rows, int paper_form, int *status,
                                             const StereoSource stereo) {
  constexpr int NG = basis_n(B), C1 = NG + 1, NC = basis_channels_in(B), RAW = NC + K;
  constexpr int REC = record_floats(NG), CP = coef_floats(NG);
  constexpr bool STAGE = stage_records<B>(), kCoefReload = coef_reload(NG);
  extern __shared__ __align__(128) float smem_raw[];
  // layout: record boxes (128-byte aligned, STAGE) | 2 mbarriers | two scan buffers | (ring)
  const int TW = NT - 2 * r, BW = record_box_width(r);
  const int RBUF = (REC * BW + 31) / 32 * 32;        // floats per record box, 128-byte multiple
  float *recs = align_smem128(smem_raw);             // [kRecordBuffers][REC][BW] (STAGE)
  uint64_t *bars = reinterpret_cast<uint64_t *>(recs + (STAGE ? kRecordBuffers * RBUF : 0));
  // two scan buffers used on alternate rows: a warp may start the next row's vertical update
  // while others still read this row's window sums, so no barrier is needed at the end of a row
  float *sA0 = reinterpret_cast<float *>(bars + 2);
  float *ring = sA0 + 2 * K * C1 * kRowStride;       // [2r+1][RAW][NT], private
  __shared__ int s_fail;
  const int R = 2 * r + 1;
  const size_t HW = (size_t)H * W;
  const size_t plane = coef_plane_floats(NG, HW);  // floats per label in the coefficient workspace
  // grid: x = label pass (fastest, so every pass over one strip and band runs back to back and
  // they share the strip's inverse records through L2), y = strip, z = band
  const int t = threadIdx.x;
  const int x0 = blockIdx.y * TW;
  const int xi = x0 - r + t;
  const bool col_ok = xi >= 0 && xi < W;
  const int Y0 = blockIdx.z * band_rows;
  const int Y1 = min(H, Y0 + band_rows);
  const int k0 = blockIdx.x * K;
  const int nk = min(K, n_chunk - k0);
  const int add_lo = max(0, Y0 - r);
  const int s_begin = Y0 - r, s_end = Y1 + r;

  for (int i = t; i < 2 * K * C1; i += NT) sA0[i * kRowStride + 3] = 0.f;
  float sh[NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) sh[i] = __ldg(shift + i);
  // record box of row y: columns [xr, xr + BW), xr = x0 rounded down to a multiple of 4 (the
  // tensor copy's alignment rule); column x0 + j sits at j + ro
  const int xr = x0 & ~3, ro = x0 - xr;
  const size_t rpitch = (size_t)record_pitch(W);
  const uint32_t rec_bytes = (uint32_t)(REC * BW * sizeof(float));
  // buffer and mbarrier of row y, and the phase parity its copy completes
  auto rbuf = [&](int y) { return kRecordBuffers == 1 ? 0 : (y - Y0) & 1; };
  auto rpar = [&](int y) -> uint32_t {
    return kRecordBuffers == 1 ? (y - Y0) & 1 : ((y - Y0) >> 1) & 1;
  };
  auto issue_records = [&](int y) {  // thread 0 only
    tma_load_3d(recs + rbuf(y) * RBUF, &rec_map, xr, y, 0, rec_bytes, &bars[rbuf(y)]);
  };
  if (STAGE) {
    if (t == 0) {
      s_fail = 0;
      mbar_init(&bars[0], 1);
      mbar_init(&bars[1], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (t == 0) issue_records(Y0);  // the first row has the warm-up rows to arrive
  }

  constexpr bool STEREO = std::is_same<CT, StereoTag>::value;
  const CT *cbase = STEREO ? nullptr : cost + (size_t)(l_first + k0) * HW;
  auto load_row = [&](int row, float *v) {
    if (col_ok && row >= 0 && row < H) {
      const size_t pix = (size_t)row * W + xi;
#pragma unroll
      for (int c = 0; c < NC; ++c) v[c] = __ldg(img + (size_t)c * HW + pix);
      if constexpr (STEREO) {
        // the cost of hgf_cost_volume, computed here: the guidance image is the reference view
        const size_t rowoff = (size_t)row * W;
        const float dI = __ldg(stereo.grad + pix);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          float val = 0.f;
          if (k < nk) {
            const int l = l_first + k0 + k;
            const int xs = min(max(xi - stereo.direction * l, 0), W - 1);
            float col = 0.f;
#pragma unroll
            for (int c = 0; c < NC; ++c)
              col += fabsf(v[c] - __ldg(stereo.other + (size_t)c * HW + rowoff + xs));
            val = stereo_cost(col, NC, dI, __ldg(stereo.grad + HW + rowoff + xs), stereo.alpha,
                              stereo.tau_c, stereo.tau_g);
          }
          v[NC + k] = val;
        }
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k)
          v[NC + k] = k < nk ? load_cost(cbase, (size_t)k * HW + pix) : 0.f;
      }
    }
  };
  float pa[RAW], pb[RAW], pc[RAW];
  constexpr int OR = kCoefReload ? RAW : 1;  // outgoing-row buffers (reload mode only)
  float oa[OR], ob[OR], oc[OR];
#pragma unroll
  for (int c = 0; c < RAW; ++c) pa[c] = pb[c] = pc[c] = 0.f;
#pragma unroll
  for (int c = 0; c < OR; ++c) oa[c] = ob[c] = oc[c] = 0.f;
  auto load_old = [&](int row, float *v) {
    if (kCoefReload && row >= add_lo) load_row(row, v);
  };
  load_row(s_begin, pa);
  load_row(s_begin + 1, pb);
  load_old(s_begin - 2 * r - 1, oa);
  load_old(s_begin + 1 - 2 * r - 1, ob);

  float V[K][C1];
  float Vc[COMP ? K : 1][COMP ? C1 : 1];  // Kahan compensation terms (COMP only)
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < C1; ++c) V[k][c] = 0.f;
#pragma unroll
  for (int k = 0; k < (COMP ? K : 1); ++k)
#pragma unroll
    for (int c = 0; c < (COMP ? C1 : 1); ++c) Vc[k][c] = 0.f;

  // One step per input row s: `cur` holds row s (loaded two steps earlier) and row s + 2 is
  // loaded into `nxt`. The loop is unrolled three times so that the three buffers rotate roles
  // without register copies (a copy would wait for the load it copies).
  bool failed = false;
  auto step = [&](const int s, const float *cur, float *nxt, const float *cur_o, float *nxt_o) {
    if (s >= s_end || failed) return;
    load_row(s + 2, nxt);
    load_old(s + 2 - 2 * r - 1, nxt_o);
    const int y1 = s - r;
    const int x = x0 + t;
    const bool coef_here = y1 >= Y0 && t < TW && x < W;
    // ---- phase A: vertical running sums over input rows [s-2r, s]
    if (col_ok) {
      float *slot = ring + (size_t)(((s - s_begin) % R) * RAW) * NT + t;
      const int so = s - 2 * r - 1;
      if (so >= add_lo) {  // the outgoing row occupies the slot the new row will take
        float xo[NC], go[NG];
#pragma unroll
        for (int c = 0; c < NC; ++c) xo[c] = kCoefReload ? cur_o[kCoefReload ? c : 0] : slot[c * NT];
        eval_basis<B>(xo, sh, go);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float p = kCoefReload ? cur_o[kCoefReload ? NC + k : 0] : slot[(NC + k) * NT];
          if constexpr (COMP) {
            kahan_add(V[k][0], Vc[k][0], -p);
#pragma unroll
            for (int i = 0; i < NG; ++i) kahan_add(V[k][i + 1], Vc[k][i + 1], -go[i] * p);
          } else {
            V[k][0] -= p;
            if constexpr (STAGE) {
              fma_channels<NG>(V[k], go, -p);  // fmaf(go, -p, .) == fmaf(-go, p, .)
            } else {
#pragma unroll
              for (int i = 0; i < NG; ++i) V[k][i + 1] = fmaf(-go[i], p, V[k][i + 1]);
            }
          }
        }
      }
      if (s >= 0 && s < H) {
        float g[NG];
        eval_basis<B>(cur, sh, g);
        if (!kCoefReload) {
#pragma unroll
          for (int c = 0; c < RAW; ++c) slot[c * NT] = cur[c];
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float p = cur[NC + k];
          if constexpr (COMP) {
            kahan_add(V[k][0], Vc[k][0], p);
#pragma unroll
            for (int i = 0; i < NG; ++i) kahan_add(V[k][i + 1], Vc[k][i + 1], g[i] * p);
          } else {
            V[k][0] += p;
            if constexpr (STAGE) {
              fma_channels<NG>(V[k], g, p);
            } else {
#pragma unroll
              for (int i = 0; i < NG; ++i) V[k][i + 1] = fmaf(g[i], p, V[k][i + 1]);
            }
          }
        }
      }
    }
    if (y1 < Y0) return;  // warm-up rows: no coefficient row complete yet (uniform per CTA)
    float *sA = sA0 + ((y1 - Y0) & 1) * K * C1 * kRowStride;

    // ---- phase B: horizontal window sums via inclusive prefix scans
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < C1; ++c)
        sA[(k * C1 + c) * kRowStride + 4 + t] = COMP ? V[k][c] - Vc[COMP ? k : 0][COMP ? c : 0]
                                                     : V[k][c];
    __syncthreads();
    // every thread is past the previous row's phase C: that row's record buffer is free
    if (STAGE && t == 0) {
      if (kRecordBuffers == 2 && y1 + 1 < Y1) issue_records(y1 + 1);
      if (kRecordBuffers == 1 && y1 > Y0) issue_records(y1);
    }
    scan_rows<(K * C1 + NT / 32 - 1) / (NT / 32)>(sA, nk * C1);
    if (STAGE && !mbar_wait(&bars[rbuf(y1)], rpar(y1), kWaitLimitNs)) s_fail = 1;
    __syncthreads();
    if (STAGE && s_fail) {  // a copy never completed: report, drain with a bound, stop
      if (t == 0) {
        atomicExch(status, 1);
        if (kRecordBuffers == 2 && y1 + 1 < Y1) mbar_wait(&bars[rbuf(y1 + 1)], rpar(y1 + 1), kWaitLimitNs);
      }
      failed = true;
      return;
    }

    // ---- phase C: coefficients at (x, y1)
    if (coef_here) {
      const size_t pix = (size_t)y1 * W + x;
      const float invN = 1.f / (float)(clipped_count(x, r, W) * clipped_count(y1, r, H));
      const float *rrow = recs + rbuf(y1) * RBUF + t + ro;
      const float *grow = rec + (size_t)y1 * rpitch + x;  // plane-major records (not staged)
      const size_t gplane = (size_t)H * rpitch;
      int stride = BW;  // made opaque per label pair below so that addresses are not hoisted
      auto recv = [&](int e) -> float {
        return STAGE ? rrow[e * stride] : __ldg(grow + (size_t)e * gplane);
      };
      if (paper_form) {
        // paper form: v = Mt b~ with b~ = [B(p), B(G~_i p)], the raw window sums (no means)
        constexpr int KP = K < 2 ? K : 2;
#pragma unroll 1
        for (int kb = 0; kb < K; kb += KP) {
          if (kb >= nk) break;
          asm volatile("" : "+r"(stride));
          float bs[KP][C1], v[KP][C1];
#pragma unroll
          for (int kk = 0; kk < KP; ++kk) {
            const float *row = sA + (kb + kk) * C1 * kRowStride;
#pragma unroll
            for (int c = 0; c < C1; ++c) {
              bs[kk][c] = window(row + c * kRowStride, t, r);
              v[kk][c] = 0.f;
            }
          }
#pragma unroll
          for (int i = 0; i < C1; ++i) {
#pragma unroll
            for (int j = i; j < C1; ++j) {
              const float Mij = recv(tri_index(C1, i, j));
#pragma unroll
              for (int kk = 0; kk < KP; ++kk) {
                v[kk][i] = fmaf(Mij, bs[kk][j], v[kk][i]);
                if (j != i) v[kk][j] = fmaf(Mij, bs[kk][i], v[kk][j]);
              }
            }
          }
#pragma unroll
          for (int kk = 0; kk < KP; ++kk) {
            if (kb + kk < nk) {
              float o[CP];
#pragma unroll
              for (int i = 0; i < C1; ++i) o[i] = v[kk][i];
#pragma unroll
              for (int i = C1; i < CP; ++i) o[i] = 0.f;
              float2 *dst = reinterpret_cast<float2 *>(coef + (size_t)(k0 + kb + kk) * plane) +
                            coef_pair_index(NG, pix, 0);
#pragma unroll
              for (int q = 0; q < CP / 2; ++q) dst[q * 32] = make_float2(o[2 * q], o[2 * q + 1]);
            }
          }
        }
        return;
      }
      float m[NG];
#pragma unroll
      for (int i = 0; i < NG; ++i) m[i] = recv(i);
      // labels in pairs, one pair at a time: only two labels' cov and a are live next to the
      // record, so four or eight labels per pass fit in registers
      constexpr int KP = K < 2 ? K : 2;
#pragma unroll 1
      for (int kb = 0; kb < K; kb += KP) {
        if (kb >= nk) break;
        asm volatile("" : "+r"(stride));
        float cov[KP][NG], a[KP][NG], pbar[KP];
#pragma unroll
        for (int kk = 0; kk < KP; ++kk) {
          const float *row = sA + (kb + kk) * C1 * kRowStride;
          pbar[kk] = window(row, t, r) * invN;
#pragma unroll
          for (int i = 0; i < NG; ++i) {
            const float mi = window(row + (i + 1) * kRowStride, t, r) * invN;
            cov[kk][i] = fmaf(-m[i], pbar[kk], mi);
            a[kk][i] = 0.f;
          }
        }
        if constexpr (KP == 2 && STAGE) {
          // the pair's two mat-vecs as packed two-lane FMAs (the same roundings in the same order;
          // measured slower at n = 19, whose records are read from L2, so kept to n <= 9)
          float2 a2[NG], c2[NG];
#pragma unroll
          for (int i = 0; i < NG; ++i) {
            c2[i] = make_float2(cov[0][i], cov[1][i]);
            a2[i] = make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int i = 0; i < NG; ++i) {
#pragma unroll
            for (int j = i; j < NG; ++j) {
              const float Mij = recv(NG + tri_index(NG, i, j));
              const float2 M2 = make_float2(Mij, Mij);
              a2[i] = fma2(M2, c2[j], a2[i]);
              if (j != i) a2[j] = fma2(M2, c2[i], a2[j]);
            }
          }
#pragma unroll
          for (int i = 0; i < NG; ++i) {
            a[0][i] = a2[i].x;
            a[1][i] = a2[i].y;
          }
        } else {
#pragma unroll
          for (int i = 0; i < NG; ++i) {
#pragma unroll
            for (int j = i; j < NG; ++j) {
              const float Mij = recv(NG + tri_index(NG, i, j));
#pragma unroll
              for (int kk = 0; kk < KP; ++kk) {
                a[kk][i] = fmaf(Mij, cov[kk][j], a[kk][i]);
                if (j != i) a[kk][j] = fmaf(Mij, cov[kk][i], a[kk][j]);
              }
            }
          }
        }
#pragma unroll
        for (int kk = 0; kk < KP; ++kk) {
          if (kb + kk < nk) {
            float b = pbar[kk];
#pragma unroll
            for (int i = 0; i < NG; ++i) b = fmaf(-a[kk][i], m[i], b);
            float o[CP];
            o[0] = b;
#pragma unroll
            for (int i = 0; i < NG; ++i) o[i + 1] = a[kk][i];
#pragma unroll
            for (int i = C1; i < CP; ++i) o[i] = 0.f;
            float2 *dst = reinterpret_cast<float2 *>(coef + (size_t)(k0 + kb + kk) * plane) +
                          coef_pair_index(NG, pix, 0);
#pragma unroll
            for (int q = 0; q < CP / 2; ++q) dst[q * 32] = make_float2(o[2 * q], o[2 * q + 1]);
          }
        }
      }
    }
  };
  for (int s = s_begin; s < s_end && !failed; s += 3) {
    step(s, pa, pc, oa, oc);
    step(s + 1, pb, pa, ob, oa);
    step(s + 2, pc, pb, oc, ob);
  }
}

template <int B, bool RING>
constexpr size_t apply_smem_bytes(int r) {
  return sizeof(float) * ((size_t)2 * (basis_n(B) + 1) * kRowStride +
                          (RING ? (size_t)(2 * r + 1) * (basis_n(B) + 1) * NT : 0));
}

// One label per CTA. RING: the outgoing coefficient row comes from the thread's shared-memory
// ring; otherwise it is reloaded from device memory (used when the ring does not fit).
// No minimum CTA count for n <= 9: capping registers for 5, 6 or 8 CTAs per SM made k_apply
// slower (450x375, n = 9: 0.29 ms -> 0.41-0.44 ms). At n = 19 a cap for three CTAs per SM (221 ->
// 168 registers, a few spills) made it faster (1280x960, L = 128: 8.38 -> 7.90 ms).
template <int B>
__host__ __device__ constexpr int apply_min_blocks() { return basis_n(B) > 9 ? 3 : 1; }

template <int B, bool RING, bool COMP>
__global__ void __launch_bounds__(NT, apply_min_blocks<B>()) k_apply(const float *__restrict__ coef, int H, int W, int r,
                                              const float *__restrict__ img,
                                              const float *__restrict__ shift,
                                              unsigned long long *__restrict__ keys,
                                              unsigned long long *__restrict__ keys2,
                                              float *__restrict__ filtered, int l_first,
                                              int band_rows) {
  constexpr int NG = basis_n(B), C1 = NG + 1, NC = basis_channels_in(B), CP = coef_floats(NG);
  extern __shared__ __align__(16) float smem[];
  float *sA0 = smem;                         // two scan buffers, alternate rows (see k_coef)
  float *ring = smem + 2 * C1 * kRowStride;  // [2r+1][C1][NT]
  const int R = 2 * r + 1;
  const size_t HW = (size_t)H * W;
  // grid: x = label (fastest), y = strip, z = band
  const int t = threadIdx.x;
  const int TW = NT - 2 * r;
  const int x0 = blockIdx.y * TW;
  const int xc = x0 - r + t;
  const bool col_ok = xc >= 0 && xc < W;
  const int Y0 = blockIdx.z * band_rows;
  const int Y1 = min(H, Y0 + band_rows);
  const int k = blockIdx.x;
  const int add_lo = max(0, Y0 - r);
  const int s_begin = Y0 - r, s_end = Y1 + r;

  if (t < 2 * C1) sA0[t * kRowStride + 3] = 0.f;
  float sh[NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) sh[i] = __ldg(shift + i);
  const float *cb = coef + (size_t)k * coef_plane_floats(NG, HW);
  auto load_row = [&](int row, float *v) {
    if (col_ok && row >= 0 && row < H) {
      const float2 *src =
          reinterpret_cast<const float2 *>(cb) + coef_pair_index(NG, (size_t)row * W + xc, 0);
#pragma unroll
      for (int q = 0; q < CP / 2; ++q) {
        const float2 u = __ldg(src + q * 32);
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
  float V[C1], Vc[COMP ? C1 : 1];
#pragma unroll
  for (int c = 0; c < C1; ++c) V[c] = 0.f;
#pragma unroll
  for (int c = 0; c < (COMP ? C1 : 1); ++c) Vc[c] = 0.f;
  auto acc = [&](int c, float x) {  // V[c] += x, compensated in the COMP instantiation
    if constexpr (COMP) kahan_add(V[c], Vc[c], x);
    else V[c] += x;
  };
  // V[c] += sign * x[c] for every channel; uncompensated: channel pairs as packed two-lane adds
  // (x * -1 + V is exactly V - x), the same roundings as V[c] += sign * x[c]
  auto acc_all = [&](const float *x, float sign) {
    if constexpr (COMP) {
#pragma unroll
      for (int c = 0; c < C1; ++c) acc(c, sign * x[c]);
    } else {
      const float2 sg = make_float2(sign, sign);
#pragma unroll
      for (int c = 0; c + 1 < C1; c += 2) {
        const float2 v = fma2(make_float2(x[c], x[c + 1]), sg, make_float2(V[c], V[c + 1]));
        V[c] = v.x;
        V[c + 1] = v.y;
      }
      if (C1 % 2) V[C1 - 1] = fmaf(x[C1 - 1], sign, V[C1 - 1]);
    }
  };

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
          for (int c = 0; c < C1; ++c) acc(c, -slot[c * NT]);
        }
        if (s >= 0 && s < H) {
#pragma unroll
          for (int c = 0; c < C1; ++c) {
            acc(c, cur[c]);
            slot[c * NT] = cur[c];
          }
        }
      } else {
        if (so >= add_lo) acc_all(cur_o, -1.f);
        if (s >= 0 && s < H) acc_all(cur, 1.f);
      }
    }
    if (y2 < Y0) return;
    float *sA = sA0 + ((y2 - Y0) & 1) * C1 * kRowStride;

#pragma unroll
    for (int c = 0; c < C1; ++c)
      sA[c * kRowStride + 4 + t] = COMP ? V[c] - Vc[COMP ? c : 0] : V[c];
    __syncthreads();
    scan_rows<(C1 + NT / 32 - 1) / (NT / 32)>(sA, C1);
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
      if (keys) {
        const unsigned long long key = wta_key(q, label);
        if (keys2) {
          // second-smallest key: every key but the final minimum reaches keys2 exactly once,
          // either directly (it lost to the minimum so far) or when a smaller key displaces it
          const unsigned long long old = atomicMin(keys + pix, key);
          atomicMin(keys2 + pix, old > key ? old : key);
        } else {
          atomicMin(keys + pix, key);
        }
      }
    }
  };
  for (int s = s_begin; s < s_end; s += 3) {
    step(s, pa, pc, oa, oc);
    step(s + 1, pb, pa, ob, oa);
    step(s + 2, pc, pb, oc, ob);
  }
}


// Raises a kernel's dynamic shared-memory limit to `bytes`. The default limit (48 KB) covers
// static and dynamic shared memory together, and the kernels' 128-byte aligned dynamic base may
// start up to 128 bytes past their static variables, so the limit is raised well before 48 KB.
template <typename Kern>
cudaError_t set_smem(Kern k, size_t bytes) {
  if (bytes <= 32 * 1024) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) note_failed("cudaFuncSetAttribute (dynamic shared memory)");
  return e;
}

// Rows per band for a kernel whose grid is strips x bands x slabs: the band count that minimises
// (waves of resident CTAs) x (rows streamed per CTA, including the 2r warm-up rows). Callers pass
// a nominal slab count fixed per call (from min(64, L), never from the chunk or from K): the band
// boundaries decide the order of the running sums, so results are then identical whether an
// image is aggregated alone, in a batch, in the serving loop, in label chunks or with any K.
// Small label counts get more, shorter bands, so that a single slice still fills the GPU.
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

template <typename Kern>
static int resident_ctas(Kern k, size_t smem, int threads = NT) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  return std::max(1, per_sm) * std::max(1, sms);
}

template <int B, int K, bool COMP>
cudaError_t launch_chunk(const hgf_guidance *g, const void *cost, int cost_dtype, int l_first,
                         int nc, float *filtered, float *coef_ws, unsigned long long *keys,
                         unsigned long long *keys2,
                         int band_rows, bool apply_ring, int nominal, int *status,
                         const StereoSource &stereo, const CUtensorMap &map, cudaStream_t s,
                         Profiler *prof) {
  const int H = g->H, W = g->W, r = g->r;
  const int TW = NT - 2 * r;
  const unsigned strips = (W + TW - 1) / TW;
  cudaError_t e;
  {
    const size_t sm = coef_smem(basis_n(B), basis_channels_in(B), K, r);
    // the shared-memory limit is raised before the occupancy query so that every call (the
    // first included) plans the same bands
    e = set_smem(k_coef<B, K, float, COMP>, sm);
    if (e == cudaSuccess) e = set_smem(k_coef<B, K, __nv_bfloat16, COMP>, sm);
    if (e == cudaSuccess) e = set_smem(k_coef<B, K, __half, COMP>, sm);
    if (e == cudaSuccess) e = set_smem(k_coef<B, K, StereoTag, COMP>, sm);
    if (e != cudaSuccess) return e;
    const int passes = (nc + K - 1) / K;
    // bands planned for the two-label, uncompensated kernel whatever K is, so that K never
    // changes a result and compensation changes only the rounding of the sums
    const size_t sm2 = coef_smem(basis_n(B), basis_channels_in(B), 2, r);
    e = set_smem(k_coef<B, 2, float, false>, sm2);
    if (e != cudaSuccess) return e;
    const int rows = band_rows > 0 ? band_rows
                                   : choose_band_rows(H, r, (long long)strips * std::max(1, nominal / 2),
                                                      resident_ctas(k_coef<B, 2, float, false>, sm2));
    dim3 grid(passes, strips, (H + rows - 1) / rows);
    if (prof) {
      const int pl[8] = {2, TW, TW, rows, 0, K, nc, (int)(grid.x * grid.y * grid.z)};
      for (int i = 0; i < 8; ++i) prof->plan[i] = pl[i];
    }
    LaunchScope ls(prof, "k_coef", s);
#define HGF_COEF(CT)                                                                          \
  k_coef<B, K, CT, COMP><<<grid, NT, sm, s>>>((const CT *)cost, H, W, r, g->img, g->shift,    \
                                              g->rec, map, coef_ws, l_first, nc, rows,        \
                                              g->form == HGF_FORM_PAPER ? 1 : 0, status,      \
                                              stereo);
    switch (cost_dtype) {
      case HGF_F32: HGF_COEF(float) break;
      case HGF_BF16: HGF_COEF(__nv_bfloat16) break;
      case HGF_F16: HGF_COEF(__half) break;
      case kCostStereo: HGF_COEF(StereoTag) break;
      default: return cudaErrorInvalidValue;
    }
#undef HGF_COEF
  }
  {
    LaunchScope ls(prof, "k_apply", s);
    const size_t ring_sm = apply_smem_bytes<B, true>(r);
    bool ringed = false;
    if constexpr (!COMP) {
      if (apply_ring && ring_sm <= 227 * 1024) {
        ringed = true;
        e = set_smem(k_apply<B, true, false>, ring_sm);
        if (e != cudaSuccess) return e;
        const int rows = band_rows > 0 ? band_rows
                                       : choose_band_rows(H, r, (long long)strips * nominal,
                                                          resident_ctas(k_apply<B, true, false>,
                                                                        ring_sm));
        dim3 grid(nc, strips, (H + rows - 1) / rows);
        if (prof) prof->plan[4] = rows;
        k_apply<B, true, false><<<grid, NT, ring_sm, s>>>(coef_ws, H, W, r, g->img, g->shift,
                                                          keys, keys2, filtered, l_first,
                                                          rows);
      }
    }
    if (!ringed) {
      const size_t sm = apply_smem_bytes<B, false>(r);
      e = set_smem(k_apply<B, false, COMP>, sm);
      if (e == cudaSuccess && COMP) e = set_smem(k_apply<B, false, false>, sm);
      if (e != cudaSuccess) return e;
      const int rows = band_rows > 0 ? band_rows
                                     : choose_band_rows(H, r, (long long)strips * nominal,
                                                        resident_ctas(k_apply<B, false, false>,
                                                                      sm));
      dim3 grid(nc, strips, (H + rows - 1) / rows);
      if (prof) prof->plan[4] = rows;
      k_apply<B, false, COMP><<<grid, NT, sm, s>>>(coef_ws, H, W, r, g->img, g->shift, keys,
                                                   keys2, filtered, l_first, rows);
    }
  }
  return cudaGetLastError();
}

}  // namespace

// Every chunk of labels of one aggregation for basis B (one explicit instantiation per
// translation unit hgf_fused_*.cu, so that the kernels compile in parallel): the single-pass
// kernel (hgf_onepass.cuh, instantiated for n <= 9) when the plan selects it, else k_coef +
// k_apply per chunk.
template <int B>
cudaError_t launch_basis(const hgf_guidance *g, const void *cost, int cost_dtype, int L,
                         float *filtered, float *coef_ws, unsigned long long *keys,
                         const AggregatePlan &p, int *status, const StereoSource &stereo,
                         const CUtensorMap &map, cudaStream_t s, Profiler *prof) {
  cudaError_t e = cudaSuccess;
  unsigned long long *keys2 = keys && p.second ? keys + (size_t)g->H * g->W : nullptr;
  if constexpr (onepass_built(B)) {
    if (p.onepass)
      return launch_onepass<B>(g, cost, cost_dtype, L, filtered, keys, keys2, p, status, stereo,
                               map, coef_ws, p.onepass_ctas, s, prof);
  }
  if (p.onepass) return cudaErrorInvalidValue;
  for (int l0 = 0; l0 < L && e == cudaSuccess; l0 += p.chunk) {
    const int nc = std::min(p.chunk, L - l0);
    if (g->compensated)  // compensated sums: two labels per pass only
      e = launch_chunk<B, 2, true>(g, cost, cost_dtype, l0, nc, filtered, coef_ws, keys,
                                   keys2, p.band_rows, false, p.nominal, status, stereo, map, s,
                                   prof);
    else if (p.K == 1) {
      // one label per pass: built for the bases whose records are not staged (n = 19)
      if constexpr (!stage_records<B>())
        e = launch_chunk<B, 1, false>(g, cost, cost_dtype, l0, nc, filtered, coef_ws, keys,
                                      keys2, p.band_rows, p.apply_ring, p.nominal, status, stereo,
                                      map, s, prof);
      else
        e = cudaErrorInvalidValue;
    } else if (p.K == 4)
      e = launch_chunk<B, 4, false>(g, cost, cost_dtype, l0, nc, filtered, coef_ws, keys, keys2,
                                    p.band_rows, p.apply_ring, p.nominal, status, stereo, map, s,
                                    prof);
    else if (p.K == 8)
      e = launch_chunk<B, 8, false>(g, cost, cost_dtype, l0, nc, filtered, coef_ws, keys, keys2,
                                    p.band_rows, p.apply_ring, p.nominal, status, stereo, map, s,
                                    prof);
    else
      e = launch_chunk<B, 2, false>(g, cost, cost_dtype, l0, nc, filtered, coef_ws, keys, keys2,
                                    p.band_rows, p.apply_ring, p.nominal, status, stereo, map, s,
                                    prof);
  }
  return e;
}

}  // namespace hgf

#define HGF_INSTANTIATE_BASIS(B)                                                               \
  template cudaError_t hgf::launch_basis<B>(const hgf_guidance *, const void *, int, int,      \
                                            float *, float *, unsigned long long *,           \
                                            const hgf::AggregatePlan &, int *,                \
                                            const hgf::StereoSource &, const CUtensorMap &,   \
                                            cudaStream_t, hgf::Profiler *);
