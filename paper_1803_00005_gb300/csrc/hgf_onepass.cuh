// Single-pass multi-label aggregation + WTA (included by the hgf_onepass_*.cu translation units,
// each of which instantiates launch_onepass for some guidance bases).
//
// One persistent kernel carries the whole per-label part of the filter (Sec. 5.1 with the box
// stages of Sec. 4.1, Eq. HGF_z1 and Sec. 4.3, Eq. HGF_z2) for every label, reading each cost
// slice once and folding WTA into the same pass. A CTA of 128 threads (one per column of a
// 128-column strip) takes work items (K labels, strip, band of rows) in turn and streams the
// band's rows:
//   stage 1: vertical running sums of (p, G_1 p, .., G_n p) for the K labels in registers,
//            horizontal window sums by prefix scans of shared rows, then per coefficient pixel
//            cov = A(G p) - mu A(p), a = Minv cov, b = A(p) - a.mu, with the pixel's inverse
//            record (staged by one tensor copy per row) read once for all K labels;
//   stage 2: the coefficient rows (b, a_1..a_n) are scanned in shared rows; their horizontal
//            window sums go into a (2r+1)-row ring per output column and label, whose vertical
//            running sums in registers give B(b), B(a_i); then q = (sum_i B(a_i) G_i + B(b)) / N,
//            and one packed 64-bit atomicMin per pixel for the K labels together.
// The ring lives in a small device buffer, one slot per resident CTA (the grid is persistent), so
// that it stays in L2: each entry is written once and read back 2r+1 rows later, and nothing of
// it needs to reach DRAM. Shared memory then holds only the scan rows and the record box, which
// leaves room for K = 2 labels per CTA and three CTAs per SM.
// Thread t holds column x0 - 2r + t: the middle 128 - 2r threads produce coefficients, the middle
// 128 - 4r produce outputs, so a strip advances by 128 - 4r columns. The input row leaving the
// stage-1 window is re-read (it is still in L2) two rows ahead, like the incoming rows; the same
// buffer gives the guidance of the output row, which trails the incoming row by 2r. Windows are
// clipped at the image border: samples outside the image never enter a sum, and the means divide
// by the in-image count N(x, y) of each stage's own pixel.
#pragma once
#include "hgf_fused.cuh"

namespace hgf {

namespace {

// Everything a work item of the single-pass kernels reads of its job.
struct FusedJob {
  const void *cost;             // L x H x W of cost_dtype (unused for a stereo source)
  const float *img, *shift;     // guidance image C x H x W, channel shifts c_i
  unsigned long long *keys, *keys2;  // WTA keys (H x W; keys2 for the margin or NULL)
  float *filtered;              // L x H x W or NULL
  int H, W, r, L, band_rows, n_strips, n_bands, paper_form, basis, cost_dtype;
  StereoSource stereo;
};

// Shared-memory layout and per-CTA state of the single-pass kernels.
struct FusedCta {
  float *recs;   // [REC][kFusedBoxWidth] record box, 128-byte aligned
  uint64_t *bar; // its mbarrier
  float *S1, *S2;  // scan rows of the two stages
  int *s_fail;
  float *ring;   // this CTA's ring slot in device memory
  uint64_t keep; // L2 policy of the ring
  uint32_t copies;  // record copies completed so far (the parity of the next wait)
  bool failed;
};

// Lays out the shared memory (a record box of rec_floats elements, rows scan rows per stage),
// zeroes the scan rows' prefix slots and initialises the mbarrier (then a CTA barrier).
__device__ __forceinline__ void fused_cta_init(FusedCta &c, float *smem_raw, int rec_floats,
                                               int rows, int *s_fail, float *ring) {
  c.recs = align_smem128(smem_raw);
  c.bar = reinterpret_cast<uint64_t *>(c.recs + rec_floats * kFusedBoxWidth);
  c.S1 = reinterpret_cast<float *>(c.bar + 2);
  c.S2 = c.S1 + rows * kRowStride;
  c.s_fail = s_fail;
  c.ring = ring;
  c.keep = l2_policy_evict_last();
  c.copies = 0;
  c.failed = false;
  for (int i = threadIdx.x; i < 2 * rows; i += NT) c.S1[i * kRowStride + 3] = 0.f;
  if (threadIdx.x == 0) {
    *s_fail = 0;
    mbar_init(c.bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// One work item (K labels from l0, one strip, one band) of the single-pass kernels: streams the
// band's rows through both box stages, the coefficients and the output with WTA.
template <int B, int K, typename CT, bool COMP>
__device__ __forceinline__ void fused_item(const FusedJob &jb, const CUtensorMap *map,
                                           long long item, FusedCta &cta, int *status) {
  constexpr int NG = basis_n(B), C1 = NG + 1, NC = basis_channels_in(B), RAW = NC + K;
  constexpr int REC = record_floats(NG);
  constexpr bool STEREO = std::is_same<CT, StereoTag>::value;
  constexpr int BW = kFusedBoxWidth;
  const int H = jb.H, W = jb.W, r = jb.r, L = jb.L, band_rows = jb.band_rows;
  const int n_strips = jb.n_strips, paper_form = jb.paper_form;
  const CT *__restrict__ cost = static_cast<const CT *>(jb.cost);
  const float *__restrict__ img = jb.img;
  unsigned long long *__restrict__ keys = jb.keys;
  unsigned long long *__restrict__ keys2 = jb.keys2;
  float *__restrict__ filtered = jb.filtered;
  const StereoSource &stereo = jb.stereo;
  const int R = 2 * r + 1, TWo = NT - 4 * r;
  float *recs = cta.recs, *S1 = cta.S1, *S2 = cta.S2;
  uint64_t *bar = cta.bar;
  int &s_fail = *cta.s_fail;
  uint32_t &copies = cta.copies;
  bool &failed = cta.failed;
  const uint64_t keep = cta.keep;
  const size_t HW = (size_t)H * W;
  const int t = threadIdx.x;
  const bool coef_col = t >= r && t < NT - r;
  const bool out_col = t >= 2 * r && t < NT - 2 * r;
  // this CTA's ring slot: [R][K][C1][TWo], this thread's output column
  float *ring = cta.ring + (out_col ? t - 2 * r : 0);
  const uint32_t rec_bytes = (uint32_t)(REC * BW * sizeof(float));
  float sh[NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) sh[i] = __ldg(jb.shift + i);
  const int n_lg = (L + K - 1) / K;
  const int lg = (int)(item % n_lg);
  const long long rest = item / n_lg;
  const int strip = (int)(rest % n_strips), band = (int)(rest / n_strips);
  const int l0 = lg * K, nk = min(K, L - l0);
  const int x0 = strip * TWo;    // first output column of the strip
  const int xi = x0 - 2 * r + t;  // this thread's column
  const bool col_ok = xi >= 0 && xi < W;
  const bool coef_t = col_ok && coef_col;
  const bool out_t = col_ok && out_col;
  const int Y0 = band * band_rows;
  const int Y1 = min(H, Y0 + band_rows);
  const int lo1 = max(0, Y0 - 2 * r);                      // first input row summed by stage 1
  const int c_lo = max(0, Y0 - r), c_hi = min(H, Y1 + r);  // coefficient rows of the band
  const int s_begin = Y0 - 2 * r, s_end = Y1 + 2 * r;
  // record box of a row: columns [xr, xr + BW) with xr the first coefficient column x0 - r
  // rounded down to a multiple of 4 (the tensor copy's alignment rule); column t reads box
  // column t - r + ro. Every thread is past the previous item's last use of the box (its last
  // coefficient row ended with a barrier), so the first copy can start at once.
  const int xr = (x0 - r) & ~3;
  const int ro = (x0 - r) - xr;
  if (t == 0) tma_load_3d(recs, map, xr, c_lo, 0, rec_bytes, bar);

  const CT *cbase = STEREO ? nullptr : cost + (size_t)l0 * HW;
  auto load_row = [&](int row, float *v) {
    if (col_ok && row >= 0 && row < H) {
      const size_t pix = (size_t)row * W + xi;
#pragma unroll
      for (int c = 0; c < NC; ++c) v[c] = __ldg(img + (size_t)c * HW + pix);
      if constexpr (STEREO) {
        const size_t rowoff = (size_t)row * W;
        const float dI = __ldg(stereo.grad + pix);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          float val = 0.f;
          if (k < nk) {
            const int xs = min(max(xi - stereo.direction * (l0 + k), 0), W - 1);
            float col = 0.f;
#pragma unroll
            for (int c = 0; c < NC; ++c)
              col += fabsf(v[c] - __ldg(stereo.other + (size_t)c * HW + rowoff + xs));
            val = stereo_cost(col, NC, dI, __ldg(stereo.grad + HW + rowoff + xs),
                              stereo.alpha, stereo.tau_c, stereo.tau_g);
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
  auto load_old = [&](int row, float *v) {
    if (row >= lo1) load_row(row, v);
  };
  float pa[RAW], pb[RAW], oa[RAW], ob[RAW];
#pragma unroll
  for (int c = 0; c < RAW; ++c) pa[c] = pb[c] = oa[c] = ob[c] = 0.f;
  load_row(s_begin, pa);
  load_old(s_begin - R, oa);

  float V1[K][C1], V2[K][C1];
  float V1c[COMP ? K : 1][COMP ? C1 : 1], V2c[COMP ? K : 1][COMP ? C1 : 1];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < C1; ++c) V1[k][c] = V2[k][c] = 0.f;
#pragma unroll
  for (int k = 0; k < (COMP ? K : 1); ++k)
#pragma unroll
    for (int c = 0; c < (COMP ? C1 : 1); ++c) V1c[k][c] = V2c[k][c] = 0.f;
  auto acc1 = [&](int k, int c, float x) {
    if constexpr (COMP) kahan_add(V1[k][c], V1c[COMP ? k : 0][COMP ? c : 0], x);
    else V1[k][c] += x;
  };
  auto acc2 = [&](int k, int c, float x) {
    if constexpr (COMP) kahan_add(V2[k][c], V2c[COMP ? k : 0][COMP ? c : 0], x);
    else V2[k][c] += x;
  };

  // One step per input row s, with the loads of the next step issued at its start (a step is
  // long enough to cover their latency; two buffers each, alternating): cur = row s,
  // nxt <- row s + 1; cur_o = row s - 2r - 1 (leaving stage 1), nxt_o <- row s - 2r, which is
  // also the output row of this step (its guidance is first used at the end of the step).
  auto step = [&](const int s, const float *cur, float *nxt, const float *cur_o,
                  float *nxt_o) {
    if (s >= s_end || failed) return;
    load_row(s + 1, nxt);
    load_old(s + 1 - R, nxt_o);
    const float *mid_o = nxt_o;
    const int y1 = s - r, y2 = s - 2 * r, yo = y1 - R;
    const bool have_c = y1 >= c_lo && y1 < c_hi;  // uniform over the CTA
    const bool have_o = yo >= c_lo && yo < c_hi;  // a coefficient row leaves stage 2
    // the ring entries of the leaving row (written 2r+1 rows ago by this thread: read through
    // L2), fetched before the second scan so that its latency overlaps the scan
    float old[K][C1];
    float *rs = ring + (size_t)((y1 - (Y0 - 3 * r)) % R) * K * C1 * TWo;
    auto fetch_old = [&]() {
      if (out_t && have_o) {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
          for (int c = 0; c < C1; ++c) old[k][c] = ld_l2_hint(rs + (size_t)(k * C1 + c) * TWo, keep);
      }
    };
    // ---- stage 1, vertical: input rows [s - 2r, s]
    if (col_ok) {
      if (s - R >= lo1) {
        float go[NG];
        eval_basis<B>(cur_o, sh, go);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float p = cur_o[NC + k];
          if constexpr (COMP) {
            acc1(k, 0, -p);
#pragma unroll
            for (int i = 0; i < NG; ++i) acc1(k, i + 1, -go[i] * p);
          } else {
            V1[k][0] -= p;
            fma_channels<NG>(V1[k], go, -p);  // fmaf(go, -p, .) == fmaf(-go, p, .)
          }
        }
      }
      if (s >= 0 && s < H) {
        float g[NG];
        eval_basis<B>(cur, sh, g);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float p = cur[NC + k];
          if constexpr (COMP) {
            acc1(k, 0, p);
#pragma unroll
            for (int i = 0; i < NG; ++i) acc1(k, i + 1, g[i] * p);
          } else {
            V1[k][0] += p;
            fma_channels<NG>(V1[k], g, p);
          }
        }
      }
    }
    if (!have_c && y2 < Y0) return;  // stage-1 warm-up rows
    if (!have_c) fetch_old();
    if (have_c) {
      // ---- stage 1, horizontal: window sums over [xi - r, xi + r]
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int c = 0; c < C1; ++c)
          S1[(k * C1 + c) * kRowStride + 4 + t] =
              COMP ? V1[k][c] - V1c[COMP ? k : 0][COMP ? c : 0] : V1[k][c];
      __syncthreads();
      scan_rows<(K * C1 + NT / 32 - 1) / (NT / 32)>(S1, nk * C1);
      if (!mbar_wait(bar, copies & 1u, kWaitLimitNs)) s_fail = 1;
      __syncthreads();
      ++copies;
      if (s_fail) {  // the record copy never completed: report and stop
        if (t == 0) atomicExch(status, 1);
        failed = true;
        return;
      }
      // ---- coefficients at (xi, y1) for the K labels: [b, a_1..a_n] (centred) or
      // [v_0..v_n] (paper form), zero outside the image
      float cf[K][C1];
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int c = 0; c < C1; ++c) cf[k][c] = 0.f;
      if (coef_t) {
        // the record elements sit at compile-time offsets e * BW of rrow; the pointer is made
        // opaque per row of the mat-vec, so that the loads of a row are not hoisted ahead of it
        const float *rrow = recs + (t - r + ro);
        auto opaque = [](const float *q) {
          asm volatile("" : "+l"(q));
          return q;
        };
        if (paper_form) {
          float bs[K][C1];
#pragma unroll
          for (int k = 0; k < K; ++k)
#pragma unroll
            for (int c = 0; c < C1; ++c)
              bs[k][c] = window(S1 + (k * C1 + c) * kRowStride, t - r, r);
#pragma unroll
          for (int i = 0; i < C1; ++i) {
            const float *rr = opaque(rrow);
#pragma unroll
            for (int j = i; j < C1; ++j) {
              const float Mij = rr[tri_index(C1, i, j) * BW];
#pragma unroll
              for (int k = 0; k < K; ++k) {
                cf[k][i] = fmaf(Mij, bs[k][j], cf[k][i]);
                if (j != i) cf[k][j] = fmaf(Mij, bs[k][i], cf[k][j]);
              }
            }
          }
        } else {
          const float invN =
              1.f / (float)(clipped_count(xi, r, W) * clipped_count(y1, r, H));
          float m[NG];
#pragma unroll
          for (int i = 0; i < NG; ++i) m[i] = rrow[i * BW];
          if constexpr (K == 2 && !COMP) {
            // the two labels in packed two-lane arithmetic: window sums, means, cov, the mat-vec
            // and b, with the same roundings in the same order as the scalar branch below
            // (fmaf(-a, m, b) == fmaf(a, -m, b))
            const float2 iN2 = make_float2(invN, invN);
            const float *r0 = S1, *r1 = S1 + C1 * kRowStride;
            const int ia = 4 + (t - r) + 2 * r, ib = 3 + (t - r);
            auto win2 = [&](int c) {
              return sub2(make_float2(r0[c * kRowStride + ia], r1[c * kRowStride + ia]),
                          make_float2(r0[c * kRowStride + ib], r1[c * kRowStride + ib]));
            };
            const float2 pb2 = mul2(win2(0), iN2);
            float2 a2[NG], c2[NG];
#pragma unroll
            for (int i = 0; i < NG; ++i) {
              c2[i] = fma2(make_float2(-m[i], -m[i]), pb2, mul2(win2(i + 1), iN2));
              a2[i] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < NG; ++i) {
              const float *rr = opaque(rrow);
#pragma unroll
              for (int j = i; j < NG; ++j) {
                const float Mij = rr[(NG + tri_index(NG, i, j)) * BW];
                const float2 M2 = make_float2(Mij, Mij);
                a2[i] = fma2(M2, c2[j], a2[i]);
                if (j != i) a2[j] = fma2(M2, c2[i], a2[j]);
              }
            }
            float2 b2 = pb2;
#pragma unroll
            for (int i = 0; i < NG; ++i) {
              b2 = fma2(a2[i], make_float2(-m[i], -m[i]), b2);
              cf[0][i + 1] = a2[i].x;
              cf[1][i + 1] = a2[i].y;
            }
            cf[0][0] = b2.x;
            cf[1][0] = b2.y;
          } else {
            float cov[K][NG], pbar[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const float *row = S1 + k * C1 * kRowStride;
              pbar[k] = window(row, t - r, r) * invN;
#pragma unroll
              for (int i = 0; i < NG; ++i) {
                const float mi = window(row + (i + 1) * kRowStride, t - r, r) * invN;
                cov[k][i] = fmaf(-m[i], pbar[k], mi);
              }
            }
#pragma unroll
            for (int i = 0; i < NG; ++i) {
              const float *rr = opaque(rrow);
#pragma unroll
              for (int j = i; j < NG; ++j) {
                const float Mij = rr[(NG + tri_index(NG, i, j)) * BW];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                  cf[k][i + 1] = fmaf(Mij, cov[k][j], cf[k][i + 1]);
                  if (j != i) cf[k][j + 1] = fmaf(Mij, cov[k][i], cf[k][j + 1]);
                }
              }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
              float b = pbar[k];
#pragma unroll
              for (int i = 0; i < NG; ++i) b = fmaf(-cf[k][i + 1], m[i], b);
              cf[k][0] = b;
            }
          }
        }
      }
      // ---- stage 2, horizontal: the coefficient rows
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int c = 0; c < C1; ++c) S2[(k * C1 + c) * kRowStride + 4 + t] = cf[k][c];
      fetch_old();
      __syncthreads();
      // every thread is past its coefficients: the record box is free for the next row
      if (t == 0 && y1 + 1 < c_hi) tma_load_3d(recs, map, xr, y1 + 1, 0, rec_bytes, bar);
      scan_rows<(K * C1 + NT / 32 - 1) / (NT / 32)>(S2, nk * C1);
      __syncthreads();
    }
    // ---- stage 2, vertical: coefficient rows [y1 - 2r, y1] through this column's ring
    if (!out_t) return;
    if (have_o) {
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int c = 0; c < C1; ++c) acc2(k, c, -old[k][c]);
    }
    if (have_c) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int c = 0; c < C1; ++c) {
          const float hv = window(S2 + (k * C1 + c) * kRowStride, t - r, r);
          st_l2_hint(rs + (size_t)(k * C1 + c) * TWo, hv, keep);
          acc2(k, c, hv);
        }
      }
    }
    if (y2 < Y0) return;
    // ---- output q at (xi, y2) for the K labels, and WTA
    float g[NG];
    eval_basis<B>(mid_o, sh, g);
    const float invN = 1.f / (float)(clipped_count(xi, r, W) * clipped_count(y2, r, H));
    const size_t pix = (size_t)y2 * W + xi;
    unsigned long long klo = ~0ull, khi = ~0ull;  // smallest and second-smallest key
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (k < nk) {
        float wv[C1];
#pragma unroll
        for (int c = 0; c < C1; ++c)
          wv[c] = COMP ? V2[k][c] - V2c[COMP ? k : 0][COMP ? c : 0] : V2[k][c];
        float q = wv[0];
#pragma unroll
        for (int i = 0; i < NG; ++i) q = fmaf(wv[i + 1], g[i], q);
        q *= invN;
        if (filtered) filtered[(size_t)(l0 + k) * HW + pix] = q;
        const unsigned long long key = wta_key(q, l0 + k);
        if (key < klo) {
          khi = klo;
          klo = key;
        } else if (key < khi) {
          khi = key;
        }
      }
    }
    if (keys) {
      if (keys2) {
        // second-smallest key over all labels: every key but the final minimum reaches keys2
        // (the pair's larger key directly; the smaller one or the old minimum, whichever loses)
        const unsigned long long old_min = atomicMin(keys + pix, klo);
        const unsigned long long lose = old_min > klo ? old_min : klo;
        atomicMin(keys2 + pix, lose < khi ? lose : khi);
      } else {
        atomicMin(keys + pix, klo);
      }
    }
  };
  for (int s = s_begin; s < s_end && !failed; s += 2) {
    step(s, pa, pb, oa, ob);
    step(s + 1, pb, pa, ob, oa);
  }
}

template <int B, int K, typename CT, bool COMP>
__global__ void __launch_bounds__(NT, fused_ctas_per_sm(basis_n(B)))
    k_fused(const __grid_constant__ FusedJob jb, const __grid_constant__ CUtensorMap rec_map,
            float *__restrict__ ring_ws, size_t ring_stride, int *status) {
  constexpr int C1 = basis_n(B) + 1, REC = record_floats(basis_n(B));
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ int s_fail;
  FusedCta cta;
  fused_cta_init(cta, smem_raw, REC, K * C1, &s_fail, ring_ws + (size_t)blockIdx.x * ring_stride);
  const long long n_items = (long long)((jb.L + K - 1) / K) * jb.n_strips * jb.n_bands;
  // work items in order label group, strip, band: the CTAs running at one time share a strip
  // and band, and so the record rows they stage, through L2
  for (long long item = blockIdx.x; item < n_items && !cta.failed; item += gridDim.x)
    fused_item<B, K, CT, COMP>(jb, &rec_map, item, cta, status);
}


// Many jobs in one launch (hgf_batch with hgf_tuning.kernel = 1): the persistent CTAs take work
// items of every job from one atomic counter, largest jobs first. Each job's items are processed
// by the same fused_item as when it runs alone, with its own bands, records and outputs, so the
// results do not depend on the mix. The bases are the RGB monomials of degree 1 and 2 (n = 3, 9),
// with float32, bfloat16 or float16 costs; the shared memory is laid out for n = 9.
constexpr int kMaxBatchJobs = kOnepassBatchJobsPerLaunch;
struct FusedBatch {
  CUtensorMap maps[kMaxBatchJobs];           // each job's record tensor map
  FusedJob jobs[kMaxBatchJobs];
  long long item_start[kMaxBatchJobs + 1];   // prefix sums of the jobs' item counts
  int n_jobs;
};

template <int K>
__global__ void __launch_bounds__(NT, kFusedCtasPerSm)
    k_fused_batch(const __grid_constant__ FusedBatch bp, float *__restrict__ ring_ws,
                  size_t ring_stride, unsigned long long *counter, int *status) {
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ int s_fail;
  __shared__ long long s_item;
  FusedCta cta;
  fused_cta_init(cta, smem_raw, record_floats(basis_n(B_RGB_MONO2)),
                 K * (basis_n(B_RGB_MONO2) + 1), &s_fail, ring_ws + (size_t)blockIdx.x * ring_stride);
  const long long total = bp.item_start[bp.n_jobs];
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long item = s_item;
    if (item >= total || cta.failed) break;  // uniform over the CTA
    int j = 0;
    while (j + 1 < bp.n_jobs && bp.item_start[j + 1] <= item) ++j;
    const FusedJob &jb = bp.jobs[j];
    const long long local = item - bp.item_start[j];
    const CUtensorMap *map = &bp.maps[j];
#define HGF_BATCH_CASE(BB, DT, CT) \
  case BB * 4 + DT:                 \
    fused_item<BB, K, CT, false>(jb, map, local, cta, status); \
    break;
    switch (jb.basis * 4 + jb.cost_dtype) {
      HGF_BATCH_CASE(B_RGB_MONO1, HGF_F32, float)
      HGF_BATCH_CASE(B_RGB_MONO1, HGF_BF16, __nv_bfloat16)
      HGF_BATCH_CASE(B_RGB_MONO1, HGF_F16, __half)
      HGF_BATCH_CASE(B_RGB_MONO2, HGF_F32, float)
      HGF_BATCH_CASE(B_RGB_MONO2, HGF_BF16, __nv_bfloat16)
      HGF_BATCH_CASE(B_RGB_MONO2, HGF_F16, __half)
      default:
        break;
    }
#undef HGF_BATCH_CASE
    __syncthreads();  // every thread has read s_item and finished the item's shared rows
  }
}

}  // namespace

// Single-pass aggregation of every label: one persistent launch per call; ring_ws holds
// onepass_ring_bytes(g) bytes.
template <int B>
cudaError_t launch_onepass(const hgf_guidance *g, const void *cost, int cost_dtype, int L,
                           float *filtered, unsigned long long *keys, unsigned long long *keys2,
                           const AggregatePlan &p, int *status, const StereoSource &stereo,
                           const CUtensorMap &map, float *ring_ws, int grid_ctas, cudaStream_t s,
                           Profiler *prof) {
  constexpr int K = kFusedLabels;
  const int H = g->H, W = g->W, r = g->r;
  const int TWo = NT - 4 * r;
  if (TWo < 1 || grid_ctas < 1) return cudaErrorInvalidValue;
  const int strips = (W + TWo - 1) / TWo;
  const size_t sm = onepass_smem(basis_n(B), r);
  cudaError_t e = set_smem(k_fused<B, K, float, false>, sm);
  if (e == cudaSuccess) e = set_smem(k_fused<B, K, __nv_bfloat16, false>, sm);
  if (e == cudaSuccess) e = set_smem(k_fused<B, K, __half, false>, sm);
  if (e == cudaSuccess) e = set_smem(k_fused<B, K, StereoTag, false>, sm);
  if (e == cudaSuccess) e = set_smem(k_fused<B, K, float, true>, sm);
  if (e == cudaSuccess) e = set_smem(k_fused<B, K, __nv_bfloat16, true>, sm);
  if (e == cudaSuccess) e = set_smem(k_fused<B, K, __half, true>, sm);
  if (e == cudaSuccess) e = set_smem(k_fused<B, K, StereoTag, true>, sm);
  if (e != cudaSuccess) return e;
  // bands planned from the nominal label count of the call and the persistent grid (CTAs that
  // run at once), never from the mix of a batch, so that where sums restart depends on the
  // image shape only
  const int rows = p.band_rows > 0
                       ? p.band_rows
                       : choose_band_rows(H, 2 * r, (long long)strips * ((p.nominal + K - 1) / K),
                                          grid_ctas);
  const int bands = (H + rows - 1) / rows;
  const long long items = (long long)((L + K - 1) / K) * strips * bands;
  const int grid = (int)std::min<long long>(grid_ctas, items);
  const int pf = g->form == HGF_FORM_PAPER ? 1 : 0;
  if (prof) {
    const int pl[8] = {1, TWo, NT - 2 * r, rows, rows, K, L, grid};
    for (int i = 0; i < 8; ++i) prof->plan[i] = pl[i];
  }
  FusedJob jb{};
  jb.cost = cost;
  jb.img = g->img;
  jb.shift = g->shift;
  jb.keys = keys;
  jb.keys2 = keys2;
  jb.filtered = filtered;
  jb.H = H;
  jb.W = W;
  jb.r = r;
  jb.L = L;
  jb.band_rows = rows;
  jb.n_strips = strips;
  jb.n_bands = bands;
  jb.paper_form = pf;
  jb.basis = B;
  jb.cost_dtype = cost_dtype;
  jb.stereo = stereo;
  const size_t ring_stride = onepass_ring_bytes(basis_n(B), r, 1) / sizeof(float);
  LaunchScope ls(prof, "k_fused", s);
#define HGF_FUSED(CT, COMP) \
  k_fused<B, K, CT, COMP><<<grid, NT, sm, s>>>(jb, map, ring_ws, ring_stride, status);
#define HGF_FUSED_DT(COMP)                                     \
  switch (cost_dtype) {                                        \
    case HGF_F32: HGF_FUSED(float, COMP) break;                \
    case HGF_BF16: HGF_FUSED(__nv_bfloat16, COMP) break;       \
    case HGF_F16: HGF_FUSED(__half, COMP) break;               \
    case kCostStereo: HGF_FUSED(StereoTag, COMP) break;        \
    default: return cudaErrorInvalidValue;                     \
  }
  if (g->compensated) {
    HGF_FUSED_DT(true)
  } else {
    HGF_FUSED_DT(false)
  }
#undef HGF_FUSED_DT
#undef HGF_FUSED
  return cudaGetLastError();
}

}  // namespace hgf

#define HGF_INSTANTIATE_ONEPASS(B)                                                             \
  template cudaError_t hgf::launch_onepass<B>(                                                 \
      const hgf_guidance *, const void *, int, int, float *, unsigned long long *,             \
      unsigned long long *, const hgf::AggregatePlan &, int *, const hgf::StereoSource &,      \
      const CUtensorMap &, float *, int, cudaStream_t, hgf::Profiler *);
