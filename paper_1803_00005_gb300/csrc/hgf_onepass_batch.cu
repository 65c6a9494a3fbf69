// The single-pass kernel over a whole batch (hgf_batch with hgf_tuning.kernel = 1): one
// persistent launch takes the work items of every eligible job (see k_fused_batch).
#include "hgf_onepass.cuh"

#include <numeric>

namespace hgf {

bool onepass_batch_eligible(const hgf_guidance *g) {
  const int b = basis_id(g->C, g->degree, g->basis);
  return (b == B_RGB_MONO1 || b == B_RGB_MONO2) && !g->compensated && onepass_fits(g);
}

size_t onepass_batch_ring_floats(const hgf_guidance *g) {
  return onepass_ring_bytes(g->n, g->r, 1) / sizeof(float);
}

cudaError_t launch_onepass_batch(const OnepassBatchJob *jobs, int n, float *ring_ws,
                                 size_t ring_stride, int grid_ctas, int band_rows_tuned,
                                 unsigned long long *counters, int *status, cudaStream_t s,
                                 Profiler *prof) {
  constexpr int K = kFusedLabels;
  if (n < 1 || grid_ctas < 1) return cudaErrorInvalidValue;
  const size_t sm = onepass_smem(basis_n(B_RGB_MONO2), 0);
  cudaError_t e = set_smem(k_fused_batch<K>, sm);
  if (e != cudaSuccess) return e;
  struct Prep {
    FusedJob jb;
    CUtensorMap map;
    long long items;
    double item_cost;
  };
  std::vector<Prep> pr(n);
  for (int i = 0; i < n; ++i) {
    const hgf_guidance *g = jobs[i].g;
    const int H = g->H, W = g->W, r = g->r, TWo = NT - 4 * r;
    if (TWo < 1 || ring_stride < onepass_batch_ring_floats(g)) return cudaErrorInvalidValue;
    const int strips = (W + TWo - 1) / TWo;
    // the same bands as the job alone (launch_onepass): from its nominal label count and the
    // persistent grid, never from the batch
    const int rows = band_rows_tuned > 0
                         ? band_rows_tuned
                         : choose_band_rows(H, 2 * r,
                                            (long long)strips * ((jobs[i].nominal + K - 1) / K),
                                            grid_ctas);
    const int bands = (H + rows - 1) / rows;
    Prep &p = pr[i];
    p.jb = FusedJob{};
    p.jb.cost = jobs[i].cost;
    p.jb.img = g->img;
    p.jb.shift = g->shift;
    p.jb.keys = jobs[i].keys;
    p.jb.keys2 = nullptr;
    p.jb.filtered = jobs[i].filtered;
    p.jb.H = H;
    p.jb.W = W;
    p.jb.r = r;
    p.jb.L = jobs[i].L;
    p.jb.band_rows = rows;
    p.jb.n_strips = strips;
    p.jb.n_bands = bands;
    p.jb.paper_form = g->form == HGF_FORM_PAPER ? 1 : 0;
    p.jb.basis = basis_id(g->C, g->degree, g->basis);
    p.jb.cost_dtype = jobs[i].cost_dtype;
    p.items = (long long)((jobs[i].L + K - 1) / K) * strips * bands;
    p.item_cost = (double)(rows + 4 * r) * (g->n + 1) * (g->n + 1);
    e = make_record_map(g, &p.map, kFusedBoxWidth);
    if (e != cudaSuccess) return e;
  }
  // largest items first, so that the last items the CTAs take are the short ones
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return pr[a].item_cost > pr[b].item_cost; });
  for (int c0 = 0, chunk = 0; c0 < n; c0 += kMaxBatchJobs, ++chunk) {
    FusedBatch bp{};
    bp.n_jobs = std::min(kMaxBatchJobs, n - c0);
    bp.item_start[0] = 0;
    for (int k = 0; k < bp.n_jobs; ++k) {
      const Prep &p = pr[order[c0 + k]];
      bp.maps[k] = p.map;
      bp.jobs[k] = p.jb;
      bp.item_start[k + 1] = bp.item_start[k] + p.items;
    }
    const int grid = (int)std::min<long long>(grid_ctas, bp.item_start[bp.n_jobs]);
    if (prof) {
      const int pl[8] = {1, 0, 0, 0, 0, K, 0, grid};
      for (int i = 0; i < 8; ++i) prof->plan[i] = pl[i];
    }
    LaunchScope ls(prof, "k_fused_batch", s);
    k_fused_batch<K><<<grid, NT, sm, s>>>(bp, ring_ws, ring_stride, counters + chunk, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace hgf
