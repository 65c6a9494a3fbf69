"""CPU checks of the device-memory layouts the fused kernels index, on the library's own code.

The coefficient workspace (one plane per label, tiled by 32 pixels: coef_pair_index,
coef_plane_floats), the plane-major inverse records (record_pitch, record_total_floats) and the
boxes the strip kernels stage from them by tensor copies (record_box_width) are computed by
host-and-device inline functions of the CUDA sources. This test compiles those
functions into a small host program with nvcc (no GPU is used) and checks, over many image sizes,
basis sizes and radii, that every index the kernels form is inside the buffer the host sizes for
it and that no two records share a slot: a layout mistake here would be an out-of-bounds write on
the GPU, so it is caught before any kernel runs."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1803_00005_gb300", "csrc")

PROGRAM = r"""
#include "hgf_internal.cuh"
#include <cstdio>
#include <vector>

using namespace hgf;

static int fail(const char *what, int n, size_t H, size_t W) {
  std::printf("FAIL %s n=%d H=%zu W=%zu\n", what, n, H, W);
  return 1;
}

int main() {
  const int ns[] = {1, 2, 3, 5, 9, 19};
  const size_t shapes[][2] = {{1, 1}, {1, 31}, {1, 32}, {1, 33}, {3, 7}, {48, 64}, {17, 1031},
                              {375, 450}, {5, 1400}, {2, 4099}};
  for (int n : ns) {
    const int CP = coef_floats(n);
    if (CP % 2 || CP < n + 1) return fail("coef_floats", n, 0, 0);
    for (auto &hw : shapes) {
      const size_t H = hw[0], W = hw[1], HW = H * W;
      const size_t plane = coef_plane_floats(n, HW);
      if (plane % 2 || plane < HW * CP || plane > (HW + 31) * CP) return fail("plane", n, H, W);
      // two labels of a chunk, as the kernels address them: label k at k * plane floats
      const int chunk = 2;
      std::vector<unsigned char> used(chunk * plane / 2, 0);
      for (int k = 0; k < chunk; ++k)
        for (size_t p = 0; p < HW; ++p)
          for (int q = 0; q < CP / 2; ++q) {
            const size_t i = (size_t)k * plane / 2 + coef_pair_index(n, p, q);
            if (i >= used.size()) return fail("coef index out of range", n, H, W);
            if (used[i]++) return fail("coef index collision", n, H, W);
          }
      // a warp's 32 consecutive pixels of one row touch at most two tiles per pair
      for (size_t y = 0; y < H; ++y)
        for (size_t x0 = 0; x0 < W; x0 += 7) {
          const size_t p0 = y * W + x0, p1 = y * W + std::min(W, x0 + 32) - 1;
          if ((p1 >> 5) - (p0 >> 5) > 1) return fail("warp spans more than two tiles", n, H, W);
        }
    }
  }
  // plane-major inverse records: element e of (x, y) at (e * H + y) * P + x, P = record_pitch(W)
  for (int n : {1, 3, 9, 19}) {
    const int REC = record_floats(n);
    if (REC % 4) return fail("record_floats", n, 0, 0);
    for (auto &hw : shapes) {
      const size_t H = hw[0], W = hw[1], P = record_pitch((int)W);
      if (P < W || P % 4 || P >= W + 4) return fail("record pitch", n, H, W);
      const size_t total = record_total_floats((int)H, (int)W, n);
      std::vector<unsigned char> used(total, 0);
      for (int e = 0; e < REC; ++e)
        for (size_t y = 0; y < H; ++y) {
          // every row of every element plane starts 16-byte aligned (the tensor map's strides)
          if ((((size_t)e * H + y) * P * sizeof(float)) % 16) return fail("row alignment", n, H, W);
          for (size_t x = 0; x < W; ++x) {
            const size_t i = ((size_t)e * H + y) * P + x;
            if (i >= total) return fail("record index out of range", n, H, W);
            if (used[i]++) return fail("record index collision", n, H, W);
          }
        }
    }
  }
  // staged record boxes: both strip kernels load columns [xr, xr + BW) of one row with xr a
  // multiple of 4; every coefficient column a thread reads lies in the box, at a box index < BW
  for (int r : {0, 1, 4, 9, 20, 24, 40, 63}) {
    const int BW = record_box_width(r), TW = kStripThreads - 2 * r;
    if (BW % 4 || BW > 256 || BW < TW + 3) return fail("box width", r, 0, 0);
    for (auto &hw : shapes) {
      const long W = (long)hw[1];
      // k_coef: strip s, coefficient columns x0 + t for t < TW, box index t + ro
      for (long x0 = 0; x0 < W; x0 += TW) {
        const long xr = x0 & ~3L, ro = x0 - xr;
        if (xr % 4 || ro < 0 || ro > 3) return fail("k_coef box origin", r, 0, (size_t)W);
        for (long t = 0; t < TW; ++t)
          if (t + ro >= BW || x0 + t < xr || x0 + t >= xr + BW) return fail("k_coef box", r, 0, W);
      }
      // k_fused: output strip of 128 - 4r columns at x0; coefficient columns x0 - 2r + t for
      // t in [r, 128 - r), box index t - r + ro, in a box kFusedBoxWidth wide
      const int TWo = kStripThreads - 4 * r;
      if (kFusedBoxWidth < BW || kFusedBoxWidth % 4 || kFusedBoxWidth > 256)
        return fail("k_fused box width", r, 0, W);
      if (TWo < 32) continue;
      for (long x0 = 0; x0 < W; x0 += TWo) {
        const long c0 = x0 - r, xr = c0 & ~3L, ro = c0 - xr;
        if (((xr % 4) + 4) % 4 || ro < 0 || ro > 3) return fail("k_fused box origin", r, 0, W);
        for (long t = r; t < kStripThreads - r; ++t) {
          const long x = x0 - 2 * r + t, j = t - r + ro;
          if (j < 0 || j >= kFusedBoxWidth || x != xr + j) return fail("k_fused box", r, 0, W);
        }
      }
    }
  }
  std::printf("ok\n");
  return 0;
}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_layout_indices_in_bounds_and_distinct(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src, exe = tmp_path / "layout.cu", tmp_path / "layout"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
