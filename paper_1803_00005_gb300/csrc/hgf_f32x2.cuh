// Packed two-lane float32 arithmetic (fma.rn.f32x2 / add.rn.f32x2, sm_100 and later): one
// instruction does two IEEE round-to-nearest operations, so results are bit-identical to two
// fmaf / __fadd_rn calls while the issue slots they take halve. The strip kernels are bound by
// instruction issue, and they pair the two labels of a pass (or two channels of one label) this
// way.
#pragma once
#include <cuda_runtime.h>

namespace hgf {

// (a.x * b.x + c.x, a.y * b.y + c.y), each rounded once
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// (a.x + b.x, a.y + b.y), each rounded once
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

}  // namespace hgf

namespace hgf {

// v[1..n] += g[0..n-1] * p for one label's vertical running sums, channel pairs packed; the same
// rounding as v[i + 1] = fmaf(g[i], p, v[i + 1]) for each i.
template <int N>
__device__ __forceinline__ void fma_channels(float *v, const float *g, float p) {
  const float2 pp = make_float2(p, p);
#pragma unroll
  for (int i = 0; i + 1 < N; i += 2) {
    const float2 r = fma2(make_float2(g[i], g[i + 1]), pp, make_float2(v[i + 1], v[i + 2]));
    v[i + 1] = r.x;
    v[i + 2] = r.y;
  }
  if (N % 2) v[N] = fmaf(g[N - 1], p, v[N]);
}

}  // namespace hgf

namespace hgf {

// (a.x - b.x, a.y - b.y), each rounded once
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// (a.x * b.x, a.y * b.y), each rounded once
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

}  // namespace hgf
