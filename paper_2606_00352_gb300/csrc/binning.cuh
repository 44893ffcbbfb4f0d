// Gaussian-to-macro-tile binning test (Sec. 3.2, 4.3), evaluated once per
// (view, gaussian) where the record is made (projection, or the conversion
// of precomputed splats) and stored as a compact binning record that the
// count and fill passes walk:
//   uint4 {x0 | y0 << 16, x1 | y1 << 16, mask bits 0-31, mask bits 32-63}
// [x0, x1] x [y0, y1] is the gaussian's 3-sigma rectangle in macro cells
// (empty when x0 > x1); the mask has bit (y - y0) * nx + (x - x0) for every
// kept cell.  Rectangles of more than 64 cells keep every cell.
#pragma once
#include "common.cuh"

namespace hg {

constexpr int BIN_CLASSIC = 0;  // {mx, my, radius, key} (plain path)
constexpr int BIN_CELLS_RECT = 1;
constexpr int BIN_CELLS_ELLIPSE = 2;

// bw and bh, the macro cell's size in pixels, are powers of two (macro
// tiles of 4 or 8 render tiles of 8 pixels), so the cell of a pixel
// coordinate is an arithmetic shift (the floor for negative coordinates too).
__device__ __forceinline__ bool macro_rect(int px, int py, int rad, int bw, int bh, int gx, int gy, int& x0, int& x1,
                                           int& y0, int& y1) {
  if (rad <= 0) return false;
  const int xl = px - rad, xh = px + rad, yl = py - rad, yh = py + rad;
  const int sw = 31 - __clz(bw), sh = 31 - __clz(bh);
  x0 = xl < 0 ? 0 : xl >> sw;
  x1 = xh < 0 ? -1 : min(xh >> sw, gx - 1);
  y0 = yl < 0 ? 0 : yl >> sh;
  y1 = yh < 0 ? -1 : min(yh >> sh, gy - 1);
  return x0 <= x1 && y0 <= y1;
}

// Ellipse test, every operation rounded to float32 as written (no
// contraction), so the pairs are reproducible bit for bit:
//   level  E = min(9 log2(e) / 2, lb(255 o)) + 2^-12, lb(z) = k + (B m + A)
//          from z = m 2^k, m in [0.5, 1) (A = -475/256, B = 123/64: a line
//          above log2 on [0.5, 1]), an upper bound of the blend-test level
//   band   rows [ya, yb]: the x extremes of the ellipse
//          (L0 dx + L1 dy)^2 + (L2 dy)^2 <= E over the band's part of
//          [-hy, hy], at the leftmost / rightmost point when the band holds
//          it, else at the band end nearer to it, widened by
//          2^-6 + 2^-10 |offset| pixels
constexpr float ELL_A = -475.f / 256.f;
constexpr float ELL_B = 123.f / 64.f;
constexpr float ELL_MARGIN_E = 1.f / 4096.f;
constexpr float ELL_PAD = 1.f / 64.f;
constexpr float ELL_REL = 1.f / 1024.f;
constexpr float ELL_LIM = 1073741824.f;  // 2^30

__device__ __forceinline__ float ell_level(float o) {
  const float z = __fmul_rn(255.f, o);
  int k;
  const float m = frexpf(z, &k);
  const float lb = __fadd_rn((float)k, __fadd_rn(__fmul_rn(ELL_B, m), ELL_A));
  return __fadd_rn(fminf(SUPPORT_E, lb), ELL_MARGIN_E);
}

__device__ __forceinline__ float ell_half(float L2, float E, float dy) {
  const float t = __fmul_rn(L2, dy);
  return __fsqrt_rn(fmaxf(0.f, __fsub_rn(E, __fmul_rn(t, t))));
}

// Per-gaussian part of the ellipse test (L0, L2 > 0): the y half-extent hy
// (and hy widened), the leftmost point dyl with its x offset xl_ext (the
// rightmost is at -dyl, offset xr_ext), reciprocals of L0.
struct EllGauss {
  float E, hy, hyw, dyl, x_l, x_r, iL0;
};

__device__ __forceinline__ EllGauss ell_gauss(float L0, float L1, float L2, float E) {
  EllGauss g;
  g.E = fmaxf(E, 0.f);
  const float sE = __fsqrt_rn(g.E);
  g.iL0 = __fdiv_rn(1.f, L0);
  const float iL2 = __fdiv_rn(1.f, L2);
  g.hy = __fmul_rn(sE, iL2);
  g.hyw = __fadd_rn(__fmul_rn(g.hy, 1.f + ELL_REL), ELL_PAD);
  const float nrm = __fsqrt_rn(__fadd_rn(__fmul_rn(L1, L1), __fmul_rn(L2, L2)));
  g.dyl = __fdiv_rn(__fmul_rn(L1, sE), __fmul_rn(L2, nrm));
  const float h = ell_half(L2, g.E, g.dyl);
  const float t = __fmul_rn(-L1, g.dyl);
  g.x_l = __fmul_rn(__fsub_rn(t, h), g.iL0);
  g.x_r = __fmul_rn(__fadd_rn(__fmul_rn(L1, g.dyl), h), g.iL0);
  return g;
}

// x span of the ellipse over rows [ya, yb]; false when the band misses it.
// The left edge (-L1 dy - h(dy)) / L0 is convex in dy: over the band's part
// [a, b] of [-hy, hy] its minimum is at dyl when dyl is in [a, b], else at
// the end nearer to dyl (the right edge likewise with -dyl).
__device__ __forceinline__ bool ell_span(const EllGauss& g, float mx, float my, float L1, float L2, float ya,
                                         float yb, bool live, float& xl, float& xr) {
  const float ra = __fsub_rn(ya, my), rb = __fsub_rn(yb, my);
  if (!live || !(fmaxf(ra, -g.hyw) <= fminf(rb, g.hyw))) return false;
  float a = fmaxf(ra, -g.hy), b = fminf(rb, g.hy);
  if (!(a <= b)) a = b = rb < -g.hy ? -g.hy : g.hy;  // meets only the widened range: the tip
  const float nL1 = -L1;
  float lo, hi;
  if (g.dyl >= a && g.dyl <= b) {
    lo = g.x_l;
  } else {
    const float d = g.dyl < a ? a : b;
    lo = __fmul_rn(__fsub_rn(__fmul_rn(nL1, d), ell_half(L2, g.E, d)), g.iL0);
  }
  if (-g.dyl >= a && -g.dyl <= b) {
    hi = g.x_r;
  } else {
    const float d = -g.dyl < a ? a : b;
    hi = __fmul_rn(__fadd_rn(__fmul_rn(nL1, d), ell_half(L2, g.E, d)), g.iL0);
  }
  xl = __fsub_rn(__fadd_rn(mx, lo), __fadd_rn(__fmul_rn(fabsf(lo), ELL_REL), ELL_PAD));
  xr = __fadd_rn(__fadd_rn(mx, hi), __fadd_rn(__fmul_rn(fabsf(hi), ELL_REL), ELL_PAD));
  xl = fminf(fmaxf(xl, -ELL_LIM), ELL_LIM);
  xr = fminf(fmaxf(xr, -ELL_LIM), ELL_LIM);
  return true;
}

// Binning record of one (view, gaussian): the rectangle in macro cells of
// bw x bh pixels on a gx x gy grid, refined by the ellipse test for
// rectangles of 2..64 cells when `ellipse` (Gaussians with degenerate
// factors keep the rectangle).
__device__ __forceinline__ uint4 bin_cells(float mx, float my, int rad, float L0, float L1, float L2, float o,
                                           int bw, int bh, int gx, int gy, bool ellipse) {
  int x0, x1, y0, y1;
  if (!macro_rect((int)floorf(mx), (int)floorf(my), rad, bw, bh, gx, gy, x0, x1, y0, y1))
    return make_uint4(1u, 0u, 0u, 0u);  // x0 = 1 > x1 = 0: empty
  const int nx = x1 - x0 + 1, ny = y1 - y0 + 1, cells = nx * ny;
  const uint4 head = make_uint4((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16), 0u, 0u);
  if (cells > 64) return make_uint4(head.x, head.y, 0xffffffffu, 0xffffffffu);
  unsigned long long m = cells == 64 ? ~0ull : ((1ull << cells) - 1ull);
  if (ellipse && cells > 1 && L0 > 0.f && L2 > 0.f) {
    const float E = ell_level(o);
    const EllGauss g = ell_gauss(L0, L1, L2, E);
    m = 0;
    for (int y = y0; y <= y1; ++y) {
      float xl, xr;
      if (!ell_span(g, mx, my, L1, L2, (float)(y * bh), (float)(y * bh + bh - 1), E > 0.f, xl, xr)) continue;
      const int sw = 31 - __clz(bw);
      const int c0 = max(x0, (int)ceilf(xl) >> sw);
      const int c1 = min(x1, (int)floorf(xr) >> sw);
      if (c0 > c1) continue;
      m |= ((1ull << (c1 - c0 + 1)) - 1ull) << ((y - y0) * nx + (c0 - x0));
    }
  }
  return make_uint4(head.x, head.y, (uint32_t)m, (uint32_t)(m >> 32));
}

// Calls fn(cell) for every cell of a binning record (cell = y * gx + x).
template <class Fn>
__device__ __forceinline__ void for_each_cell(const uint4& b, int gx, Fn fn) {
  const int x0 = (int)(b.x & 0xffffu), y0 = (int)(b.x >> 16), x1 = (int)(b.y & 0xffffu), y1 = (int)(b.y >> 16);
  if (x0 > x1) return;
  const int nx = x1 - x0 + 1, ny = y1 - y0 + 1;
  if (nx * ny > 64) {
    for (int y = y0; y <= y1; ++y)
      for (int x = x0; x <= x1; ++x) fn(y * gx + x);
    return;
  }
  unsigned long long m = (unsigned long long)b.z | ((unsigned long long)b.w << 32);
  while (m) {
    const int k = __ffsll((long long)m) - 1;
    m &= m - 1;
    fn((y0 + k / nx) * gx + x0 + k % nx);
  }
}

}  // namespace hg
