// Per-pixel front-to-back blend step (Sec. 3.4 rules of 3DGS): support
// q <= 9, alpha = min(0.99, o exp(-q/2)), skip alpha < 1/255, stop before
// T (1 - alpha) < 1e-4.  q is evaluated as the sum of squares of the
// prescaled Cholesky factors (Sec. 3.5), e = (l0 dx + l1 dy)^2 + (l2 dy)^2 =
// q log2(e) / 2, so alpha = o exp2(-e).
#pragma once
#include "common.cuh"

namespace hg {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct PixelAcc {
  float r, g, b, T;
  bool done;      // stopped (or outside the image)
  bool stopped;   // stopped by the termination rule
};

__device__ __forceinline__ void pixel_init(PixelAcc& p, bool inside, float t_in = 1.f) {
  p.r = p.g = p.b = 0.f;
  p.T = t_in;
  p.done = !inside;
  p.stopped = false;
}

// One gaussian (g0 = {mx, my, l0', l1'}, g1 = {l2', o, ., .}, g2 = {r, g, b, .})
// at pixel offset (dx, dy) from its centre.  Returns true if the pixel
// stopped at this gaussian.
__device__ __forceinline__ bool blend_one(PixelAcc& p, float ubase, float dy, const float4& g0, const float4& g1,
                                          const float4& g2) {
  if (p.done) return false;
  const float u = fmaf(g0.w, dy, ubase);
  const float w = g1.x * dy;
  const float e = fmaf(u, u, w * w);
  if (e > SUPPORT_E) return false;
  const float al = fminf(ALPHA_MAX, g1.y * ex2_approx(-e));
  if (al < ALPHA_MIN) return false;
  const float tn = p.T * (1.f - al);
  if (tn < T_EPS) {
    p.done = true;
    p.stopped = true;
    return true;
  }
  const float wt = al * p.T;
  p.r = fmaf(g2.x, wt, p.r);
  p.g = fmaf(g2.y, wt, p.g);
  p.b = fmaf(g2.z, wt, p.b);
  p.T = tn;
  return false;
}

// Branch-free form of blend_one with the same arithmetic (so every kernel
// that blends the same gaussian at the same pixel gets the same bits).
__device__ __forceinline__ bool blend_bf(PixelAcc& p, float ubase, float dy, const float4& g0, const float4& g1,
                                         const float4& g2) {
  const float u = fmaf(g0.w, dy, ubase);
  const float w = g1.x * dy;
  const float e = fmaf(u, u, w * w);
  const float al = fminf(ALPHA_MAX, g1.y * ex2_approx(-e));
  const bool ok = !p.done && (e <= SUPPORT_E) && (al >= ALPHA_MIN);
  const float tn = p.T * (1.f - al);
  const bool stop = ok && (tn < T_EPS);
  const bool contrib = ok && !stop;
  const float wt = contrib ? al * p.T : 0.f;
  p.r = fmaf(g2.x, wt, p.r);
  p.g = fmaf(g2.y, wt, p.g);
  p.b = fmaf(g2.z, wt, p.b);
  p.T = contrib ? tn : p.T;
  p.done = p.done || stop;
  p.stopped = p.stopped || stop;
  return stop;
}

// blend_bf split in two: the alpha of a gaussian at a pixel does not depend
// on the pixel's transmittance, so several gaussians' alphas can be computed
// independently (instruction-level parallelism) before the ordered updates.
// Together they perform exactly the operations of blend_bf.
__device__ __forceinline__ float alpha_of(float ubase, float dy, const float4& g0, const float4& g1, bool& ok) {
  const float u = fmaf(g0.w, dy, ubase);
  const float w = g1.x * dy;
  const float e = fmaf(u, u, w * w);
  const float al = fminf(ALPHA_MAX, g1.y * ex2_approx(-e));
  ok = (e <= SUPPORT_E) && (al >= ALPHA_MIN);
  return al;
}

// alpha_of that also returns the unclamped o 2^-e (for the backward).
__device__ __forceinline__ float alpha_raw_of(float ubase, float dy, const float4& g0, const float4& g1, bool& ok,
                                              float& raw) {
  const float u = fmaf(g0.w, dy, ubase);
  const float w = g1.x * dy;
  const float e = fmaf(u, u, w * w);
  raw = g1.y * ex2_approx(-e);
  const float al = fminf(ALPHA_MAX, raw);
  ok = (e <= SUPPORT_E) && (al >= ALPHA_MIN);
  return al;
}

__device__ __forceinline__ bool apply_alpha(PixelAcc& p, float al, bool ok_in, const float4& g2) {
  const bool ok = !p.done && ok_in;
  const float tn = p.T * (1.f - al);
  const bool stop = ok && (tn < T_EPS);
  const bool contrib = ok && !stop;
  const float wt = contrib ? al * p.T : 0.f;
  p.r = fmaf(g2.x, wt, p.r);
  p.g = fmaf(g2.y, wt, p.g);
  p.b = fmaf(g2.z, wt, p.b);
  p.T = contrib ? tn : p.T;
  p.done = p.done || stop;
  p.stopped = p.stopped || stop;
  return stop;
}

// Largest prescaled q a pixel can have and still pass the blend test:
// alpha >= 1/255 needs o 2^-e >= 1/255, i.e. e <= log2(255 o), and the
// support is e <= SUPPORT_E.  Slightly enlarged so that float32 rounding in
// the blend can never pass a pixel this level excludes; negative = nothing.
__device__ __forceinline__ float support_level(float o) {
  if (!(o >= ALPHA_MIN)) return -1.f;
  const float lv = fminf(SUPPORT_E, log2f(255.f * o));
  return lv * 1.0001f + 1e-4f;
}

// x-range (pixel-centre coordinates) covered by the ellipse
// (l0 dx + l1 dy)^2 + (l2 dy)^2 <= E over the rows y in [ya, yb]; false if
// the rows miss it.  The left edge -(l1 dy + s(dy)) / l0 is convex in dy and
// the right edge concave, so their extremes lie at the band's ends or at the
// ellipse's leftmost / rightmost points.  Widened by 0.01 px.
__device__ __forceinline__ bool ellipse_row_span(const float4& g0, const float4& g1, float E, float ya, float yb,
                                                 float& xl, float& xr) {
  const float l0 = g0.z, l1 = g0.w, l2 = g1.x;
  if (!(l0 > 0.f) || !(l2 > 0.f)) {  // degenerate factors: keep the whole band
    xl = -1e6f;
    xr = 1e6f;
    return true;
  }
  const float sE = sqrtf(E);
  const float hy = sE / l2;
  const float a = fmaxf(ya - g0.y, -hy), b = fminf(yb - g0.y, hy);
  if (a > b) return false;
  const float il0 = 1.f / l0;
  const float nrm = sqrtf(fmaf(l1, l1, l2 * l2));
  const float dyl = l1 * sE / (l2 * nrm);  // leftmost point of the ellipse
  auto half = [&](float dy) { return sqrtf(fmaxf(0.f, fmaf(-(l2 * dy), l2 * dy, E))); };
  float lo = fminf((-l1 * a - half(a)) * il0, (-l1 * b - half(b)) * il0);
  float hi = fmaxf((-l1 * a + half(a)) * il0, (-l1 * b + half(b)) * il0);
  if (dyl >= a && dyl <= b) lo = fminf(lo, (-l1 * dyl - half(dyl)) * il0);
  if (-dyl >= a && -dyl <= b) hi = fmaxf(hi, (l1 * dyl + half(-dyl)) * il0);
  xl = fmaxf(g0.x + lo - 0.01f, -1e6f);
  xr = fminf(g0.x + hi + 0.01f, 1e6f);
  return xl <= xr;
}

// Conservative test of a gaussian's 3-sigma rectangle against render tile
// (tx, ty) (same integer rule as the macro binning, at 8x8 granularity).
__device__ __forceinline__ void tile_rect(const float4& g0, const float4& g1, int& x0, int& x1, int& y0, int& y1) {
  const int rad = __float_as_int(g1.z);
  const int px = (int)floorf(g0.x), py = (int)floorf(g0.y);
  x0 = floordiv(px - rad, TILE);
  x1 = floordiv(px + rad, TILE);
  y0 = floordiv(py - rad, TILE);
  y1 = floordiv(py + rad, TILE);
}

}  // namespace hg
