// Per-pixel front-to-back blend step (Sec. 3.4 rules of 3DGS): support
// q <= 9, alpha = min(0.99, o exp(-q/2)), skip alpha < 1/255, stop before
// T (1 - alpha) < 1e-4.  q is evaluated as the sum of squares of the
// prescaled Cholesky factors (Sec. 3.5), e = (l0 dx + l1 dy)^2 + (l2 dy)^2 =
// q log2(e) / 2, so alpha = o exp2(-e).  Every kernel that blends (forward
// raster, merge replay, plain path, backward replay) uses these functions, so
// the same gaussian at the same pixel gives the same bits everywhere.  The
// decisions are written as saturated multiply-adds, which keeps the inner
// loop off the integer/compare pipe.
#pragma once
#include "common.cuh"

namespace hg {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Pixel state.  T is the live transmittance: it is 0 once the pixel has
// stopped (and for pixels outside the image), so later gaussians add nothing;
// Ts is the transmittance at the stop (0 while the pixel is live).  The final
// transmittance is T + Ts (one of the two is 0).
struct PixelAcc {
  float r, g, b, T, Ts;
};

__device__ __forceinline__ void pixel_init(PixelAcc& p, bool inside, float t_in = 1.f) {
  p.r = p.g = p.b = 0.f;
  p.T = inside ? t_in : 0.f;
  p.Ts = 0.f;
}

__device__ __forceinline__ bool pixel_live(const PixelAcc& p) { return p.T > 0.f; }
__device__ __forceinline__ float pixel_final_T(const PixelAcc& p) { return p.T + p.Ts; }

// Stored per-pixel state (per-tile chain state, partials, saved prefixes):
// {r, g, b, w} with w = T while live and -Ts once stopped.
__device__ __forceinline__ float4 pixel_state(const PixelAcc& p) {
  return make_float4(p.r, p.g, p.b, p.T > 0.f ? p.T : -p.Ts);
}
__device__ __forceinline__ void pixel_load(PixelAcc& p, bool inside, const float4& s) {
  p.r = s.x;
  p.g = s.y;
  p.b = s.z;
  const bool st = signbit(s.w);
  p.T = inside && !st ? s.w : 0.f;
  p.Ts = st ? -s.w : 0.f;
}

// Blend test and alpha of gaussian (g0 = {mx, my, l0', l1'}, g1 = {l2', o, ., .},
// g2 = {r, g, b, E}) at pixel offset dy from its centre, ubase = l0' dx:
// e = (l0' dx + l1' dy)^2 + (l2' dy)^2 = q log2(e) / 2 and alpha =
// min(0.99, o 2^-e).  The support q <= 9 and alpha >= 1/255 together are
// e <= E with E = min(9 log2(e) / 2, log2(255 o)) (stored per gaussian).
// Returns alpha, or 0 when the gaussian fails the test; raw = o 2^-e.
// The test is the sign of E - e scaled by 2^64 and saturated (a multiply-add,
// not a compare-select): exact whenever E and e differ by at least 2^-64.
__device__ __forceinline__ float alpha_of(float ubase, float dy, const float4& g0, const float4& g1,
                                          const float4& g2, float& raw) {
  const float u = fmaf(g0.w, dy, ubase);
  const float w = g1.x * dy;
  const float e = fmaf(u, u, w * w);
  raw = g1.y * ex2_approx(-e);
  const float f = __saturatef(fmaf(g2.w - e, 18446744073709551616.f, 1.f));
  return fminf(ALPHA_MAX, raw) * f;
}

// Ordered update with the alpha from alpha_of: T' = T - alpha T; the pixel
// stops before T' < 1e-4 (that gaussian excluded).  The stop test is the
// sign of T' - 1e-4 scaled by 2^40 and saturated: exact, since two distinct
// floats near 1e-4 differ by at least 2^-37.  Returns the gaussian's weight
// alpha T (0 when it did not contribute).
__device__ __forceinline__ float apply_alpha(PixelAcc& p, float al, const float4& g2) {
  const float aT = al * p.T;
  const float tn = p.T - aT;
  const float dt = tn - T_EPS;
  const float s = __saturatef(fmaf(dt, 1099511627776.f, 1.f));  // 1: keeps going
  const float ns = __saturatef(dt * -1099511627776.f);           // 1: stops (or stopped)
  const float wt = aT * s;
  p.r = fmaf(g2.x, wt, p.r);
  p.g = fmaf(g2.y, wt, p.g);
  p.b = fmaf(g2.z, wt, p.b);
  p.Ts = fmaf(ns, p.T, p.Ts);
  p.T = tn * s;
  return wt;
}

__device__ __forceinline__ void blend(PixelAcc& p, float ubase, float dy, const float4& g0, const float4& g1,
                                      const float4& g2) {
  float raw;
  apply_alpha(p, alpha_of(ubase, dy, g0, g1, g2, raw), g2);
}

// Per-gaussian level E of the blend test (stored in the record's g2.w).
__device__ __forceinline__ float blend_level(float o) { return fminf(SUPPORT_E, log2f(255.f * o)); }

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
