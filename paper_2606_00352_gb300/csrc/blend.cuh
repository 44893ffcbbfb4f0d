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
#include <cuda_fp16.h>

#include "common.cuh"

namespace hg {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Pixel state.  T is the live transmittance: it is 0 once the pixel has
// stopped (and for pixels outside the image), so later gaussians add nothing;
// U is the final transmittance: equal to T (bit for bit) while the pixel is
// live, frozen at the transmittance of the stop afterwards.
struct PixelAcc {
  float r, g, b, T, U;
};

__device__ __forceinline__ void pixel_init(PixelAcc& p, bool inside, float t_in = 1.f) {
  p.r = p.g = p.b = 0.f;
  p.T = inside ? t_in : 0.f;
  p.U = p.T;
}

__device__ __forceinline__ bool pixel_live(const PixelAcc& p) { return p.T > 0.f; }
__device__ __forceinline__ float pixel_final_T(const PixelAcc& p) { return p.U; }

// Stored per-pixel state (per-tile chain state, partials, saved prefixes):
// {r, g, b, w} with w = T while live and -U once stopped.
__device__ __forceinline__ float4 pixel_state(const PixelAcc& p) {
  return make_float4(p.r, p.g, p.b, p.T > 0.f ? p.T : -p.U);
}
__device__ __forceinline__ void pixel_load(PixelAcc& p, bool inside, const float4& s) {
  p.r = s.x;
  p.g = s.y;
  p.b = s.z;
  const bool st = signbit(s.w);
  p.T = inside && !st ? s.w : 0.f;
  p.U = st ? -s.w : p.T;
}

// Blend test and alpha of gaussian (g0 = {mx, my, l0', l1'}, g1 = {l2', o, ., .},
// g2 = {r, g, b, E''}) at pixel offset dy from its centre, ubase = l0' dx:
// e = (l0' dx + l1' dy)^2 + (l2' dy)^2 = q log2(e) / 2 and alpha =
// min(0.99, o 2^-e).  The support q <= 9 and alpha >= 1/255 together are
// e <= E with E = min(9 log2(e) / 2, log2(255 o)) per gaussian.  The record
// stores E'' = E' 2^64 with E' the next float above max(E, 2^-40)
// (blend_level), and the test is one saturated multiply-add, (E' - e) 2^64:
// E' - E >= 2^-63, so it is >= 2 (1 after saturation) when e <= E and <= 0
// when e >= E', and no float lies between E and E'.  (Only for E < 2^-40,
// alpha within a factor 2^(2^-40) of 1/255, does it accept e up to 2^-40.)
// Returns alpha, or 0 when the gaussian fails the test; raw = o 2^-e.
// alpha_terms also returns ex = 2^-e, the derivative of raw with respect to
// the opacity (the backward's d alpha / d o).
__device__ __forceinline__ float alpha_terms(float ubase, float dy, const float4& g0, const float4& g1,
                                             const float4& g2, float& raw, float& ex) {
  const float u = fmaf(g0.w, dy, ubase);
  const float w = g1.x * dy;
  const float e = fmaf(u, u, w * w);
  ex = ex2_approx(-e);
  raw = g1.y * ex;
  const float f = __saturatef(fmaf(e, -18446744073709551616.f, g2.w));
  return fminf(ALPHA_MAX, raw) * f;
}
__device__ __forceinline__ float alpha_of(float ubase, float dy, const float4& g0, const float4& g1,
                                          const float4& g2, float& raw) {
  float ex;
  return alpha_terms(ubase, dy, g0, g1, g2, raw, ex);
}

// Per-gaussian level of the blend test as the record stores it (g2.w):
// E'' = E' 2^64 with E = min(SUPPORT_E, log2(255 o)) and E' the next float
// above max(E, 2^-40); a negative E (a gaussian that never passes) is stored
// as E 2^64.  record_level recovers E' (exact: a power-of-two scale).
__device__ __forceinline__ float blend_level(float o) {
  const float E = fminf(SUPPORT_E, log2f(255.f * o));
  const float Ep = E >= 0.f ? nextafterf(fmaxf(E, 9.094947017729282e-13f), INFINITY) : E;
  return Ep * 18446744073709551616.f;
}
__device__ __forceinline__ float record_level(const float4& g2) { return g2.w * 5.421010862427522e-20f; }

// Ordered update with the alpha from alpha_of: T' = T - alpha T; the pixel
// stops before T' < 1e-4 (that gaussian excluded).  The stop test is one
// saturated multiply-add, (T' - e') 2^40 with e' the float below 1e-4: two
// distinct floats near 1e-4 differ by at least 2^-37, so it is >= 8 (1 after
// saturation) exactly when T' >= 1e-4 and <= 0 otherwise.  U drops by the
// weight, so it follows T' while the pixel goes on and keeps the stop's T.
// Returns the gaussian's weight alpha T (0 when it did not contribute).
__device__ __forceinline__ float apply_alpha(PixelAcc& p, float al, const float4& g2) {
  const float aT = al * p.T;
  const float tn = p.T - aT;
  const float s = __saturatef(fmaf(tn, 1099511627776.f, -109951152.0f));  // 1: keeps going
  const float wt = aT * s;
  p.r = fmaf(g2.x, wt, p.r);
  p.g = fmaf(g2.y, wt, p.g);
  p.b = fmaf(g2.z, wt, p.b);
  p.U -= wt;
  p.T = tn * s;
  return wt;
}

// One gaussian at one pixel; returns its weight alpha T (0: no contribution).
__device__ __forceinline__ float blend(PixelAcc& p, float ubase, float dy, const float4& g0, const float4& g1,
                                       const float4& g2) {
  float raw;
  return apply_alpha(p, alpha_of(ubase, dy, g0, g1, g2, raw), g2);
}

// ---- half-precision rasterisation (HG_FLAG_FP16, Sec. 3.5 / 4.5)
// The staged record's first two float4 are rewritten as half2 pairs
// {my, my} {l1', l1'} {l2', l2'} {o, o} | {mx, mx} {l0', l0'} {E, E} {0, 0},
// positions relative to the macro-tile centre (so every operand of the
// Mahalanobis sum stays far inside the fp16 range, at the finest spacing the
// macro-tile allows); the colour float4 stays.
__device__ __forceinline__ uint32_t h2_bits(float x) {
  const __half2 h = __float2half2_rn(x);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void half_record(float4* r, float ox, float oy) {
  const float4 g0 = r[0], g1 = r[1], g2 = r[2];
  uint4* q = reinterpret_cast<uint4*>(r);
  q[0] = make_uint4(h2_bits(g0.y - oy), h2_bits(g0.w), h2_bits(g1.x), h2_bits(g1.y));
  q[1] = make_uint4(h2_bits(g0.x - ox), h2_bits(g0.z), h2_bits(record_level(g2)), 0u);
}

// alpha of one gaussian at the two pixels a thread owns, in half2: hpx the
// pixel column, hpy the two pixel rows (relative to the macro-tile centre).  The blend test
// e <= E is the saturated multiply-add of the float32 path at half scale
// (fp16 spacing at e = 6.5 is 2^-8, so (E - e) 2^10 + 1 is <= -3 when e > E).
__device__ __forceinline__ float2 half_alpha2(const float4* r, __half2 hpx, __half2 hpy) {
  const uint4 q0 = reinterpret_cast<const uint4*>(r)[0], q1 = reinterpret_cast<const uint4*>(r)[1];
  const __half2 my = *reinterpret_cast<const __half2*>(&q0.x), l1 = *reinterpret_cast<const __half2*>(&q0.y);
  const __half2 l2 = *reinterpret_cast<const __half2*>(&q0.z), o = *reinterpret_cast<const __half2*>(&q0.w);
  const __half2 mx = *reinterpret_cast<const __half2*>(&q1.x), l0 = *reinterpret_cast<const __half2*>(&q1.y);
  const __half2 E = *reinterpret_cast<const __half2*>(&q1.z);
  const __half2 ub = __hmul2(l0, __hsub2(hpx, mx));
  const __half2 dy = __hsub2(hpy, my);
  const __half2 u = __hfma2(l1, dy, ub);
  const __half2 w = __hmul2(l2, dy);
  const __half2 e = __hfma2(u, u, __hmul2(w, w));
  const __half2 a = __hmin2(__hmul2(o, h2exp2(__hneg2(e))), __float2half2_rn(ALPHA_MAX));
  const __half2 f = __hfma2_sat(__hsub2(E, e), __float2half2_rn(1024.f), __float2half2_rn(1.f));
  return __half22float2(__hmul2(a, f));
}


// Tile-mask geometry of one gaussian (Alg. 1 phase 1, the opacity-threshold
// ellipse of Sec. 4.5).  The blend test passes only where
// e = (l0' dx + l1' dy)^2 + (l2' dy)^2 <= E, E the record's level.
// Masks only need to be conservative, so this uses fast approximate
// arithmetic (rsqrt, fast reciprocal) with margins far above its error: the
// level is enlarged by 2^-10 relative + 2^-12, the y extent and the row spans
// by 0.02 px + 2^-10 of the offset.  Computed once per gaussian: the y half
// extent hy, the leftmost point dyl with its offset x_l (rightmost at -dyl,
// offset x_r).
struct MaskGauss {
  float E, hy, hyw, dyl, x_l, x_r, il0, l1, l2;
  bool live, ok;
};

__device__ __forceinline__ float fast_sqrt0(float v) { return v > 0.f ? v * rsqrtf(v) : 0.f; }

__device__ __forceinline__ MaskGauss mask_gauss(const float4& g0, const float4& g1, const float4& g2) {
  MaskGauss m;
  m.live = g2.w >= 0.f;
  m.E = fmaf(record_level(g2), 1.f + 1.f / 1024.f, 1.f / 4096.f);
  m.l1 = g0.w;
  m.l2 = g1.x;
  m.ok = g0.z > 0.f && g1.x > 0.f;
  if (!m.ok || !m.live) return m;
  const float sE = fast_sqrt0(m.E);
  m.il0 = __fdividef(1.f, g0.z);
  const float il2 = __fdividef(1.f, g1.x);
  m.hy = sE * il2;
  m.hyw = fmaf(m.hy, 1.f + 1.f / 1024.f, 0.02f);
  m.dyl = m.l1 * sE * il2 * rsqrtf(fmaf(m.l1, m.l1, m.l2 * m.l2));
  const float t = m.l2 * m.dyl;
  const float h = fast_sqrt0(fmaf(-t, t, m.E));
  m.x_l = (-m.l1 * m.dyl - h) * m.il0;
  m.x_r = (m.l1 * m.dyl + h) * m.il0;
  return m;
}

// x span (pixel-centre coordinates) of the gaussian's mask ellipse over the
// rows [ya, yb]; false when the rows miss it.  The left edge
// (-l1 dy - h(dy)) / l0 is convex in dy: over the rows' part [a, b] of
// [-hy, hy] its minimum is at dyl when dyl is in [a, b], else at the end
// nearer to dyl (the right edge, concave, likewise with -dyl).
__device__ __forceinline__ bool mask_row_span(const MaskGauss& m, float mx, float my, float ya, float yb, float& xl,
                                              float& xr) {
  const float ra = ya - my, rb = yb - my;
  if (!(fmaxf(ra, -m.hyw) <= fminf(rb, m.hyw))) return false;
  float a = fmaxf(ra, -m.hy), b = fminf(rb, m.hy);
  if (!(a <= b)) a = b = rb < -m.hy ? -m.hy : m.hy;
  float lo, hi;
  if (m.dyl >= a && m.dyl <= b) {
    lo = m.x_l;
  } else {
    const float d = m.dyl < a ? a : b, t = m.l2 * d;
    lo = (-m.l1 * d - fast_sqrt0(fmaf(-t, t, m.E))) * m.il0;
  }
  if (-m.dyl >= a && -m.dyl <= b) {
    hi = m.x_r;
  } else {
    const float d = -m.dyl < a ? a : b, t = m.l2 * d;
    hi = (-m.l1 * d + fast_sqrt0(fmaf(-t, t, m.E))) * m.il0;
  }
  xl = fmaxf(mx + lo - fmaf(fabsf(lo), 1.f / 1024.f, 0.02f), -1e6f);
  xr = fminf(mx + hi + fmaf(fabsf(hi), 1.f / 1024.f, 0.02f), 1e6f);
  return xl <= xr;
}

// Conservative test of a gaussian's 3-sigma rectangle against render tile
// (tx, ty) (same integer rule as the macro binning, at 8x8 granularity).
__device__ __forceinline__ void tile_rect(const float4& g0, const float4& g1, int& x0, int& x1, int& y0, int& y1) {
  const int rad = __float_as_int(g1.z);
  const int px = (int)floorf(g0.x), py = (int)floorf(g0.y);
  x0 = (px - rad) >> TILE_SHIFT;
  x1 = (px + rad) >> TILE_SHIFT;
  y0 = (py - rad) >> TILE_SHIFT;
  y1 = (py + rad) >> TILE_SHIFT;
}

}  // namespace hg
