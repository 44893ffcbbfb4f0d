// Pieces shared by the forward and backward rasterisers: the warp bit
// transpose, the per-unit tile-mask builder (Alg. 1 phase 1) and an acquire
// load for the batch chain.
#pragma once
#include "blend.cuh"

namespace hg {

// 32 x 32 bit-matrix transpose across a warp (5-stage shuffle butterfly):
// lane i holds row i on entry and column i on return.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int w = 16 >> s;
    const uint32_t m = masks[s];
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, w);
    x = (lane & w) ? ((x & ~m) | ((y & ~m) >> w)) : ((x & m) | ((y & m) << w));
  }
  return x;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Phase 1 of a processing unit: every warp takes mini-batches of 32 staged
// gaussians, computes each gaussian's render-tile masks inside the macro-tile
// for the top (rows 0-3) and bottom (rows 4-7) half of every tile and
// transposes the 32 x M bit matrices, so that s_top[k * M + t] and
// s_bot[k * M + t] hold, for tile t, the bits of the mini-batch-k gaussians
// that can pass the blend test in its top / bottom half.  Per tile row the
// 3-sigma rectangle is refined by the x span of the blend-test ellipse over
// the row's 8 pixel rows; a half keeps those columns when its 4 pixel rows
// meet the ellipse's y extent.  With s_cnt, lane t also adds the number of
// (gaussian, half) entries of tile t to s_cnt[t] (the tile's work, for the
// queue order).  With REV the mask words are stored bit-reversed (gaussian
// j of a mini-batch in bit 31 - j), so a front-to-back walk takes the
// highest set bit first (one leading-bit search per gaussian).
template <int MW, int MH, bool REV = false>
__device__ __forceinline__ void build_tile_masks(const float4* s_rec, uint32_t* s_top, uint32_t* s_bot,
                                                 uint32_t count, const ViewDesc& V, int mtx0, int mty0,
                                                 int n_warps, uint32_t* s_cnt = nullptr) {
  constexpr int M = MW * MH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int K = (int)((count + 31) / 32);
  for (int k = warp; k < K; k += n_warps) {
    const uint32_t j = (uint32_t)k * 32 + lane;
    unsigned long long gt = 0, gb = 0;
    if (j < count) {
      const float4 g0 = s_rec[j * 3 + 0], g1 = s_rec[j * 3 + 1], g2 = s_rec[j * 3 + 2];
      int x0, x1, y0, y1;
      tile_rect(g0, g1, x0, x1, y0, y1);
      x0 = max(max(x0, mtx0), 0) - mtx0;
      x1 = min(min(x1, mtx0 + MW - 1), V.tiles_x - 1) - mtx0;
      y0 = max(max(y0, mty0), 0) - mty0;
      y1 = min(min(y1, mty0 + MH - 1), V.tiles_y - 1) - mty0;
      const MaskGauss mg = mask_gauss(g0, g1, g2);
      if (x0 <= x1 && y0 <= y1 && mg.live) {
        const unsigned long long full = ((1ull << (x1 - x0 + 1)) - 1ull) << x0;
        for (int y = y0; y <= y1; ++y) {
          if (!mg.ok) {
            gt |= full << (y * MW);
            gb |= full << (y * MW);
            continue;
          }
          const float ya = (float)((mty0 + y) * TILE);
          float xl, xr;
          if (!mask_row_span(mg, g0.x, g0.y, ya, ya + (float)(TILE - 1), xl, xr)) continue;
          const int c0 = max(x0, ((int)ceilf(xl) >> TILE_SHIFT) - mtx0);
          const int c1 = min(x1, ((int)floorf(xr) >> TILE_SHIFT) - mtx0);
          if (c0 > c1) continue;
          const unsigned long long bits = (((1ull << (c1 - c0 + 1)) - 1ull) << c0) << (y * MW);
          const float ry = ya - g0.y;  // offset of the tile's first pixel row
          if (ry <= mg.hyw && ry + (float)(TILE / 2 - 1) >= -mg.hyw) gt |= bits;
          if (ry + (float)(TILE / 2) <= mg.hyw && ry + (float)(TILE - 1) >= -mg.hyw) gb |= bits;
        }
      }
    }
    // TransposeMasks: lane t receives the 32-gaussian masks of tile t
    if constexpr (M <= 16) {
      // both halves in one word (top masks in bits 0-15, bottom in 16-31):
      // lane t < 16 receives tile t's top masks, lane 16 + t its bottom ones
      const uint32_t tb = transpose32((uint32_t)gt | ((uint32_t)gb << 16), lane);
      if ((lane & 15) < M) {
        (lane < 16 ? s_top : s_bot)[k * M + (lane & 15)] = REV ? __brev(tb) : tb;
        if (s_cnt) atomicAdd(&s_cnt[lane & 15], (uint32_t)__popc(tb));
      }
      continue;
    }
    const uint32_t tlo = transpose32((uint32_t)gt, lane), blo = transpose32((uint32_t)gb, lane);
    if (lane < M) {
      s_top[k * M + lane] = REV ? __brev(tlo) : tlo;
      s_bot[k * M + lane] = REV ? __brev(blo) : blo;
      if (s_cnt) atomicAdd(&s_cnt[lane], (uint32_t)(__popc(tlo) + __popc(blo)));
    }
    if (M > 32) {
      const uint32_t thi = transpose32((uint32_t)(gt >> 32), lane), bhi = transpose32((uint32_t)(gb >> 32), lane);
      s_top[k * M + 32 + lane] = REV ? __brev(thi) : thi;
      s_bot[k * M + 32 + lane] = REV ? __brev(bhi) : bhi;
      if (s_cnt) atomicAdd(&s_cnt[32 + lane], (uint32_t)(__popc(thi) + __popc(bhi)));
    }
  }
}

}  // namespace hg
