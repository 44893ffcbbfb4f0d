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
// gaussians, computes each gaussian's render-tile mask inside the macro-tile
// (3-sigma rectangle refined by the ellipse of the blend test per tile row) and
// transposes the 32 x M bit matrix so that s_mask[k * M + t] holds, for tile
// t, the bits of the mini-batch-k gaussians that overlap it.
template <int MW, int MH>
__device__ __forceinline__ void build_tile_masks(const float4* s_rec, uint32_t* s_mask, uint32_t count,
                                                 const ViewDesc& V, int mtx0, int mty0, int n_warps) {
  constexpr int M = MW * MH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int K = (int)((count + 31) / 32);
  for (int k = warp; k < K; k += n_warps) {
    const uint32_t j = (uint32_t)k * 32 + lane;
    unsigned long long gm = 0;
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
        for (int y = y0; y <= y1; ++y) {
          int c0 = x0, c1 = x1;
          if (mg.ok) {
            float xl, xr;
            const float ya = (float)((mty0 + y) * TILE);
            if (!mask_row_span(mg, g0.x, g0.y, ya, ya + (float)(TILE - 1), xl, xr)) continue;
            c0 = max(c0, floordiv((int)ceilf(xl), TILE) - mtx0);
            c1 = min(c1, floordiv((int)floorf(xr), TILE) - mtx0);
          }
          if (c0 <= c1) gm |= (((1ull << (c1 - c0 + 1)) - 1ull) << c0) << (y * MW);
        }
      }
    }
    // TransposeMasks: lane t receives the 32-gaussian mask of tile t
    const uint32_t lo = transpose32((uint32_t)gm, lane);
    if (lane < M) s_mask[k * M + lane] = lo;
    if (M > 32) {
      const uint32_t hi = transpose32((uint32_t)(gm >> 32), lane);
      s_mask[k * M + 32 + lane] = hi;
    }
  }
}

}  // namespace hg
