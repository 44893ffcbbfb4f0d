// Stable block-wide radix ranking (8-bit digits) used by the onesweep passes
// of the segmented sort.
//
// Items are held warp-striped: item slot i of lane l in warp w is element
// w * 32 * IPT + i * 32 + l of the block's range, so ranking slot by slot and
// lane by lane inside a warp, then warp by warp, is the element order and the
// resulting ranks are stable.
#pragma once
#include "common.cuh"

namespace hg {

constexpr uint32_t NO_DIGIT = 256;  // item not ranked (tail of a partial tile)

template <int NT>
struct RankSmem {
  uint32_t hist[NT / 32][256];
  uint32_t digit_start[256];
  uint32_t digit_count[256];
};

// Lanes of the warp holding the same digit (9 bits, NO_DIGIT included) as
// this lane, from one ballot per bit (measured faster than match.any here).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    const bool bit = (d >> b) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

// dig[i] in [0, 256) or NO_DIGIT.  On return pos[i] is the item's position in
// the block sorted stably by digit (undefined for NO_DIGIT), and
// digit_start / digit_count describe the sorted block.
template <int NT, int IPT>
__device__ __forceinline__ void block_rank(const uint32_t (&dig)[IPT], uint32_t (&pos)[IPT], RankSmem<NT>& s) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = lane; j < 256; j += 32) s.hist[warp][j] = 0;
  __syncwarp();
  const uint32_t lt = lanemask_lt();
  uint32_t rk[IPT];
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t d = dig[i];
    const uint32_t peers = digit_peers(d);
    const uint32_t leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (d < 256) base = s.hist[warp][d];
    __syncwarp();
    if (d < 256 && lane == (int)leader) s.hist[warp][d] = base + __popc(peers);
    __syncwarp();
    rk[i] = base + __popc(peers & lt);
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, column total
  for (int d = threadIdx.x; d < 256; d += NT) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      uint32_t c = s.hist[w][d];
      s.hist[w][d] = run;
      run += c;
    }
    s.digit_count[d] = run;
  }
  __syncthreads();
  // exclusive scan of the 256 digit totals by warp 0 (8 per lane)
  if (warp == 0) {
    uint32_t v[8], sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v[k] = s.digit_count[lane * 8 + k];
      sum += v[k];
    }
    uint32_t inc = warp_incl_scan(sum);
    uint32_t run = inc - sum;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      s.digit_start[lane * 8 + k] = run;
      run += v[k];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t d = dig[i];
    pos[i] = d < 256 ? s.digit_start[d] + s.hist[warp][d] + rk[i] : 0xffffffffu;
  }
}

template <int IPT>
__device__ __forceinline__ int striped_index(int i) {
  return (threadIdx.x >> 5) * 32 * IPT + i * 32 + (threadIdx.x & 31);
}

}  // namespace hg
