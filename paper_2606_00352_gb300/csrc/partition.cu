// Gaussian partitioning over macro-tiles (Sec. 3.2, 4.3) and batch split
// (Sec. 3.1):
//   count   one CTA per (partitioning batch of B_p = 8192 gaussians, view):
//           shared-memory histogram with one counter per macro-tile, flushed
//           as uint16 into H[N_B][S]
//   colscan exclusive prefix over partitioning batches per macro-tile column
//           (32 x 32 threads per 32 columns) and the column totals
//   segscan one CTA: segment offsets, batch offsets, sort-tier lists, onesweep
//           tile descriptors, the batch-rank histogram of the raster schedule
//           and the capacity checks
//   fill    replays the binning test and writes (depth key, gaussian id) at
//           seg_off + column prefix + shared-memory cursor
//   batches batch table {segment, start, count, rank} and the raster order
//           (all rank-0 batches first, then rank 1, ...)
// Binning test: the cells of each (view, gaussian) come from its binning
// record (binning.cuh: the 3-sigma rectangle, optionally refined by the
// opacity-aware ellipse), made by the projection.
#include "binning.cuh"
#include "kernels.cuh"

namespace hg {

namespace {

constexpr int PART_THREADS = 512;
constexpr int UNR = 2;  // entries per thread per round in count / fill

__global__ void __launch_bounds__(PART_THREADS) k_count(PartitionArgs a) {
  pdl_wait();
  extern __shared__ uint32_t hist[];
  if (read_status(a.fc)) return;
  const int v = blockIdx.y, b = blockIdx.x, tid = threadIdx.x;
  const ViewDesc& V = a.views[v];
  const int nm = V.mgx * V.mgy;
  for (int m = tid; m < nm; m += PART_THREADS) hist[m] = 0;
  __syncthreads();
  const long long i_end = min(a.n, (long long)(b + 1) * BP);
  const uint32_t* vis = a.vis + (size_t)v * a.vis_words;
  // UNR entries per thread per round: all their loads are issued before any
  // is used (the loop is bound by memory latency, not bandwidth)
  for (long long i0 = (long long)b * BP + tid; i0 < i_end; i0 += UNR * PART_THREADS) {
    uint4 rec[UNR];
    bool on[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const long long i = i0 + (long long)u * PART_THREADS;
      on[u] = i < i_end && ((vis[i >> 5] >> (i & 31)) & 1u);
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u)
      if (on[u]) rec[u] = a.bin[(size_t)v * a.n + i0 + (long long)u * PART_THREADS];
#pragma unroll
    for (int u = 0; u < UNR; ++u)
      if (on[u]) for_each_cell(rec[u], V.mgx, [&](int m) { atomicAdd(&hist[m], 1u); });
  }
  __syncthreads();
  uint16_t* row = a.hist + (size_t)b * a.n_seg + V.seg_base;
  for (int m = tid; m < nm; m += PART_THREADS) row[m] = (uint16_t)hist[m];
}

// 32 columns x 32 batch chunks per CTA.
__global__ void __launch_bounds__(1024) k_colscan(PartitionArgs a) {
  pdl_wait();
  __shared__ uint32_t part[32][33];
  if (read_status(a.fc)) return;
  const int sx = threadIdx.x, cy = threadIdx.y;
  const int s = blockIdx.x * 32 + sx;
  const int nb = a.n_pb, chunk = (nb + 31) / 32;
  const int b0 = min(nb, cy * chunk), b1 = min(nb, b0 + chunk);
  uint32_t sum = 0;
  if (s < a.n_seg)
    for (int b = b0; b < b1; ++b) sum += a.hist[(size_t)b * a.n_seg + s];
  part[cy][sx] = sum;
  __syncthreads();
  uint32_t run = 0;
  for (int c = 0; c < cy; ++c) run += part[c][sx];
  if (s < a.n_seg) {
    for (int b = b0; b < b1; ++b) {
      a.colpre[(size_t)b * a.n_seg + s] = run;
      run += a.hist[(size_t)b * a.n_seg + s];
    }
    if (cy == 31) a.seg_tot[s] = run;
  }
}

__device__ __forceinline__ int seg_tier(uint32_t n) {
  if (n <= 1) return TIER_NONE;
  if (n <= (uint32_t)TIER0_MAX) return 0;
  if (n <= (uint32_t)TIER1_MAX) return 1;
  if (n <= (uint32_t)TIER2_MAX) return 2;
  if (n <= (uint32_t)TIER3_MAX) return 3;
  return TIER_OS;
}

__global__ void __launch_bounds__(1024) k_segscan(PartitionArgs a) {
  pdl_wait();
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t rank_hist[MAX_RANKS];
  __shared__ uint32_t rank_last;
  __shared__ uint32_t red_max[32];
  if (read_status(a.fc)) return;
  const int tid = threadIdx.x, NT = 1024;
  const int S = a.n_seg, per = (S + NT - 1) / NT;
  const int s0 = min(S, tid * per), s1 = min(S, s0 + per);
  const uint32_t cap = (uint32_t)a.batch_cap;
  for (int j = tid; j < MAX_RANKS; j += NT) rank_hist[j] = 0;
  if (tid == 0) rank_last = 0;
  __syncthreads();
  uint32_t c_pairs = 0, c_batches = 0, c_tier[N_TIERS] = {}, c_tiles = 0, mx = 0;
  // segments of 1 to 4 batches (nearly all) are counted in registers and
  // summed per warp: shared-memory atomics on the same few counters from
  // every thread serialise
  constexpr int FEW = 4;
  uint32_t few[FEW] = {};
  for (int s = s0; s < s1; ++s) {
    const uint32_t n = a.seg_tot[s];
    const uint32_t nb = (n + cap - 1) / cap;
    c_pairs += n;
    c_batches += nb;
    const int t = seg_tier(n);
    c_tier[t]++;
    if (t == TIER_OS) c_tiles += (n + OS_TILE - 1) / OS_TILE;
    mx = max(mx, n);
#pragma unroll
    for (int k = 0; k < FEW; ++k) few[k] += nb == (uint32_t)(k + 1);
    if (nb > (uint32_t)FEW) {
      atomicAdd(&rank_hist[min(nb, (uint32_t)MAX_RANKS - 1)], 1u);
      if (nb > (uint32_t)MAX_RANKS - 1) atomicAdd(&rank_last, nb - (MAX_RANKS - 1));
    }
  }
#pragma unroll
  for (int k = 0; k < FEW; ++k) {
    const uint32_t w = warp_sum(few[k]);
    if ((tid & 31) == 0 && w) atomicAdd(&rank_hist[k + 1], w);
  }
  uint32_t t_pairs, t_batches, t_tier[N_TIERS], t_tiles;
  const uint32_t o_pairs = block_excl_scan(c_pairs, tmp, &t_pairs);
  const uint32_t o_batches = block_excl_scan(c_batches, tmp, &t_batches);
  uint32_t o_tier[N_TIERS];
  for (int t = 0; t < N_TIERS; ++t) o_tier[t] = block_excl_scan(c_tier[t], tmp, &t_tier[t]);
  const uint32_t o_tiles = block_excl_scan(c_tiles, tmp, &t_tiles);
  // max segment
  uint32_t m = mx;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) red_max[tid >> 5] = m;
  __syncthreads();
  if (tid < 32) {
    m = red_max[tid];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  const bool over = t_pairs > a.cap_pairs || t_batches > a.cap_batches || t_tiles > a.cap_tiles ||
                    t_tier[TIER_OS] > a.cap_big_segs;
  if (tid == 0) {
    a.fc->n_pairs = t_pairs;
    a.fc->n_batches = t_batches;
    a.fc->n_big_tiles = t_tiles;
    a.fc->n_big_segs = t_tier[TIER_OS];
    a.fc->max_seg = m;
    for (int t = 0; t < N_TIERS; ++t) a.fc->tier_count[t] = t_tier[t];
    if (over) set_status(a.fc, HG_ERR_CAPACITY);
  }
  if (over) return;
  // the onesweep's digit histograms of the big segments start at zero
  for (uint32_t w = tid; w < t_tier[TIER_OS] * 8u * 256u; w += NT) a.seg_hist[w] = 0;
  // raster schedule: batches of rank j = segments with more than j batches
  uint32_t hv[4], hs = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int x = tid * 4 + k;
    hv[k] = x < MAX_RANKS ? rank_hist[x] : 0u;
    hs += hv[k];
  }
  uint32_t h_total;
  uint32_t h_excl = block_excl_scan(hs, tmp, &h_total);
  uint32_t cnt[4], cs = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int x = tid * 4 + k;
    h_excl += hv[k];  // inclusive prefix up to x
    cnt[k] = (x == MAX_RANKS - 1) ? rank_last : h_total - h_excl;
    cs += cnt[k];
  }
  uint32_t c_excl = block_excl_scan(cs, tmp, (uint32_t*)nullptr);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int x = tid * 4 + k;
    if (x < MAX_RANKS) a.rank_count[x] = c_excl;
    c_excl += cnt[k];
  }
  // per-segment outputs
  uint32_t p = o_pairs, bo = o_batches, tl = o_tiles, ot[N_TIERS];
  for (int t = 0; t < N_TIERS; ++t) ot[t] = o_tier[t];
  for (int s = s0; s < s1; ++s) {
    const uint32_t n = a.seg_tot[s];
    a.seg_off[s] = p;
    a.first_batch[s] = bo;
    const int t = seg_tier(n);
    if (t < TIER_OS) {
      a.tier_list[(size_t)t * S + ot[t]] = s;
    } else if (t == TIER_OS) {
      const uint32_t bi = ot[TIER_OS];
      a.big_segs[bi] = s;
      a.big_tile_first[bi] = tl;
      const uint32_t nt = (n + OS_TILE - 1) / OS_TILE;
      for (uint32_t k = 0; k < nt; ++k)
        a.big_tiles[tl + k] = make_uint4(bi, p + k * OS_TILE, min((uint32_t)OS_TILE, n - k * OS_TILE), k);
      tl += nt;
    }
    ot[t]++;
    p += n;
    bo += (n + cap - 1) / cap;
  }
  if (tid == NT - 1) {
    a.seg_off[S] = t_pairs;
    a.first_batch[S] = t_batches;
  }
}

__global__ void __launch_bounds__(PART_THREADS) k_fill(PartitionArgs a) {
  pdl_wait();
  extern __shared__ uint32_t cursor[];
  if (read_status(a.fc)) return;
  const int v = blockIdx.y, b = blockIdx.x, tid = threadIdx.x;
  const ViewDesc& V = a.views[v];
  const int nm = V.mgx * V.mgy;
  const uint32_t* pre = a.colpre + (size_t)b * a.n_seg + V.seg_base;
  for (int m = tid; m < nm; m += PART_THREADS) cursor[m] = a.seg_off[V.seg_base + m] + pre[m];
  __syncthreads();
  const long long i_end = min(a.n, (long long)(b + 1) * BP);
  const uint32_t* vis = a.vis + (size_t)v * a.vis_words;
  for (long long i0 = (long long)b * BP + tid; i0 < i_end; i0 += UNR * PART_THREADS) {
    uint4 rec[UNR];
    uint32_t key[UNR];
    bool on[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const long long i = i0 + (long long)u * PART_THREADS;
      on[u] = i < i_end && ((vis[i >> 5] >> (i & 31)) & 1u);
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      if (!on[u]) continue;
      const size_t o = (size_t)v * a.n + i0 + (long long)u * PART_THREADS;
      rec[u] = a.bin[o];
      key[u] = a.dkeys[o];
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      if (!on[u]) continue;
      const uint32_t id = (uint32_t)(i0 + (long long)u * PART_THREADS);
      for_each_cell(rec[u], V.mgx, [&](int m) {
        const uint32_t pos = atomicAdd(&cursor[m], 1u);
        a.keys[pos] = key[u];
        a.vals[pos] = id;
      });
    }
  }
}

__global__ void k_batches(PartitionArgs a) {
  pdl_wait();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n_seg || read_status(a.fc)) return;
  const uint32_t cap = (uint32_t)a.batch_cap;
  const uint32_t st = a.seg_off[s], n = a.seg_off[s + 1] - st;
  const uint32_t nb = (n + cap - 1) / cap, fb = a.first_batch[s];
  const uint32_t active = __activemask();
  const int lane = threadIdx.x & 31;
  for (uint32_t j = 0;; ++j) {
    // every lane still in the loop takes a slot of rank j: one atomic per
    // warp and rank (the ranks' cursors are shared by all segments)
    const uint32_t m = __ballot_sync(active, j < nb);
    if (!m) break;
    if (j >= nb) continue;
    const uint32_t r = fb + j;
    a.batches[r] = make_uint4((uint32_t)s, st + j * cap, min(cap, n - j * cap), j);
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&a.rank_count[min(j, (uint32_t)MAX_RANKS - 1)], (uint32_t)__popc(m));
    base = __shfl_sync(m, base, leader);
    a.batch_order[base + __popc(m & lanemask_lt())] = r;
  }
}

}  // namespace

cudaError_t launch_partition(const PartitionArgs& a, cudaStream_t st) {
  const size_t sm = (size_t)a.max_nm * 4;
  cudaError_t e;
  if (sm > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(k_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(k_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
      return e;
  }
  if (a.n_pb == 0 || a.n_seg == 0) return cudaSuccess;
  dim3 g(a.n_pb, a.n_views);
  // each kernel of the chain launches while the previous one drains
  // (programmatic dependent launch) and waits for it before its first read
  if ((e = launch_pdl(k_count, g, dim3(PART_THREADS), sm, st, a)) != cudaSuccess) return e;
  if ((e = launch_pdl(k_colscan, dim3((a.n_seg + 31) / 32), dim3(32, 32), 0, st, a)) != cudaSuccess) return e;
  if ((e = launch_pdl(k_segscan, dim3(1), dim3(1024), 0, st, a)) != cudaSuccess) return e;
  if ((e = launch_pdl(k_fill, g, dim3(PART_THREADS), sm, st, a)) != cudaSuccess) return e;
  return launch_pdl(k_batches, dim3((a.n_seg + 255) / 256), dim3(256), 0, st, a);
}

}  // namespace hg
