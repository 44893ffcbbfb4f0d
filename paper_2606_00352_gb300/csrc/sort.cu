// Segmented depth sort (Sec. 3.3, 4.4).  Every (view, macro-tile) segment of
// (32-bit depth key, gaussian id) pairs is sorted ascending by (key, id):
//   * segments of <= 1K, <= 4K, <= 8K and <= 16K pairs: one CTA of 128, 256,
//     512 or 1,024 threads sorts the segment in shared memory with one
//     counting scatter into 2^12, 2^13, 2^14 or 2^15 buckets (at least two
//     per pair) by the top bits of (key - min key), then puts each run of
//     pairs that share a bucket in (key, id) order, the warps ranking the
//     pairs of whole runs by shuffles; this also breaks key ties by id (the
//     fill pass writes a segment in a data-dependent order).  A segment with a run of more
//     than 32 pairs is sorted again by a bitonic network over (key, id), so
//     the cost stays bounded whatever the keys.  The smaller CTAs fit more
//     segments per SM;
//   * larger segments (> 16K): a segment-local onesweep (one kernel per 8-bit
//     digit pass, decoupled look-back across the segment's tiles, tiles
//     claimed in order through an atomic counter so every awaited
//     predecessor is running), preceded by one histogram kernel for all
//     digits.  Its passes are stable, so it sorts by the id's four digits
//     first and then by the key's: (key, id) order with no fix-up.
#include <mutex>
#include <string>
#include <utility>

#include "internal.h"
#include "kernels.cuh"
#include "radix.cuh"

namespace hg {

namespace {

// ------------------------------------------------------------ tier sorts
__device__ __forceinline__ bool pair_less(uint32_t ka, uint32_t va, uint32_t kb, uint32_t vb) {
  return ka < kb || (ka == kb && va < vb);
}

// Block-wide min and max of one value per thread (red: [2][NT / 32]).
template <int NT>
__device__ __forceinline__ void block_min_max(uint32_t& mn, uint32_t& mx, uint32_t (*red)[NT / 32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    red[0][warp] = mn;
    red[1][warp] = mx;
  }
  __syncthreads();
  mn = 0xffffffffu;
  mx = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) {
    mn = min(mn, red[0][w]);
    mx = max(mx, red[1][w]);
  }
  __syncthreads();
}

// Significant bits of the span kmax - kmin (0 when every key is equal).
__device__ __forceinline__ int radix_bits(uint32_t kmin, uint32_t kmax) {
  const uint32_t span = kmax - kmin;
  return span ? 32 - __clz(span) : 0;
}

// Next entry of a tier's segment list for this CTA (dynamic claiming: the
// segments differ in size, so CTAs take the next one when they are done).
__device__ __forceinline__ uint32_t claim_segment(FrameCounters* fc, int tier, uint32_t* s_claim) {
  if (threadIdx.x == 0) *s_claim = atomicAdd(&fc->tier_claim[tier], 1u);
  __syncthreads();
  return *s_claim;
}

// ------------------------------------------------------------ bucket tiers
// Segments of up to NT * IPT pairs in one CTA, all in shared memory: the
// pairs are held in registers (slot i of thread t: element t + i * NT),
// counted into 2^BBITS buckets by the top BBITS bits of (key - min key)
// (16-bit counters, two per word, shared-memory atomics), the bucket
// counts scanned into offsets, and the pairs scattered to their buckets
// (atomic cursors: any order inside a bucket).  With at least two buckets
// per pair, a bucket holds a few pairs, and the warps put every run of
// pairs that share a bucket in (key, id) order, so the order is exactly
// (key, id) whatever the scatter's order.  A segment with a run of more
// than 32 pairs (keys packed into few buckets, or many equal keys) is
// sorted again by a bitonic network over (key, id) instead:
// O(n log^2 n) with no register arrays, linear in the number of stages.
// Shared-memory index of counter word w: one pad word after every 16, so
// the 16 words a thread scans start 17 words after its neighbour's (no two
// lanes on one bank).
__device__ __forceinline__ uint32_t cnt_word(uint32_t w) { return w + (w >> 4); }

template <int NT, int IPT, int BBITS>
struct BucketSortSmem {
  uint32_t keys[NT * IPT];
  uint32_t vals[NT * IPT];
  uint32_t cnt[(1 << BBITS) / 2 + (1 << BBITS) / 32];  // bucket b: bits 16 (b & 1) .. of word cnt_word(b / 2)
  uint32_t red[2][NT / 32];
  uint32_t scan[33];
};

// Bitonic sort of the n pairs of a shared-memory region by (key, id), the
// region padded to the next power of two (at most `cap`) with the largest
// pair.
template <int NT>
__device__ __forceinline__ void bitonic_region(uint32_t* keys, uint32_t* vals, int n, int cap) {
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  if (n2 > cap) n2 = cap;
  for (int j = n + (int)threadIdx.x; j < n2; j += NT) keys[j] = vals[j] = 0xffffffffu;
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < n2 / 2; i += NT) {
        const int lo = ((i & ~(jj - 1)) << 1) | (i & (jj - 1)), hi = lo + jj;
        const uint32_t ka = keys[lo], va = vals[lo], kb = keys[hi], vb = vals[hi];
        const bool up = (lo & k) == 0;
        if (pair_less(kb, vb, ka, va) == up) {
          keys[lo] = kb;
          vals[lo] = vb;
          keys[hi] = ka;
          vals[hi] = va;
        }
      }
      __syncthreads();
    }
  }
}

template <int NT, int IPT, int BBITS>
__global__ void __launch_bounds__(NT, 65536 / (NT * 64)) k_bucket_sort(SortArgs a, int tier) {
  constexpr int B = 1 << BBITS, W = B / 2, CW = W / NT;  // words of counters per thread
  static_assert(W % NT == 0 && CW % 16 == 0, "counter words (and their pad words) must divide evenly over the threads");
  static_assert(NT * IPT <= 65535, "16-bit bucket counters");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BucketSortSmem<NT, IPT, BBITS>& s = *reinterpret_cast<BucketSortSmem<NT, IPT, BBITS>*>(smem_raw);
  __shared__ uint32_t s_claim;
  __shared__ int s_long_run;
  if (read_status(a.fc)) return;
  const uint32_t count = a.fc->tier_count[tier];
  const uint32_t* list = a.tier_list + (size_t)tier * a.n_seg;
  const int tid = threadIdx.x;
  for (uint32_t idx = claim_segment(a.fc, tier, &s_claim); idx < count;
       idx = claim_segment(a.fc, tier, &s_claim)) {
    const uint32_t seg = list[idx];
    const uint32_t start = a.seg_off[seg];
    const int n = (int)(a.seg_off[seg + 1] - start);
    uint32_t k[IPT], v[IPT];
    uint32_t kmin = 0xffffffffu, kmax = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const int j = tid + i * NT;
      k[i] = v[i] = 0xffffffffu;
      if (j < n) {
        k[i] = __ldcg(a.keys + start + j);
        v[i] = __ldcg(a.vals + start + j);
      }
    }
#pragma unroll
    for (int i = 0; i < IPT; ++i)
      if (tid + i * NT < n) {
        kmin = min(kmin, k[i]);
        kmax = max(kmax, k[i]);
      }
#pragma unroll
    for (int q = 0; q < CW + CW / 16; ++q) s.cnt[tid + q * NT] = 0;
    block_min_max<NT>(kmin, kmax, s.red);  // its barriers also order the clearing
    const int bits = radix_bits(kmin, kmax);
    const int lo = bits > BBITS ? bits - BBITS : 0;
    // bucket counts
#pragma unroll
    for (int i = 0; i < IPT; ++i)
      if (tid + i * NT < n) {
        const uint32_t d = (k[i] - kmin) >> lo;
        atomicAdd(&s.cnt[cnt_word(d >> 1)], (d & 1u) ? 0x10000u : 1u);
      }
    __syncthreads();
    // bucket offsets: thread t scans the words [t * CW, (t + 1) * CW)
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < CW; ++q) {
      const uint32_t w = s.cnt[cnt_word(tid * CW + q)];
      sum += (w & 0xffffu) + (w >> 16);
    }
    uint32_t run = block_excl_scan(sum, s.scan, (uint32_t*)nullptr);
#pragma unroll
    for (int q = 0; q < CW; ++q) {
      const uint32_t w = s.cnt[cnt_word(tid * CW + q)], c0 = w & 0xffffu;
      s.cnt[cnt_word(tid * CW + q)] = run | ((run + c0) << 16);
      run += c0 + (w >> 16);
    }
    __syncthreads();
    // scatter to the buckets
#pragma unroll
    for (int i = 0; i < IPT; ++i)
      if (tid + i * NT < n) {
        const uint32_t d = (k[i] - kmin) >> lo;
        const uint32_t old = atomicAdd(&s.cnt[cnt_word(d >> 1)], (d & 1u) ? 0x10000u : 1u);
        const uint32_t pos = (d & 1u) ? old >> 16 : old & 0xffffu;
        s.keys[pos] = k[i];
        s.vals[pos] = v[i];
      }
    if (tid == 0) s_long_run = 0;
    __syncthreads();
    // runs of pairs that share a bucket, in (key, id) order.  The counters
    // now hold each bucket's end, so a pair's run is [end of the bucket
    // before, end of its bucket).  Warp w takes the pairs from the first
    // run start at or after w * n / NW to the first at or after
    // (w + 1) * n / NW, 32 positions at a time, cut back to the last run
    // that ends inside them: every lane ranks its pair against the pairs of
    // its own run (shuffles, as many steps as the chunk's longest run) and
    // writes it to its place in the chunk, which no other warp touches.
    {
      const int lane = tid & 31, warp = tid >> 5;
      constexpr int NW = NT / 32;
      auto bucket_end = [&](uint32_t b) -> int {
        const uint32_t w = s.cnt[cnt_word(b >> 1)];
        return (int)((b & 1u) ? w >> 16 : w & 0xffffu);
      };
      auto run_start_from = [&](int pos) -> int {  // first run start at or after pos
        if (pos <= 0 || pos >= n) return pos <= 0 ? 0 : n;
        const uint32_t b = (s.keys[pos] - kmin) >> lo;
        const int rs = b ? bucket_end(b - 1) : 0;
        return rs == pos ? pos : bucket_end(b);
      };
      const int c_end = run_start_from((int)(((long long)(warp + 1) * n) / NW));
      for (int c = run_start_from((int)(((long long)warp * n) / NW)); c < c_end;) {
        const int p = c + lane;
        uint32_t k = 0, v = 0;
        int rs = 0, re = 0x7fffffff;
        if (p < c_end) {
          k = s.keys[p];
          v = s.vals[p];
          const uint32_t b = (k - kmin) >> lo;
          rs = b ? bucket_end(b - 1) : 0;
          re = bucket_end(b);
        }
        const bool fits = re <= c + 32;  // runs ending inside the chunk (a prefix of the lanes)
        const int len = __popc(__ballot_sync(0xffffffffu, fits));
        if (len == 0) {  // a run of more than 32 pairs starts at c
          if (lane == 0) s_long_run = 1;
          break;
        }
        const int rl = fits ? re - rs : 0, off = rs - c;
        const int steps = __reduce_max_sync(0xffffffffu, (unsigned)rl);
        int rank = 0;
        for (int d = 0; d < steps; ++d) {
          const int src = (off + d) & 31;
          const uint32_t kd = __shfl_sync(0xffffffffu, k, src), vd = __shfl_sync(0xffffffffu, v, src);
          if (d < rl) rank += pair_less(kd, vd, k, v);
        }
        __syncwarp();
        if (fits && rl > 1) {
          s.keys[rs + rank] = k;
          s.vals[rs + rank] = v;
        }
        __syncwarp();
        c += len;
      }
    }
    __syncthreads();
    if (s_long_run) {
      if (tid == 0) atomicAdd(&a.fc->sort_resorts, 1u);
      bitonic_region<NT>(s.keys, s.vals, n, NT * IPT);
    }
    for (int j = tid; j < n; j += NT) {
      a.keys[start + j] = s.keys[j];
      a.vals[start + j] = s.vals[j];
    }
    __syncthreads();
  }
}

}  // namespace

// ------------------------------------------------------------ onesweep
// Look-back words: bits 30-31 flag, bits 0-29 count.
constexpr uint32_t LB_AGG = 1u << 30;
constexpr uint32_t LB_INC = 2u << 30;
constexpr uint32_t LB_MASK = (1u << 30) - 1;

template <typename K>
struct OneSweepSmem {
  K keys[OS_TILE];
  uint32_t vals[OS_TILE];
  RankSmem<OS_THREADS> rank;
  uint32_t gbase[256];
  uint32_t tile_claim;
};



// Digit histograms of every pass for each onesweep segment, and the clearing
// of the tiles' look-back words.  Pass p sorts by digit p % sizeof(K) of its
// key word: with `lo` set (32-bit keys, NPASS = 8) passes 0-3 take the
// digits of lo[] (the values, sorted first) and passes 4-7 those of keys[];
// otherwise pass p takes digit p of keys[].  Every tile's look-back words of
// every pass ([NPASS][lb_stride] words, 256 per tile) are zeroed here, so
// the passes need no memset; seg_hist must be zero on entry.
template <typename K, int NPASS>
__global__ void __launch_bounds__(OS_THREADS) k_os_hist(OsTileView tv, const K* keys, const uint32_t* lo,
                                                        uint32_t* seg_hist, uint32_t* lookback, size_t lb_stride,
                                                        FrameCounters* fc) {
  constexpr int DIG = (int)sizeof(K);
  __shared__ uint32_t h[NPASS][256];
  if (read_status(fc)) return;
  const uint32_t nt = *tv.tile_count;
  for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
    for (int j = threadIdx.x; j < NPASS * 256; j += OS_THREADS) {
      (&h[0][0])[j] = 0;
      lookback[(size_t)(j >> 8) * lb_stride + (size_t)t * 256 + (j & 255)] = 0;
    }
    __syncthreads();
    const uint4 td = tv.tiles[t];
    for (uint32_t j = threadIdx.x; j < td.z; j += OS_THREADS) {
      const K k = keys[td.y + j];
      if (lo) {
        const uint32_t l = lo[td.y + j];
#pragma unroll
        for (int p = 0; p < 4; ++p) atomicAdd(&h[p][(l >> (8 * p)) & 0xffu], 1u);
#pragma unroll
        for (int p = 4; p < NPASS; ++p) atomicAdd(&h[p][(uint32_t)(k >> (8 * (p - 4))) & 0xffu], 1u);
      } else {
#pragma unroll
        for (int p = 0; p < NPASS; ++p) atomicAdd(&h[p][(uint32_t)(k >> (8 * (p % DIG))) & 0xffu], 1u);
      }
    }
    __syncthreads();
    uint32_t* dst = seg_hist + (size_t)td.x * NPASS * 256;
    for (int j = threadIdx.x; j < NPASS * 256; j += OS_THREADS) {
      uint32_t c = (&h[0][0])[j];
      if (c) atomicAdd(dst + j, c);
    }
    __syncthreads();
  }
}

// One stable pass: every tile of the segments is ranked by digit
// pass % sizeof(K) of src_k in shared memory and scattered to the segment's
// output ranges (digit offsets from the segment histogram of this pass plus
// the exclusive prefix of the earlier tiles, found by decoupled look-back in
// this pass's look-back words).
template <typename K, int NPASS>
__global__ void __launch_bounds__(OS_THREADS) k_os_pass(OsTileView tv, const K* src_k, const uint32_t* src_v,
                                                        K* dst_k, uint32_t* dst_v, uint32_t* lookback,
                                                        uint32_t* claim, int pass, uint32_t wait_polls,
                                                        FrameCounters* fc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  OneSweepSmem<K>& s = *reinterpret_cast<OneSweepSmem<K>*>(smem_raw);
  if (read_status(fc)) return;
  const uint32_t nt = *tv.tile_count;
  const int shift = 8 * (pass % (int)sizeof(K));
  const int tid = threadIdx.x;
  while (true) {
    if (tid == 0) s.tile_claim = atomicAdd(claim, 1u);
    __syncthreads();
    const uint32_t t = s.tile_claim;
    __syncthreads();
    if (t >= nt) return;
    const uint4 td = tv.tiles[t];
    const uint32_t bseg = td.x, start = td.y, cnt = td.z, ti = td.w;
    K k[OS_ITEMS];
    uint32_t v[OS_ITEMS], d[OS_ITEMS], p[OS_ITEMS];
#pragma unroll
    for (int i = 0; i < OS_ITEMS; ++i) {
      int e = striped_index<OS_ITEMS>(i);
      if ((uint32_t)e < cnt) {
        k[i] = src_k[start + e];
        v[i] = src_v[start + e];
        d[i] = (uint32_t)(k[i] >> shift) & 0xffu;
      } else {
        k[i] = 0;
        v[i] = 0;
        d[i] = NO_DIGIT;
      }
    }
    block_rank<OS_THREADS, OS_ITEMS>(d, p, s.rank);
    // publish this tile's digit counts, then look back over the segment's
    // earlier tiles for the exclusive prefix of every digit
    uint32_t* lb = lookback + (size_t)t * 256;
    if (tid < 256) {
      const uint32_t c = s.rank.digit_count[tid];
      volatile uint32_t* me = lb + tid;
      if (ti == 0) {
        *me = LB_INC | c;
      } else {
        *me = LB_AGG | c;
        uint32_t excl = 0;
        uint32_t j = t - 1;
        bool ok = true;
        while (true) {
          volatile uint32_t* w = lookback + (size_t)j * 256 + tid;
          uint32_t val = *w;
          uint32_t it = 0;
          while ((val & ~LB_MASK) == 0) {
            if (++it > wait_polls) {
              ok = false;
              break;
            }
            val = *w;
          }
          if (!ok) break;
          excl += val & LB_MASK;
          if ((val & ~LB_MASK) == LB_INC) break;
          --j;
        }
        if (!ok) {
          set_status(fc, HG_ERR_DEVICE_TIMEOUT);
          atomicOr(&fc->timeout_where, 1u);
        }
        *me = LB_INC | ((excl + c) & LB_MASK);
        s.gbase[tid] = excl;
      }
      if (ti == 0) s.gbase[tid] = 0;
    }
    // segment-level digit offsets for this pass
    __syncthreads();
    if (tid < 32) {
      const uint32_t* hh = tv.seg_hist + ((size_t)bseg * NPASS + pass) * 256;
      uint32_t vv[8], sum = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        vv[q] = hh[tid * 8 + q];
        sum += vv[q];
      }
      uint32_t inc = warp_incl_scan(sum), run = inc - sum;
      const uint32_t seg_start = tv.seg_off ? tv.seg_off[tv.big_segs[bseg]] : 0u;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        int dd = tid * 8 + q;
        // destination of local sorted index j with digit dd: gbase[dd] + j
        s.gbase[dd] = seg_start + run + s.gbase[dd] - s.rank.digit_start[dd];
        run += vv[q];
      }
    }
#pragma unroll
    for (int i = 0; i < OS_ITEMS; ++i) {
      if (d[i] != NO_DIGIT) {
        s.keys[p[i]] = k[i];
        s.vals[p[i]] = v[i];
      }
    }
    __syncthreads();
    for (uint32_t j = tid; j < cnt; j += OS_THREADS) {
      K kk = s.keys[j];
      uint32_t dd = (uint32_t)(kk >> shift) & 0xffu;
      uint32_t dst = s.gbase[dd] + j;
      dst_k[dst] = kk;
      dst_v[dst] = s.vals[j];
    }
    __syncthreads();
  }
}

static int g_sms = 0;
static int num_sms() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 148;
  }
  return g_sms;
}

template <int NT, int IPT, int BBITS>
static cudaError_t launch_bucket_tier(const SortArgs& a, int tier, int blocks_per_sm, cudaStream_t st) {
  size_t sm = sizeof(BucketSortSmem<NT, IPT, BBITS>);
  cudaError_t e =
      cudaFuncSetAttribute(k_bucket_sort<NT, IPT, BBITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_bucket_sort<NT, IPT, BBITS><<<num_sms() * blocks_per_sm, NT, sm, st>>>(a, tier);
  note_launch();
  return cudaGetLastError();
}

template <typename K, int NPASS>
static cudaError_t os_passes(const OsTileView& tv, const K* keys, const uint32_t* lo, uint32_t* seg_hist,
                             size_t seg_hist_words, bool zero_hist, uint32_t* lookback, size_t lb_stride,
                             FrameCounters* fc, cudaStream_t st, int* occ_out, int max_ctas = 0) {
  cudaError_t e;
  if (zero_hist && (e = cudaMemsetAsync(seg_hist, 0, seg_hist_words * 4, st)) != cudaSuccess) return e;
  const int hgrid = max_ctas > 0 ? min(max_ctas, num_sms() * 2) : num_sms() * 2;
  k_os_hist<K, NPASS><<<hgrid, OS_THREADS, 0, st>>>(tv, keys, lo, seg_hist, lookback, lb_stride, fc);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t sm = sizeof(OneSweepSmem<K>);
  e = cudaFuncSetAttribute(k_os_pass<K, NPASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_os_pass<K, NPASS>, OS_THREADS, sm);
  *occ_out = occ < 1 ? 1 : occ;
  return cudaSuccess;
}

template <typename K, int NPASS>
cudaError_t launch_onesweep(const OsTileView& tv, K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt,
                            uint32_t* seg_hist, size_t seg_hist_words, bool zero_hist, uint32_t* lookback,
                            size_t lb_stride, uint32_t* claims, int first_pass, int npass, uint32_t wait_polls,
                            FrameCounters* fc, cudaStream_t st, bool* result_in_alt) {
  int occ = 1;
  cudaError_t e = os_passes<K, NPASS>(tv, keys, nullptr, seg_hist, seg_hist_words, zero_hist, lookback, lb_stride,
                                      fc, st, &occ);
  if (e != cudaSuccess) return e;
  const size_t sm = sizeof(OneSweepSmem<K>);
  K* sk = keys;
  uint32_t* sv = vals;
  K* dk = keys_alt;
  uint32_t* dv = vals_alt;
  for (int p = first_pass; p < first_pass + npass; ++p) {
    k_os_pass<K, NPASS><<<num_sms() * occ, OS_THREADS, sm, st>>>(tv, sk, sv, dk, dv, lookback + (size_t)p * lb_stride,
                                                                claims + p, p, wait_polls, fc);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::swap(sk, dk);
    std::swap(sv, dv);
  }
  *result_in_alt = (npass & 1) != 0;
  return cudaSuccess;
}

template cudaError_t launch_onesweep<unsigned long long, 8>(const OsTileView&, unsigned long long*, uint32_t*,
                                                            unsigned long long*, uint32_t*, uint32_t*, size_t, bool,
                                                            uint32_t*, size_t, uint32_t*, int, int, uint32_t,
                                                            FrameCounters*, cudaStream_t, bool*);
template cudaError_t launch_onesweep<uint32_t, 4>(const OsTileView&, uint32_t*, uint32_t*, uint32_t*, uint32_t*,
                                                  uint32_t*, size_t, bool, uint32_t*, size_t, uint32_t*, int, int,
                                                  uint32_t, FrameCounters*, cudaStream_t, bool*);

// Segments sorted ascending by (key, value): four stable passes over the
// value's digits, then four over the key's (8 passes, so the result ends in
// keys / vals).  seg_hist holds [segments][8][256] words, lookback
// [8][lb_stride] words.  max_ctas > 0 caps the persistent grids: any grid is
// correct (tiles are claimed in order, so every awaited predecessor is held
// by a running CTA), and a small one keeps the passes of a frame without
// big segments from taking SM slots the shared-memory tiers run on.
static cudaError_t launch_onesweep_by_val_key(const OsTileView& tv, uint32_t* keys, uint32_t* vals,
                                              uint32_t* keys_alt, uint32_t* vals_alt, uint32_t* seg_hist,
                                              size_t seg_hist_words, bool zero_hist, uint32_t* lookback,
                                              size_t lb_stride, uint32_t* claims, uint32_t wait_polls,
                                              FrameCounters* fc, cudaStream_t st, int max_ctas = 0) {
  int occ = 1;
  cudaError_t e = os_passes<uint32_t, 8>(tv, keys, vals, seg_hist, seg_hist_words, zero_hist, lookback, lb_stride,
                                         fc, st, &occ, max_ctas);
  if (e != cudaSuccess) return e;
  const size_t sm = sizeof(OneSweepSmem<uint32_t>);
  const int grid = max_ctas > 0 ? min(max_ctas, num_sms() * occ) : num_sms() * occ;
  uint32_t *ck = keys, *cv = vals, *ak = keys_alt, *av = vals_alt;
  for (int p = 0; p < 8; ++p) {
    // value passes move (value, key) pairs, key passes (key, value) pairs
    uint32_t* sk = p < 4 ? cv : ck;
    uint32_t* sv = p < 4 ? ck : cv;
    uint32_t* dk = p < 4 ? av : ak;
    uint32_t* dv = p < 4 ? ak : av;
    k_os_pass<uint32_t, 8><<<grid, OS_THREADS, sm, st>>>(tv, sk, sv, dk, dv,
                                                                    lookback + (size_t)p * lb_stride, claims + p, p,
                                                                    wait_polls, fc);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::swap(ck, ak);
    std::swap(cv, av);
  }
  return cudaSuccess;
}

static cudaError_t launch_sort_kernels(const SortArgs& a, cudaStream_t st, cudaStream_t s1, cudaStream_t s2,
                                       cudaStream_t s3) {
  cudaError_t e;
  // the largest tiers first, each on its own stream when s1..s3 differ from
  // st: their tails overlap
  if ((e = launch_bucket_tier<1024, 16, 15>(a, 3, 1, s3)) != cudaSuccess) return e;
  if ((e = launch_bucket_tier<512, 16, 14>(a, 2, 2, s2)) != cudaSuccess) return e;
  if ((e = launch_bucket_tier<256, 16, 13>(a, 1, 4, s1)) != cudaSuccess) return e;
  if ((e = launch_bucket_tier<128, 8, 12>(a, 0, 8, st)) != cudaSuccess) return e;
  OsTileView tv{a.big_tiles, &a.fc->n_big_tiles, a.seg_hist, a.seg_off, a.big_segs, a.big_tile_first};
  // the partition zeroed the big segments' histograms
  return launch_onesweep_by_val_key(tv, a.keys, a.vals, a.keys_alt, a.vals_alt, a.seg_hist, 0, false, a.lookback,
                                    (size_t)a.cap_tiles * 256, a.fc->os_claim, a.wait_polls, a.fc, st, a.os_ctas);
}

cudaError_t launch_sort(const SortArgs& a, cudaStream_t st, const SortStreams* ss) {
  if (!ss) return launch_sort_kernels(a, st, st, st, st);
  cudaError_t e = cudaEventRecord(ss->fork, st);
  if (e != cudaSuccess) return e;
  int forked = 0;
  for (; forked < 3; ++forked)
    if ((e = cudaStreamWaitEvent(ss->aux[forked], ss->fork, 0)) != cudaSuccess) break;
  if (e == cudaSuccess) e = launch_sort_kernels(a, st, ss->aux[2], ss->aux[1], ss->aux[0]);
  // join every forked stream back, also after an error (an open fork would
  // leave a stream capture unjoined)
  for (int i = 0; i < forked; ++i) {
    cudaError_t j = cudaEventRecord(ss->join[i], ss->aux[i]);
    if (j == cudaSuccess) j = cudaStreamWaitEvent(st, ss->join[i], 0);
    if (e == cudaSuccess) e = j;
  }
  return e;
}

// ------------------------------------------------------------------------
// Segmented sort with no allocation, for callers that cannot allocate
// device memory at the call site (for example code running inside another
// allocator's callback, or a host that must not touch the device heap while
// other work is being captured or served).  All scratch lives in one
// file-scope device array of fixed size that every GPU which loads this
// library keeps until the process exits.
namespace {

constexpr uint32_t NA_MAX_PAIRS = 1u << 19;                         // 524,288 pairs
constexpr uint32_t NA_MAX_SEGS = 512;
constexpr uint32_t NA_MAX_TILES = NA_MAX_PAIRS / OS_TILE + NA_MAX_SEGS;
constexpr size_t NA_FC_WORDS = 64;
constexpr size_t NA_TILE_WORDS = (size_t)NA_MAX_TILES * 4;
constexpr size_t NA_SEGS_WORDS = (size_t)NA_MAX_SEGS * 2;
constexpr size_t NA_HIST_WORDS = (size_t)NA_MAX_SEGS * 8 * 256;     // [segment][pass][digit]
constexpr size_t NA_LB_STRIDE = (size_t)NA_MAX_TILES * 256;           // look-back words of one pass
constexpr size_t NA_LB_WORDS = 8 * NA_LB_STRIDE;
constexpr size_t NA_PP_WORDS = (size_t)NA_MAX_PAIRS * 2;
constexpr size_t NA_WORDS = NA_FC_WORDS + NA_TILE_WORDS + NA_SEGS_WORDS + NA_HIST_WORDS + NA_LB_WORDS + NA_PP_WORDS;

static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

static_assert(sizeof(FrameCounters) <= NA_FC_WORDS * 4, "counter block too small");

// One CTA: onesweep tile descriptors for every segment of >= 2 pairs (the
// segment index doubles as the histogram index).
__global__ void __launch_bounds__(1024) k_na_tiles(const uint32_t* seg_off, int n_seg, uint4* tiles,
                                                   uint32_t* segs, uint32_t* tile_first, FrameCounters* fc) {
  __shared__ uint32_t tmp[33];
  const int tid = threadIdx.x;
  const int s = tid;  // n_seg <= NA_MAX_SEGS <= 1024
  uint32_t n = 0, nt = 0;
  if (s < n_seg) {
    n = seg_off[s + 1] - seg_off[s];
    nt = n >= 2 ? (n + OS_TILE - 1) / OS_TILE : 0;
  }
  uint32_t total;
  const uint32_t first = block_excl_scan(nt, tmp, &total);
  if (s < n_seg) {
    segs[s] = (uint32_t)s;
    tile_first[s] = first;
    for (uint32_t k = 0; k < nt; ++k)
      tiles[first + k] = make_uint4((uint32_t)s, seg_off[s] + k * OS_TILE, min((uint32_t)OS_TILE, n - k * OS_TILE), k);
  }
  if (tid == 0) fc->n_big_tiles = total;
}

}  // namespace

// Device address of the scratch array, looked up once per device.
static void* noalloc_scratch(int dev, hg_status* st) {
  static std::mutex mu;
  static void* addr[64] = {};
  *st = HG_OK;
  if (dev < 0 || dev >= 64) {
    *st = HG_ERR_INVALID_ARG;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      *st = hg_cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "hg_segmented_sort_noalloc set-up");
      return nullptr;
    }
    addr[dev] = p;
  }
  return addr[dev];
}

// [a, a + n) and [b, b + n) share a byte
static bool overlaps(const void* a, const void* b, size_t bytes) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bytes && y < x + bytes;
}

extern "C" hg_status hg_segmented_sort_noalloc(const uint32_t* d_seg_off, int n_seg, int64_t n_pairs,
                                               const uint32_t* d_keys_in, const uint32_t* d_vals_in,
                                               uint32_t* d_keys_out, uint32_t* d_vals_out, void* stream) {
  if (n_seg < 1 || n_pairs < 0 || !d_seg_off || (n_pairs > 0 && (!d_keys_in || !d_vals_in || !d_keys_out ||
                                                                  !d_vals_out))) {
    hg_set_error("hg_segmented_sort_noalloc: bad arguments");
    return HG_ERR_INVALID_ARG;
  }
  if ((uint64_t)n_pairs > NA_MAX_PAIRS || (uint32_t)n_seg > NA_MAX_SEGS) {
    hg_set_error("hg_segmented_sort_noalloc: at most 524288 pairs in at most 512 segments (got " +
                 std::to_string(n_pairs) + " pairs, " + std::to_string(n_seg) + " segments)");
    return HG_ERR_INVALID_ARG;
  }
  const size_t bytes = 4 * (size_t)n_pairs;
  if (n_pairs > 0) {
    // an output may be its own input (in place); no other overlap
    const bool in_place = d_keys_in == d_keys_out && d_vals_in == d_vals_out;
    const bool bad = overlaps(d_keys_out, d_vals_out, bytes) ||
                     (!in_place && (overlaps(d_keys_out, d_keys_in, bytes) || overlaps(d_keys_out, d_vals_in, bytes) ||
                                    overlaps(d_vals_out, d_keys_in, bytes) || overlaps(d_vals_out, d_vals_in, bytes))) ||
                     (in_place && overlaps(d_keys_in, d_vals_in, bytes));
    if (bad) {
      hg_set_error("hg_segmented_sort_noalloc: overlapping buffers (only keys_out == keys_in together with "
                   "vals_out == vals_in is allowed)");
      return HG_ERR_INVALID_ARG;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  {
    // the call synchronises the stream, which a capture cannot do
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return hg_cuda_status(e, "hg_segmented_sort_noalloc");
    if (cs != cudaStreamCaptureStatusNone) {
      hg_set_error("hg_segmented_sort_noalloc: the stream is capturing; the call synchronises it");
      return HG_ERR_INVALID_ARG;
    }
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hg_cuda_status(e, "hg_segmented_sort_noalloc");
  hg_status st;
  uint32_t* base = (uint32_t*)noalloc_scratch(dev, &st);
  if (!base) return st;
  // the segment table must be an ordered partition of [0, n_pairs)
  uint32_t off[NA_MAX_SEGS + 1];
  if ((e = cudaMemcpyAsync(off, d_seg_off, sizeof(uint32_t) * (n_seg + 1), cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return hg_cuda_status(e, "hg_segmented_sort_noalloc seg_off");
  if (off[0] != 0 || off[n_seg] != (uint32_t)n_pairs) {
    hg_set_error("hg_segmented_sort_noalloc: seg_off must start at 0 and end at n_pairs");
    return HG_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n_seg; ++i)
    if (off[i + 1] < off[i]) {
      hg_set_error("hg_segmented_sort_noalloc: seg_off is not non-decreasing");
      return HG_ERR_INVALID_ARG;
    }
  if (n_pairs == 0) return HG_OK;
  FrameCounters* fc = (FrameCounters*)base;
  uint4* tiles = (uint4*)(base + NA_FC_WORDS);
  uint32_t* segs = base + NA_FC_WORDS + NA_TILE_WORDS;
  uint32_t* tile_first = segs + NA_MAX_SEGS;
  uint32_t* hist = base + NA_FC_WORDS + NA_TILE_WORDS + NA_SEGS_WORDS;
  uint32_t* lb = hist + NA_HIST_WORDS;
  uint32_t* pp_k = lb + NA_LB_WORDS;
  uint32_t* pp_v = pp_k + NA_MAX_PAIRS;
  // the array keeps the previous call's contents: clear what starts at zero
  // (the counters and the digit histograms; the histogram kernel clears the
  // look-back words of the tiles it finds)
  if ((e = cudaMemsetAsync(fc, 0, NA_FC_WORDS * 4, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(hist, 0, (size_t)n_seg * 8 * 256 * 4, s)) != cudaSuccess)
    return hg_cuda_status(e, "hg_segmented_sort_noalloc clear");
  if (d_keys_out != d_keys_in &&
      ((e = cudaMemcpyAsync(d_keys_out, d_keys_in, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
       (e = cudaMemcpyAsync(d_vals_out, d_vals_in, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess))
    return hg_cuda_status(e, "hg_segmented_sort_noalloc copy");
  k_na_tiles<<<1, 1024, 0, s>>>(d_seg_off, n_seg, tiles, segs, tile_first, fc);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return hg_cuda_status(e, "hg_segmented_sort_noalloc tiles");
  OsTileView tv{tiles, &fc->n_big_tiles, hist, d_seg_off, segs, tile_first};
  // by value, then by key: (key, value) order for any input, no fix-up
  e = launch_onesweep_by_val_key(tv, d_keys_out, d_vals_out, pp_k, pp_v, hist, 0, false, lb, NA_LB_STRIDE,
                                 fc->os_claim, SPIN_LIMIT, fc, s);
  if (e != cudaSuccess) return hg_cuda_status(e, "hg_segmented_sort_noalloc passes");
  int status = 0;
  if ((e = cudaMemcpyAsync(&status, &fc->status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return hg_cuda_status(e, "hg_segmented_sort_noalloc status");
  if (status != HG_OK) hg_set_error(std::string("hg_segmented_sort_noalloc: device status ") +
                                    hg_status_str((hg_status)status));
  return (hg_status)status;
}

}  // namespace hg
