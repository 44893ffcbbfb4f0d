// Plain per-tile path (the single-tile-size baseline the paper compares
// against, Sec. 2 and 5): 3-sigma rectangle over 8x8 render tiles -> count
// -> exclusive scan -> duplicate with 64-bit keys (global tile << 32 | depth
// key) -> global onesweep radix sort over the key bits that vary -> tile
// ranges -> one 64-thread CTA per tile blending its pixels sequentially.
// It shares the projection and the blend arithmetic with the HiGS path.
#include "blend.cuh"
#include "kernels.cuh"

namespace hg {

namespace {

constexpr int SCAN_T = 1024, SCAN_I = 4, SCAN_B = SCAN_T * SCAN_I;

__device__ __forceinline__ int tile_span(const uint4& r, const ViewDesc& V, int& x0, int& x1, int& y0, int& y1) {
  const int rad = (int)r.z;
  if (rad <= 0) return 0;
  const int px = (int)floorf(__uint_as_float(r.x)), py = (int)floorf(__uint_as_float(r.y));
  x0 = max((px - rad) >> TILE_SHIFT, 0);
  x1 = min((px + rad) >> TILE_SHIFT, V.tiles_x - 1);
  y0 = max((py - rad) >> TILE_SHIFT, 0);
  y1 = min((py + rad) >> TILE_SHIFT, V.tiles_y - 1);
  if (x0 > x1 || y0 > y1) return 0;
  return (x1 - x0 + 1) * (y1 - y0 + 1);
}

// Culled (view, gaussian) entries have no record: test the visibility bit.
__device__ __forceinline__ bool visible(const PlainArgs& a, int v, long long i) {
  return (a.vis[(long long)v * a.vis_words + (i >> 5)] >> (i & 31)) & 1u;
}

__global__ void k_plain_count(PlainArgs a) {
  const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = a.n * a.n_views;
  if (o >= total) return;
  const int v = (int)(o / a.n);
  int x0, x1, y0, y1;
  a.counts[o] = visible(a, v, o - (long long)v * a.n) ? (uint32_t)tile_span(a.bin[o], a.views[v], x0, x1, y0, y1)
                                                       : 0u;
}

// exclusive scan of counts[total] into offsets[total + 1]
__global__ void __launch_bounds__(SCAN_T) k_scan_blocks(const uint32_t* in, uint32_t* out, uint32_t* sums,
                                                        long long total) {
  __shared__ uint32_t tmp[33];
  const long long base = (long long)blockIdx.x * SCAN_B + (long long)threadIdx.x * SCAN_I;
  uint32_t v[SCAN_I], s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_I; ++k) {
    v[k] = base + k < total ? in[base + k] : 0u;
    s += v[k];
  }
  uint32_t tot;
  uint32_t ex = block_excl_scan(s, tmp, &tot);
#pragma unroll
  for (int k = 0; k < SCAN_I; ++k) {
    if (base + k < total) out[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_sums(uint32_t* sums, int nblocks, uint32_t* out, long long total,
                                                      PlainArgs a) {
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nblocks; b0 += SCAN_T) {
    const int b = b0 + threadIdx.x;
    const uint32_t v = b < nblocks ? sums[b] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(v, tmp, &tot);
    if (b < nblocks) sums[b] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[total] = carry;
    const uint32_t np = carry;
    a.fc->n_pairs = np;
    const uint32_t nt = (np + OS_TILE - 1) / OS_TILE;
    a.fc->n_big_tiles = nt;
    a.fc->n_batches = 0;
    if (np > a.cap_pairs || nt > a.cap_tiles) set_status(a.fc, HG_ERR_CAPACITY);
  }
}

__global__ void k_scan_add(uint32_t* out, const uint32_t* sums, long long total) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < total) out[i] += sums[i / SCAN_B];
}

__global__ void k_plain_tiles(PlainArgs a, uint4* tiles) {
  if (read_status(a.fc)) return;
  const uint32_t nt = a.fc->n_big_tiles, np = a.fc->n_pairs;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nt; k += gridDim.x * blockDim.x)
    tiles[k] = make_uint4(0u, k * OS_TILE, min((uint32_t)OS_TILE, np - k * OS_TILE), k);
}

__global__ void k_plain_dup(PlainArgs a) {
  const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = a.n * a.n_views;
  if (o >= total || read_status(a.fc)) return;
  const int v = (int)(o / a.n);
  const ViewDesc& V = a.views[v];
  if (!visible(a, v, o - (long long)v * a.n)) return;
  const uint4 r = a.bin[o];
  int x0, x1, y0, y1;
  if (!tile_span(r, V, x0, x1, y0, y1)) return;
  uint32_t pos = a.offsets[o];
  for (int y = y0; y <= y1; ++y)
    for (int x = x0; x <= x1; ++x) {
      const unsigned long long t = (unsigned long long)(V.tile_base + y * V.tiles_x + x);
      a.keys[pos] = (t << 32) | r.w;
      a.vals[pos] = (uint32_t)o;
      ++pos;
    }
}

__global__ void k_plain_ranges(PlainArgs a, const unsigned long long* keys) {
  if (read_status(a.fc)) return;
  const uint32_t np = a.fc->n_pairs;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)(keys[i] >> 32);
    if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) a.ranges[t].x = i;
    if (i + 1 == np || (uint32_t)(keys[i + 1] >> 32) != t) a.ranges[t].y = i + 1;
  }
}

__device__ __forceinline__ int find_view_tile2(const ViewDesc* views, int n_views, int tile) {
  int v = 0;
  while (v + 1 < n_views && views[v + 1].tile_base <= tile) ++v;
  return v;
}

__global__ void __launch_bounds__(TILE_PX) k_plain_raster(PlainArgs a, const uint32_t* vals) {
  __shared__ float4 s_rec[TILE_PX * 3];
  if (read_status(a.fc)) return;
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int v = find_view_tile2(a.views, a.n_views, tile);
  const ViewDesc& V = a.views[v];
  const int lt = tile - V.tile_base, tx = lt % V.tiles_x, ty = lt / V.tiles_x;
  const int px = tx * TILE + (tid & 7), py = ty * TILE + (tid >> 3);
  const bool inside = px < V.W && py < V.H;
  PixelAcc p;
  pixel_init(p, inside);
  const uint2 rg = a.ranges[tile];
  if (tid == 0 && rg.y > rg.x) atomicMax(&a.fc->max_seg, rg.y - rg.x);  // densest tile (frame stats)
  const float fpx = (float)px, fpy = (float)py;
  for (uint32_t base = rg.x; base < rg.y; base += TILE_PX) {
    if (__syncthreads_count(pixel_live(p)) == 0) break;
    const uint32_t j = base + tid;
    if (j < rg.y) {
      const float4* rp = a.rec + (size_t)vals[j] * REC_F4;
      s_rec[tid * 3 + 0] = rp[0];
      s_rec[tid * 3 + 1] = rp[1];
      s_rec[tid * 3 + 2] = rp[2];
    }
    __syncthreads();
    const int nb = (int)min((uint32_t)TILE_PX, rg.y - base);
    for (int k = 0; k < nb; ++k) {
      const float4 g0 = s_rec[k * 3 + 0], g1 = s_rec[k * 3 + 1], g2 = s_rec[k * 3 + 2];
      blend(p, g0.z * (fpx - g0.x), fpy - g0.y, g0, g1, g2);
    }
  }
  if (inside) {
    const long long o = V.pix_base + (long long)py * V.W + px;
    const float tf = pixel_final_T(p);
    a.out_rgb[o * 3 + 0] = fmaf(tf, a.bg[0], p.r);
    a.out_rgb[o * 3 + 1] = fmaf(tf, a.bg[1], p.g);
    a.out_rgb[o * 3 + 2] = fmaf(tf, a.bg[2], p.b);
    if (a.out_T) a.out_T[o] = tf;
  }
}

}  // namespace

cudaError_t launch_plain(PlainArgs& a, cudaStream_t st, unsigned long long** sorted_keys, uint32_t** sorted_vals) {
  const long long total = a.n * a.n_views;
  cudaError_t e;
  if (total == 0) {
    // nothing to bin: every tile range is empty and the raster writes background
    *sorted_keys = a.keys;
    *sorted_vals = a.vals;
    if ((e = cudaMemsetAsync(a.ranges, 0, sizeof(uint2) * a.total_tiles, st)) != cudaSuccess) return e;
    k_plain_raster<<<a.total_tiles, TILE_PX, 0, st>>>(a, a.vals);
    note_launch();
    return cudaGetLastError();
  }
  const unsigned g = (unsigned)((total + 255) / 256);
  k_plain_count<<<g, 256, 0, st>>>(a);
  note_launch();
  const int nblk = (int)((total + SCAN_B - 1) / SCAN_B);
  k_scan_blocks<<<nblk, SCAN_T, 0, st>>>(a.counts, a.offsets, a.scan_tmp, total);
  note_launch();
  k_scan_sums<<<1, SCAN_T, 0, st>>>(a.scan_tmp, nblk, a.offsets, total, a);
  note_launch();
  k_scan_add<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a.offsets, a.scan_tmp, total);
  note_launch();
  uint4* tiles = reinterpret_cast<uint4*>(a.scan_tmp + ((nblk + 3) & ~3));
  k_plain_tiles<<<256, 256, 0, st>>>(a, tiles);
  note_launch();
  k_plain_dup<<<g, 256, 0, st>>>(a);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // passes: the depth bytes plus the bytes of the global tile index
  int tile_bits = 1;
  while ((1ll << tile_bits) < (long long)a.total_tiles) ++tile_bits;
  const int npass = 4 + (tile_bits + 7) / 8;
  OsTileView tv{tiles, &a.fc->n_big_tiles, a.digit_hist, nullptr, nullptr, nullptr};
  bool alt = false;
  e = launch_onesweep<unsigned long long, 8>(tv, a.keys, a.vals, a.keys_alt, a.vals_alt, a.digit_hist, 8 * 256,
                                             true, a.lookback, (size_t)a.cap_tiles * 256, a.fc->os_claim, 0, npass,
                                             a.wait_polls, a.fc, st, &alt);
  if (e != cudaSuccess) return e;
  unsigned long long* sk = alt ? a.keys_alt : a.keys;
  uint32_t* sv = alt ? a.vals_alt : a.vals;
  *sorted_keys = sk;
  *sorted_vals = sv;
  if ((e = cudaMemsetAsync(a.ranges, 0, sizeof(uint2) * a.total_tiles, st)) != cudaSuccess) return e;
  k_plain_ranges<<<1024, 256, 0, st>>>(a, sk);
  note_launch();
  k_plain_raster<<<a.total_tiles, TILE_PX, 0, st>>>(a, sv);
  note_launch();
  return cudaGetLastError();
}

}  // namespace hg
