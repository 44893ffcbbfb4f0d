// Macro-tile rasteriser (Alg. 1 MacroTileRasterize, Alg. 2 RasterizeTile,
// Sec. 4.5).  A persistent grid of CTAs claims processing units (macro-tile,
// batch of <= B_r sorted gaussians) in batch-rank-major order.  Per unit:
//   load    the batch's gaussian ids, then one TMA bulk copy per gaussian
//           gathers its 48-byte record into shared memory (one mbarrier)
//   phase 1 each warp takes mini-batches of 32 gaussians, computes the
//           gaussian's render-tile mask inside the macro-tile and transposes
//           the 32 x M bit matrix with ballots (per-tile gaussian masks)
//   queue   warp 0 ORs the masks per tile and compacts the active tiles;
//           tiles that an earlier batch of the macro-tile already saturated
//           are dropped (their pixels never composite this batch)
//   phase 2 warps claim tiles from the queue; a warp blends the tile's 64
//           pixels (two per lane) front to back over the set mask bits, with
//           a unanimous-vote early out when every pixel has stopped
//   store   partial (r, g, b, +-T) per pixel with streaming stores (T is
//           negated when the pixel stopped inside the batch) and the unit's
//           active-tile mask
#include "blend.cuh"
#include "kernels.cuh"

namespace hg {

namespace {

constexpr int RW = 8;  // warps per CTA
constexpr int RT = RW * 32;

template <int MW, int MH>
struct RasterShape {
  static constexpr int M = MW * MH;
};

__global__ void k_zero_u32(uint32_t* p, uint32_t v, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

template <int MW, int MH>
__global__ void __launch_bounds__(RT) k_raster(RasterArgs a, int cap) {
  constexpr int M = MW * MH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s_rec = reinterpret_cast<float4*>(smem_raw);                       // [cap][3]
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(s_rec + (size_t)cap * 3);   // [cap/32][M]
  __shared__ uint64_t bar;
  __shared__ uint32_t s_unit, s_qn, s_qhead;
  __shared__ uint8_t s_q[64];
  __shared__ unsigned long long s_active;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (read_status(a.fc)) return;
  const uint32_t n_units = a.fc->n_batches;
  uint32_t phase = 0;
  unsigned long long evals = 0;

  while (true) {
    if (tid == 0) {
      s_unit = atomicAdd(&a.fc->raster_claim, 1u);
      s_qhead = 0;
    }
    __syncthreads();
    const uint32_t u = s_unit;
    if (u >= n_units) break;
    const uint32_t r = a.batch_order[u];
    const uint4 bt = a.batches[r];
    const uint32_t seg = bt.x, start = bt.y, count = bt.z, rank = bt.w;
    const int v = find_view(a.views, a.n_views, (int)seg);
    const ViewDesc& V = a.views[v];
    const int mloc = (int)seg - V.seg_base;
    const int mtx0 = (mloc % V.mgx) * MW, mty0 = (mloc / V.mgx) * MH;  // macro origin (tiles)
    const float4* rec_v = a.rec + (size_t)v * a.n * 3;

    // gather the batch records: one bulk copy of 48 bytes per gaussian
    if (tid == 0) mbar_arrive_expect_tx(&bar, count * 48u);
    __syncthreads();
    for (uint32_t j = tid; j < count; j += RT) {
      const uint32_t id = a.vals[start + j];
      tma_load_1d(s_rec + (size_t)j * 3, rec_v + (size_t)id * 3, 48u, &bar);
    }
    if (!mbar_wait_bounded(&bar, phase)) {
      set_status(a.fc, HG_ERR_DEVICE_TIMEOUT);
      atomicOr(&a.fc->timeout_where, 2u);
      mbar_wait_bounded(&bar, phase);
      return;
    }
    phase ^= 1u;

    // phase 1: per-gaussian tile masks, transposed to per-tile masks
    const int K = (int)((count + 31) / 32);
    for (int k = warp; k < K; k += RW) {
      const uint32_t j = (uint32_t)k * 32 + lane;
      unsigned long long gm = 0;
      if (j < count) {
        const float4 g0 = s_rec[j * 3 + 0], g1 = s_rec[j * 3 + 1];
        int x0, x1, y0, y1;
        tile_rect(g0, g1, x0, x1, y0, y1);
        x0 = max(max(x0, mtx0), 0) - mtx0;
        x1 = min(min(x1, mtx0 + MW - 1), V.tiles_x - 1) - mtx0;
        y0 = max(max(y0, mty0), 0) - mty0;
        y1 = min(min(y1, mty0 + MH - 1), V.tiles_y - 1) - mty0;
        if (x0 <= x1 && y0 <= y1) {
          const unsigned long long row = ((1ull << (x1 - x0 + 1)) - 1ull) << x0;
          for (int y = y0; y <= y1; ++y) gm |= row << (y * MW);
        }
      }
#pragma unroll
      for (int t = 0; t < M; ++t) {
        const uint32_t b = __ballot_sync(0xffffffffu, (gm >> t) & 1ull);
        if (lane == (t & 31)) s_mask[k * M + t] = b;
      }
    }
    __syncthreads();

    // tile work queue (warp 0)
    if (warp == 0) {
      unsigned long long act = 0;
      int qn = 0;
#pragma unroll
      for (int h = 0; h < (M + 31) / 32; ++h) {
        const int t = h * 32 + lane;
        bool hit = false;
        if (t < M) {
          uint32_t o = 0;
          for (int k = 0; k < K; ++k) o |= s_mask[k * M + t];
          hit = o != 0;
          if (hit) {
            const int gtx = mtx0 + t % MW, gty = mty0 + t / MW;
            const uint32_t sat = a.tile_sat[V.tile_base + gty * V.tiles_x + gtx];
            if (sat < rank) hit = false;  // an earlier batch stopped every pixel
          }
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, hit);
        if (hit) s_q[qn + __popc(bal & lanemask_lt())] = (uint8_t)t;
        qn += __popc(bal);
        act |= (unsigned long long)bal << (h * 32);
      }
      if (lane == 0) {
        s_qn = (uint32_t)qn;
        s_active = act;
      }
    }
    __syncthreads();
    if (tid == 0) a.active[r] = s_active;
    const uint32_t qn = s_qn;

    // phase 2: warps claim tiles
    while (true) {
      uint32_t qi = 0;
      if (lane == 0) qi = atomicAdd(&s_qhead, 1u);
      qi = __shfl_sync(0xffffffffu, qi, 0);
      if (qi >= qn) break;
      const int t = s_q[qi];
      const int gtx = mtx0 + t % MW, gty = mty0 + t / MW;
      const int px = gtx * TILE + (lane & 7);
      const int py = gty * TILE + (lane >> 3);
      PixelAcc p0, p1;
      pixel_init(p0, px < V.W && py < V.H);
      pixel_init(p1, px < V.W && py + 4 < V.H);
      uint32_t stop0 = count, stop1 = count;
      const float fpx = (float)px, fpy = (float)py, fpy1 = (float)(py + 4);
      uint32_t n_blend = 0;
      for (int k = 0; k < K; ++k) {
        uint32_t m = s_mask[k * M + t];
        while (m) {
          const int bit = __ffs(m) - 1;
          m &= m - 1;
          const uint32_t j = (uint32_t)k * 32 + bit;
          const float4 g0 = s_rec[j * 3 + 0], g1 = s_rec[j * 3 + 1], g2 = s_rec[j * 3 + 2];
          const float dx = fpx - g0.x;
          const float ub = g0.z * dx;
          if (blend_one(p0, ub, fpy - g0.y, g0, g1, g2)) stop0 = j;
          if (blend_one(p1, ub, fpy1 - g0.y, g0, g1, g2)) stop1 = j;
          ++n_blend;
          if (__all_sync(0xffffffffu, p0.done && p1.done)) {
            m = 0;
            k = K;
          }
        }
      }
      if (lane == 0) evals += (unsigned long long)n_blend * 64ull;
      float4* out = a.partial + ((size_t)r * M + t) * TILE_PX;
      st_cs(out + lane, make_float4(p0.r, p0.g, p0.b, p0.stopped ? -p0.T : p0.T));
      st_cs(out + lane + 32, make_float4(p1.r, p1.g, p1.b, p1.stopped ? -p1.T : p1.T));
      if (a.stop_pos) {
        uint16_t* sp = a.stop_pos + ((size_t)r * M + t) * TILE_PX;
        sp[lane] = (uint16_t)stop0;
        sp[lane + 32] = (uint16_t)stop1;
      }
      // every in-image pixel stopped inside this batch: later batches skip the tile
      const bool sat0 = p0.stopped || !(px < V.W && py < V.H);
      const bool sat1 = p1.stopped || !(px < V.W && py + 4 < V.H);
      if (__all_sync(0xffffffffu, sat0 && sat1) && lane == 0)
        atomicMin(&a.tile_sat[V.tile_base + gty * V.tiles_x + gtx], rank);
    }
    __syncthreads();
  }
  if (lane == 0 && evals) atomicAdd(&a.fc->raster_evals, evals);
}

template <int MW, int MH>
cudaError_t launch_raster_shape(const RasterArgs& a, int cap, cudaStream_t st) {
  constexpr int M = MW * MH;
  const size_t sm = (size_t)cap * 48 + (size_t)((cap + 31) / 32) * M * 4;
  cudaError_t e = cudaFuncSetAttribute(k_raster<MW, MH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int occ = 1, dev = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_raster<MW, MH>, RT, sm);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (occ < 1) occ = 1;
  const int grid = a.persistent_ctas > 0 ? a.persistent_ctas : sms * occ;
  k_raster<MW, MH><<<grid, RT, sm, st>>>(a, cap);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_raster(const RasterArgs& a, cudaStream_t st) {
  const int cap = a.batch_cap;
  if (a.macro_w == 8 && a.macro_h == 4) return launch_raster_shape<8, 4>(a, cap, st);
  if (a.macro_w == 4 && a.macro_h == 4) return launch_raster_shape<4, 4>(a, cap, st);
  if (a.macro_w == 8 && a.macro_h == 8) return launch_raster_shape<8, 8>(a, cap, st);
  return cudaErrorInvalidValue;
}

}  // namespace hg
