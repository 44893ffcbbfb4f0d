// Macro-tile rasteriser (Alg. 1 MacroTileRasterize, Alg. 2 RasterizeTile,
// Sec. 4.5).  A persistent grid of CTAs claims processing units (macro-tile,
// batch of <= B_r sorted gaussians) in batch-rank-major order.  Per unit:
//   load    the batch's gaussian ids, then one TMA bulk copy per gaussian
//           gathers its 48-byte record into shared memory (one mbarrier)
//   phase 1 each warp takes mini-batches of 32 gaussians, computes the
//           gaussian's render-tile masks inside the macro-tile, one for the
//           top and one for the bottom half of each tile, and transposes the
//           32 x M bit matrices with a shuffle butterfly (per-tile masks)
//   queue   warp 0 ORs the masks per tile and compacts the active tiles
//   chain   (exact termination) the unit of rank k waits, with a bounded
//           spin, until rank k-1 of the same macro-tile has finished; it then
//           blends from the exact transmittance entering the batch, read from
//           the per-tile state, so pixels and tiles that already stopped cost
//           nothing and no merge-time replay is needed.  Units are claimed
//           rank-major, so the awaited unit was claimed earlier and is running
//           or done.  If the wait gives up, the unit renders from T = 1 (an
//           independent partial) and the merge composites it by Eq. 1 with
//           replay.
//   phase 2 warps claim tiles from the queue, longest first; a warp blends
//           the tile's 64 pixels (two per lane) front to back over the set
//           bits of the tile's mini-batch masks (warp-uniform words, so the
//           gaussians are taken straight from the masks), with a unanimous
//           vote per mini-batch and tile half: a half (4 pixel rows) whose
//           pixels have all stopped takes no more gaussians, and the tile
//           ends when both have
//   store   chained: the new per-tile state, or, for the last batch of the
//           macro-tile, the final pixels straight into the image (the
//           macro-tile's other tiles from their state or the background; the
//           merge then skips it); unchained: the partial (r, g, b, +-T) with
//           streaming stores (T negated when the pixel stopped inside it)
#include "blend.cuh"
#include "kernels.cuh"
#include "raster_common.cuh"

namespace hg {

namespace {

constexpr int RW = 8;  // warps per CTA
constexpr int RT = RW * 32;

// Final pixels of a tile (C + T bg, T) into the outputs.
__device__ __forceinline__ void write_pixels(const RasterArgs& a, const ViewDesc& V, int px, int py, bool in0,
                                             bool in1, const PixelAcc& p0, const PixelAcc& p1) {
  if (in0) {
    const long long o = V.pix_base + (long long)py * V.W + px;
    const float tf = pixel_final_T(p0);
    a.out_rgb[o * 3 + 0] = fmaf(tf, a.bg[0], p0.r);
    a.out_rgb[o * 3 + 1] = fmaf(tf, a.bg[1], p0.g);
    a.out_rgb[o * 3 + 2] = fmaf(tf, a.bg[2], p0.b);
    if (a.out_T) a.out_T[o] = tf;
  }
  if (in1) {
    const long long o = V.pix_base + (long long)(py + 4) * V.W + px;
    const float tf = pixel_final_T(p1);
    a.out_rgb[o * 3 + 0] = fmaf(tf, a.bg[0], p1.r);
    a.out_rgb[o * 3 + 1] = fmaf(tf, a.bg[1], p1.g);
    a.out_rgb[o * 3 + 2] = fmaf(tf, a.bg[2], p1.b);
    if (a.out_T) a.out_T[o] = tf;
  }
}

// STATS (HG_FLAG_PROFILE frames): also counts the intrinsic per-pixel work,
// the support evaluations (q <= 9) of live pixels up to and including each
// pixel's stop, and the contributing ones.
template <int MW, int MH, bool SAVE, bool HALF, bool STATS>
__global__ void __launch_bounds__(RT) k_raster(RasterArgs a, int cap) {
  constexpr int M = MW * MH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s_rec = reinterpret_cast<float4*>(smem_raw);                       // [cap][3]
  uint32_t* s_top = reinterpret_cast<uint32_t*>(s_rec + (size_t)cap * 3);    // [cap/32][M] top halves
  uint32_t* s_bot = s_top + (size_t)((cap + 31) / 32) * M;                   // [cap/32][M] bottom halves
  __shared__ uint64_t bar;
  __shared__ uint32_t s_unit, s_qn, s_qhead, s_mode;
  __shared__ uint8_t s_q[64];
  __shared__ unsigned long long s_active, s_blended, s_written;
  __shared__ uint32_t s_cnt[64];  // (gaussian, half) entries per tile of the unit

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (read_status(a.fc)) return;
  const uint32_t n_units = a.fc->n_batches;
  uint32_t phase = 0;
  unsigned long long evals = 0, e_sup = 0, e_con = 0, e_live = 0;

  while (true) {
    if (tid == 0) {
      // a failed wait anywhere invalidates the frame: stop claiming units
      s_unit = read_status(a.fc) ? 0xffffffffu : atomicAdd(&a.fc->raster_claim, 1u);
      s_qhead = 0;
      s_blended = 0;
      s_written = 0;
    }
    if (tid < M) s_cnt[tid] = 0;
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
    const float4* rec_v = a.rec + (size_t)v * a.n * REC_F4;
    long long t_start = a.profile ? clock64() : 0;

    // gather the batch records: one bulk copy of 48 bytes per gaussian
    if (tid == 0) mbar_arrive_expect_tx(&bar, count * 48u);
    __syncthreads();
    for (uint32_t j = tid; j < count; j += RT) {
      const uint32_t id = a.vals[start + j];
      tma_load_1d(s_rec + (size_t)j * 3, rec_v + (size_t)id * REC_F4, 48u, &bar);
    }
    if (!mbar_wait_bounded(&bar, phase, a.wait_polls)) {
      set_status(a.fc, HG_ERR_DEVICE_TIMEOUT);
      atomicOr(&a.fc->timeout_where, 2u);
      mbar_wait_bounded(&bar, phase);  // the copies in flight land before the CTA exits
      return;
    }
    phase ^= 1u;
    long long t_loaded = a.profile ? clock64() : 0;

    // phase 1: per-gaussian tile masks, transposed to per-tile masks
    const int K = (int)((count + 31) / 32);
    build_tile_masks<MW, MH, true>(s_rec, s_top, s_bot, count, V, mtx0, mty0, RW, s_cnt);
    if (HALF) {
      // each thread rewrites the records of the gaussians it built masks for
      // (no other thread reads them before the barrier below) as half2 pairs
      // relative to the macro-tile centre (the smallest offsets, so the
      // finest half-precision spacing); the colour stays float32
      __syncwarp();
      const float ox = (float)((mtx0 + MW / 2) * TILE), oy = (float)((mty0 + MH / 2) * TILE);
      for (uint32_t j = (uint32_t)warp * 32 + lane; j < count; j += RT)
        half_record(s_rec + (size_t)j * 3, ox, oy);
    }
    __syncthreads();

    // tile work queue (warp 0), longest first: a tile's work is about the
    // number of gaussians in its mask, and claiming the longest tiles first
    // shortens the wait of the other warps at the end of the unit
    if (warp == 0) {
      constexpr int H = (M + 31) / 32;
      uint32_t key[H];
      unsigned long long act = 0;
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int t = h * 32 + lane;
        const uint32_t n = t < M ? s_cnt[t] : 0u;
        // key: count above, tile index below (distinct keys, ties by index)
        key[h] = n ? ((n << 6) | (uint32_t)(63 - t)) : 0u;
        act |= (unsigned long long)__ballot_sync(0xffffffffu, n != 0) << (h * 32);
      }
      // rank of each active tile among all active tiles by descending key
#pragma unroll
      for (int h = 0; h < H; ++h) {
        uint32_t rk = 0;
#pragma unroll
        for (int h2 = 0; h2 < H; ++h2)
          for (int src = 0; src < 32; ++src) rk += __shfl_sync(0xffffffffu, key[h2], src) > key[h];
        if (key[h]) s_q[rk] = (uint8_t)(h * 32 + lane);
      }
      if (lane == 0) {
        s_qn = (uint32_t)__popcll(act);
        s_active = act;
      }
    }
    // chain: wait for the previous batch of this macro-tile
    if (tid == 0) {
      const long long t_masks = a.profile ? clock64() : 0;
      uint32_t mode = BATCH_CHAINED;
      if (rank > 0) {
        mode = BATCH_LOCAL;
        for (uint32_t it = 0; it < (a.independent ? 0u : a.chain_polls); ++it) {
          const uint32_t c = ld_acquire(&a.chain[seg]);
          if (c == rank) {
            mode = BATCH_CHAINED;
            break;
          }
          if ((c & CHAIN_BROKEN) || read_status(a.fc)) break;
          __nanosleep(256);
        }
        // the backward needs every batch chained: a frame saved for it whose
        // chain wait gave up is invalid
        if (SAVE && mode == BATCH_LOCAL) {
          set_status(a.fc, HG_ERR_DEVICE_TIMEOUT);
          atomicOr(&a.fc->timeout_where, 16u);
        }
      }
      __threadfence();
      s_mode = mode;
      if (a.profile) {
        const long long t_chain = clock64();
        atomicAdd(&a.fc->raster_cycles[0], (unsigned long long)(t_loaded - t_start));
        atomicAdd(&a.fc->raster_cycles[1], (unsigned long long)(t_masks - t_loaded));
        atomicAdd(&a.fc->raster_cycles[2], (unsigned long long)(t_chain - t_masks));
        atomicAdd(&a.fc->raster_cycles[5], 1ull);
      }
    }
    __syncthreads();
    const long long t_p2 = a.profile ? clock64() : 0;
    const uint32_t qn = s_qn;
    const bool chained = s_mode == BATCH_CHAINED;
    // the last batch of a chained macro-tile writes the image itself
    const bool write_out =
        !SAVE && a.direct_out && chained && rank + 1 == a.first_batch[seg + 1] - a.first_batch[seg];

    // phase 2: warps claim tiles
    while (true) {
      uint32_t qi = 0;
      if (lane == 0) qi = atomicAdd(&s_qhead, 1u);
      qi = __shfl_sync(0xffffffffu, qi, 0);
      if (qi >= qn) break;
      const int t = s_q[qi];
      const int gtx = mtx0 + t % MW, gty = mty0 + t / MW;
      const int gt = V.tile_base + gty * V.tiles_x + gtx;
      const int px = gtx * TILE + (lane & 7);
      const int py = gty * TILE + (lane >> 3);
      const bool in0 = px < V.W && py < V.H, in1 = px < V.W && py + 4 < V.H;
      PixelAcc p0, p1;
      pixel_init(p0, in0);
      pixel_init(p1, in1);
      if (chained && __ldcg(&a.tile_rank[gt]) != 0) {
        pixel_load(p0, in0, __ldcg(&a.tile_state[(size_t)gt * TILE_PX + lane]));
        pixel_load(p1, in1, __ldcg(&a.tile_state[(size_t)gt * TILE_PX + lane + 32]));
      }
      // halves (4 pixel rows) with a live pixel; a half whose pixels have
      // all stopped takes no more gaussians (its blends would be no-ops)
      uint32_t on_t = __any_sync(0xffffffffu, pixel_live(p0)) ? ~0u : 0u;
      uint32_t on_b = __any_sync(0xffffffffu, pixel_live(p1)) ? ~0u : 0u;
      // every pixel already stopped in an earlier batch: nothing to blend
      if (!(on_t | on_b)) {
        if (write_out) {
          write_pixels(a, V, px, py, in0, in1, p0, p1);
          if (lane == 0) atomicOr(&s_written, 1ull << t);
        }
        continue;
      }
      if (lane == 0) atomicOr(&s_blended, 1ull << t);
      // SAVE: the batch's own colour is accumulated from zero (the colour
      // entering it is added back at the end), and the index of each pixel's
      // last contributing gaussian in the batch is kept
      uint32_t last0 = NO_LAST, last1 = NO_LAST;
      float3 cin0 = make_float3(0.f, 0.f, 0.f), cin1 = cin0;
      if (SAVE) {
        cin0 = make_float3(p0.r, p0.g, p0.b);
        cin1 = make_float3(p1.r, p1.g, p1.b);
        p0.r = p0.g = p0.b = p1.r = p1.g = p1.b = 0.f;
      }
      const float fpx = (float)px, fpy = (float)py, fpy1 = (float)(py + 4);
      // pixel coordinates relative to the macro-tile centre (half mode)
      const int hox = (mtx0 + MW / 2) * TILE, hoy = (mty0 + MH / 2) * TILE;
      const __half2 hpx = __float2half2_rn((float)(px - hox));
      const __half2 hpy = __floats2half2_rn((float)(py - hoy), (float)(py + 4 - hoy));
      uint32_t n_blend = 0;
      // gaussians of this tile in depth order: the set bits of its per
      // mini-batch masks (warp-uniform, bit-reversed: the highest set bit is
      // the nearest gaussian), blended directly; the per-half votes run
      // once per mini-batch
      for (int k = 0; k < K; ++k) {
        const uint32_t mt = s_top[k * M + t] & on_t, mb = s_bot[k * M + t] & on_b;
        uint32_t m = mt | mb;
        if (!m) continue;
        n_blend += __popc(mt) + __popc(mb);  // half-tiles evaluated (32 pixels each)
        const uint32_t jk = (uint32_t)k * 32 + 31;
        do {
          const int hb = 31 - __clz(m);
          const uint32_t bit = 1u << hb;
          m ^= bit;
          const uint32_t j = jk - (uint32_t)hb;
          if (HALF) {
            const float2 al = half_alpha2(s_rec + (size_t)j * 3, hpx, hpy);
            const float4 g2 = s_rec[j * 3 + 2];
            if (mt & bit) apply_alpha(p0, al.x, g2);
            if (mb & bit) apply_alpha(p1, al.y, g2);
          } else {
            const float4 g0 = s_rec[j * 3 + 0], g1 = s_rec[j * 3 + 1], g2 = s_rec[j * 3 + 2];
            const float ub = g0.z * (fpx - g0.x);
            if (STATS) {
              // support (e <= 9 log2(e) / 2) of the pixels still live
              const float dy0 = fpy - g0.y, dy1 = fpy1 - g0.y;
              const float u0 = fmaf(g0.w, dy0, ub), w0 = g1.x * dy0, u1 = fmaf(g0.w, dy1, ub), w1 = g1.x * dy1;
              e_sup += ((mt & bit) && pixel_live(p0) && fmaf(u0, u0, w0 * w0) <= SUPPORT_E) +
                       ((mb & bit) && pixel_live(p1) && fmaf(u1, u1, w1 * w1) <= SUPPORT_E);
              e_live += ((mt & bit) && pixel_live(p0)) + ((mb & bit) && pixel_live(p1));
            }
            // a half the gaussian cannot reach is skipped (its blend is a no-op)
            if (mt & bit) {
              const float w0 = blend(p0, ub, fpy - g0.y, g0, g1, g2);
              if (SAVE && w0 > 0.f) last0 = j;
              if (STATS) e_con += w0 > 0.f;
              if (mb & bit) {
                const float w1 = blend(p1, ub, fpy1 - g0.y, g0, g1, g2);
                if (SAVE && w1 > 0.f) last1 = j;
                if (STATS) e_con += w1 > 0.f;
              }
            } else {
              const float w1 = blend(p1, ub, fpy1 - g0.y, g0, g1, g2);
              if (SAVE && w1 > 0.f) last1 = j;
              if (STATS) e_con += w1 > 0.f;
            }
          }
        } while (m);
        on_t = __any_sync(0xffffffffu, pixel_live(p0)) ? ~0u : 0u;
        on_b = __any_sync(0xffffffffu, pixel_live(p1)) ? ~0u : 0u;
        if (!(on_t | on_b)) break;
      }
      if (lane == 0) evals += (unsigned long long)n_blend * 32ull;
      if (SAVE) {
        // the backward walks the batch back to front from its colour and the
        // transmittance after its last contributor
        float4* ex = a.exitrec + ((size_t)r * M + t) * TILE_PX;
        ex[lane] = make_float4(p0.r, p0.g, p0.b, pixel_final_T(p0));
        ex[lane + 32] = make_float4(p1.r, p1.g, p1.b, pixel_final_T(p1));
        uint16_t* la = a.exitlast + ((size_t)r * M + t) * TILE_PX;
        la[lane] = (uint16_t)last0;
        la[lane + 32] = (uint16_t)last1;
        p0.r += cin0.x;
        p0.g += cin0.y;
        p0.b += cin0.z;
        p1.r += cin1.x;
        p1.g += cin1.y;
        p1.b += cin1.z;
      }
      if (write_out) {
        write_pixels(a, V, px, py, in0, in1, p0, p1);
        if (lane == 0) atomicOr(&s_written, 1ull << t);
      } else if (chained) {
        float4* st = a.tile_state + (size_t)gt * TILE_PX;
        st[lane] = pixel_state(p0);
        st[lane + 32] = pixel_state(p1);
        if (lane == 0) a.tile_rank[gt] = rank + 1;
      } else {
        float4* out = a.partial + ((size_t)r * M + t) * TILE_PX;
        st_cs(out + lane, pixel_state(p0));
        st_cs(out + lane + 32, pixel_state(p1));
      }
    }
    if (write_out) {
      // the macro-tile's other tiles: their state after the last batch that
      // blended them, or the background
      __syncthreads();
      const unsigned long long done = s_written;
      for (int t = warp; t < M; t += RW) {
        if ((done >> t) & 1ull) continue;
        const int gtx = mtx0 + t % MW, gty = mty0 + t / MW;
        if (gtx >= V.tiles_x || gty >= V.tiles_y) continue;
        const int gt = V.tile_base + gty * V.tiles_x + gtx;
        const int px = gtx * TILE + (lane & 7), py = gty * TILE + (lane >> 3);
        const bool in0 = px < V.W && py < V.H, in1 = px < V.W && py + 4 < V.H;
        PixelAcc p0, p1;
        pixel_init(p0, in0);
        pixel_init(p1, in1);
        if (__ldcg(&a.tile_rank[gt]) != 0) {
          pixel_load(p0, in0, __ldcg(&a.tile_state[(size_t)gt * TILE_PX + lane]));
          pixel_load(p1, in1, __ldcg(&a.tile_state[(size_t)gt * TILE_PX + lane + 32]));
        }
        write_pixels(a, V, px, py, in0, in1, p0, p1);
      }
    }
    // publish: the tile states are visible before the chain advances
    __threadfence();
    long long t_warp_done = a.profile ? clock64() : 0;
    __syncthreads();
    if (a.profile && lane == 0) {
      const long long t_end = clock64();
      atomicAdd(&a.fc->raster_cycles[3], (unsigned long long)(t_warp_done - t_p2));
      atomicAdd(&a.fc->raster_cycles[4], (unsigned long long)(t_end - t_warp_done));
    }
    if (tid == 0) {
      a.active[r] = chained ? s_blended : s_active;
      a.mode[r] = chained ? BATCH_CHAINED : BATCH_LOCAL;
      if (write_out)
        atomicOr(&a.chain[seg], CHAIN_DONE);
      else if (chained)
        atomicCAS(&a.chain[seg], rank, rank + 1);
      else
        atomicOr(&a.chain[seg], CHAIN_BROKEN);
    }
  }
  if (lane == 0 && evals) atomicAdd(&a.fc->raster_evals, evals);
  if (STATS) {
    e_sup = warp_sum(e_sup);
    e_con = warp_sum(e_con);
    e_live = warp_sum(e_live);
    if (lane == 0) {
      atomicAdd(&a.fc->pixel_support_evals, e_sup);
      atomicAdd(&a.fc->pixel_contrib_evals, e_con);
      atomicAdd(&a.fc->pixel_live_evals, e_live);
    }
  }
}

template <int MW, int MH, bool SAVE, bool HALF, bool STATS = false>
cudaError_t launch_raster_kernel(const RasterArgs& a, int cap, cudaStream_t st) {
  constexpr int M = MW * MH;
  const size_t sm = (size_t)cap * 48 + (size_t)((cap + 31) / 32) * M * 8;
  cudaError_t e =
      cudaFuncSetAttribute(k_raster<MW, MH, SAVE, HALF, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int occ = 1, dev = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_raster<MW, MH, SAVE, HALF, STATS>, RT, sm);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (occ < 1) occ = 1;
  const int grid = a.persistent_ctas > 0 ? a.persistent_ctas : sms * occ;
  k_raster<MW, MH, SAVE, HALF, STATS><<<grid, RT, sm, st>>>(a, cap);
  note_launch();
  return cudaGetLastError();
}

template <int MW, int MH>
cudaError_t launch_raster_shape(const RasterArgs& a, int cap, cudaStream_t st) {
  if (a.exitrec) return launch_raster_kernel<MW, MH, true, false>(a, cap, st);
  if (a.fp16) return launch_raster_kernel<MW, MH, false, true>(a, cap, st);
  return a.profile ? launch_raster_kernel<MW, MH, false, false, true>(a, cap, st)
                   : launch_raster_kernel<MW, MH, false, false>(a, cap, st);
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
