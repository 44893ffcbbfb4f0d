// Post-blend compositing (Sec. 3.4, Eq. 1; Sec. 4.5): one warp per render
// tile walks the batches of its macro-tile in depth order and accumulates
// C = C_0 + T_0 C_1 + T_0 T_1 C_2 + ..., reading a batch's partial only when
// the batch's active-tile mask has the tile's bit.
//
// Batches the rasteriser rendered in order (chained) already hold the exact
// result in the per-tile state; the merge starts from it.  For batches
// rendered from T = 1 (a broken chain), exact per-pixel termination across
// batches: let T_acc be the transmittance entering batch k.  If the pixel stopped inside batch k, or T_acc T_k < 1e-4,
// the 3DGS stop lies inside batch k; unless T_acc = 1 (then the local stop is
// the global one) the warp replays batch k for that pixel from T_acc with the
// same blend arithmetic as the rasteriser.
#include "blend.cuh"
#include "kernels.cuh"

namespace hg {

namespace {

__device__ __forceinline__ int find_view_tile(const ViewDesc* views, int n_views, int tile) {
  int v = 0;
  while (v + 1 < n_views && views[v + 1].tile_base <= tile) ++v;
  return v;
}

__device__ __forceinline__ void apply_partial(PixelAcc& p, const float4& q, bool& need) {
  need = false;
  if (!pixel_live(p)) return;
  const float tk = fabsf(q.w);
  const bool st = signbit(q.w);
  if (st || p.T * tk < T_EPS) {
    if (p.T == 1.f && st) {
      p.r += q.x;
      p.g += q.y;
      p.b += q.z;
      p.U = tk;
      p.T = 0.f;
    } else {
      need = true;
    }
    return;
  }
  p.r = fmaf(p.T, q.x, p.r);
  p.g = fmaf(p.T, q.y, p.g);
  p.b = fmaf(p.T, q.z, p.b);
  p.T *= tk;
  p.U = p.T;
}

__device__ __forceinline__ float4 shfl4(const float4& v, int src) {
  return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                     __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}

template <int MW, int MH>
__global__ void __launch_bounds__(256) k_merge(MergeArgs a) {
  pdl_wait();
  constexpr int M = MW * MH;
  if (read_status(a.fc)) return;
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long replays = 0;
  for (int tile = wg; tile < a.total_tiles; tile += nwarps) {
    const int v = find_view_tile(a.views, a.n_views, tile);
    const ViewDesc& V = a.views[v];
    const int lt = tile - V.tile_base;
    const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
    const int seg = V.seg_base + (ty / MH) * V.mgx + (tx / MW);
    if (a.chain[seg] & CHAIN_DONE) continue;  // written by the rasteriser
    const int tl = (ty % MH) * MW + (tx % MW);
    const int px = tx * TILE + (lane & 7), py = ty * TILE + (lane >> 3);
    const bool in0 = px < V.W && py < V.H, in1 = px < V.W && py + 4 < V.H;
    const float fpx = (float)px, fpy = (float)py, fpy1 = (float)(py + 4);
    PixelAcc p0, p1;
    pixel_init(p0, in0);
    pixel_init(p1, in1);
    const uint32_t r0 = a.first_batch[seg], r1 = a.first_batch[seg + 1];
    const float4* rec_v = a.rec + (size_t)v * a.n * REC_F4;
    // batches rendered in order from the exact entering transmittance: their
    // result is the per-tile state
    uint32_t g = r0;
    while (g < r1 && a.mode[g] == BATCH_CHAINED) ++g;
    if (g > r0 && a.tile_rank[tile] != 0) {
      pixel_load(p0, in0, a.tile_state[(size_t)tile * TILE_PX + lane]);
      pixel_load(p1, in1, a.tile_state[(size_t)tile * TILE_PX + lane + 32]);
    }
    // the rest (batches rendered from T = 1): Eq. 1 with replay
    for (uint32_t r = g; r < r1; ++r) {
      if (!__any_sync(0xffffffffu, pixel_live(p0) || pixel_live(p1))) break;
      if (!((a.active[r] >> tl) & 1ull)) continue;
      const float4* src = a.partial + ((size_t)r * M + tl) * TILE_PX;
      const float4 q0 = src[lane], q1 = src[lane + 32];
      bool need0, need1;
      apply_partial(p0, q0, need0);
      apply_partial(p1, q1, need1);
      const uint32_t nb0 = __ballot_sync(0xffffffffu, need0), nb1 = __ballot_sync(0xffffffffu, need1);
      if (!(nb0 | nb1)) continue;
      if (lane == 0) replays += __popc(nb0) + __popc(nb1);
      // replay batch r from T_acc for the pixels that need it
      PixelAcc q0r, q1r;
      pixel_init(q0r, need0, p0.T);
      pixel_init(q1r, need1, p1.T);
      const uint4 bt = a.batches[r];
      for (uint32_t c = 0; c < bt.z; c += 32) {
        if (!__any_sync(0xffffffffu, pixel_live(q0r) || pixel_live(q1r))) break;
        const uint32_t j = c + lane;
        float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0, g2 = g0;
        bool ov = false;
        if (j < bt.z) {
          const uint32_t id = a.vals[bt.y + j];
          const float4* rp = rec_v + (size_t)id * REC_F4;
          g0 = rp[0];
          g1 = rp[1];
          g2 = rp[2];
          int x0, x1, y0, y1;
          tile_rect(g0, g1, x0, x1, y0, y1);
          ov = x0 <= tx && tx <= x1 && y0 <= ty && ty <= y1;
        }
        uint32_t bal = __ballot_sync(0xffffffffu, ov);
        while (bal) {
          const int b = __ffs(bal) - 1;
          bal &= bal - 1;
          const float4 h0 = shfl4(g0, b), h1 = shfl4(g1, b), h2 = shfl4(g2, b);
          const float ub = h0.z * (fpx - h0.x);
          blend(q0r, ub, fpy - h0.y, h0, h1, h2);
          blend(q1r, ub, fpy1 - h0.y, h0, h1, h2);
        }
      }
      if (need0) {
        p0.r += q0r.r;
        p0.g += q0r.g;
        p0.b += q0r.b;
        p0.T = q0r.T;
        p0.U = q0r.U;
      }
      if (need1) {
        p1.r += q1r.r;
        p1.g += q1r.g;
        p1.b += q1r.b;
        p1.T = q1r.T;
        p1.U = q1r.U;
      }
    }
    if (in0) {
      const long long o = V.pix_base + (long long)py * V.W + px;
      const float tf = pixel_final_T(p0);
      const float4 f = make_float4(fmaf(tf, a.bg[0], p0.r), fmaf(tf, a.bg[1], p0.g), fmaf(tf, a.bg[2], p0.b), tf);
      a.out_rgb[o * 3 + 0] = f.x;
      a.out_rgb[o * 3 + 1] = f.y;
      a.out_rgb[o * 3 + 2] = f.z;
      if (a.out_T) a.out_T[o] = tf;
    }
    if (in1) {
      const long long o = V.pix_base + (long long)(py + 4) * V.W + px;
      const float tf = pixel_final_T(p1);
      const float4 f = make_float4(fmaf(tf, a.bg[0], p1.r), fmaf(tf, a.bg[1], p1.g), fmaf(tf, a.bg[2], p1.b), tf);
      a.out_rgb[o * 3 + 0] = f.x;
      a.out_rgb[o * 3 + 1] = f.y;
      a.out_rgb[o * 3 + 2] = f.z;
      if (a.out_T) a.out_T[o] = tf;
    }
  }
  if (lane == 0 && replays) atomicAdd(&a.fc->replays, replays);
}

template <int MW, int MH>
cudaError_t launch_merge_shape(const MergeArgs& a, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = min((a.total_tiles + 7) / 8, sms * 8);
  if (blocks < 1) blocks = 1;
  // launches while the rasteriser drains (programmatic dependent launch)
  return launch_pdl(k_merge<MW, MH>, dim3(blocks), dim3(256), 0, st, a);
}

}  // namespace

cudaError_t launch_merge(const MergeArgs& a, cudaStream_t st) {
  if (a.macro_w == 8 && a.macro_h == 4) return launch_merge_shape<8, 4>(a, st);
  if (a.macro_w == 4 && a.macro_h == 4) return launch_merge_shape<4, 4>(a, st);
  if (a.macro_w == 8 && a.macro_h == 8) return launch_merge_shape<8, 8>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace hg
