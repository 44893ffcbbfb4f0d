// Backward of the render path (the paper sketches it in Sec. 6; it is not
// part of the paper's implementation).
//
//  k_bwd_suffix   one warp per render tile walks its macro-tile's batches
//                 from the last to the first and turns each blended batch's
//                 saved colour into the colour behind the batch: T_final bg
//                 plus the colours of the later batches, a running sum from
//                 the back (Sec. 6: the merge, read backwards, is a suffix
//                 scan over the batches).
//  k_raster_bwd   one CTA per processing unit (macro-tile batch), persistent.
//                 The unit's records are staged with TMA and its tile masks
//                 rebuilt exactly as in the forward.  For every tile the
//                 batch blended, a warp walks the batch's gaussians back to
//                 front, starting at each pixel's last contributor, from the
//                 transmittance the forward left after it and the colour
//                 behind the batch.  alpha_i is recomputed with the forward's
//                 arithmetic (same bits), T_i = T_{i+1} / (1 - a_i), and the
//                 colour behind gaussian i, S_i, grows from the back by
//                 c_i a_i T_i, so no difference of pixel-sized colours enters
//                 a gradient.
//                   dL/dc_i = v a_i T_i,  dL/da_i = sum_ch v (c_i T_i - S_i/(1-a_i)),
//                 chained to d mean2d, d conic, d opacity.  A gaussian's
//                 per-pixel terms are summed over the warp by a 16-value
//                 reduce-scatter (16 shuffles), accumulated per gaussian in
//                 shared memory, and flushed with one global atomic per
//                 (unit, gaussian, component).
//  k_project_bwd  one thread per gaussian, all views: recomputes the
//                 projection in float32 as the forward did and applies the
//                 chain rule through conic, EWA covariance, Jacobian, mean,
//                 quaternion, scales, sigmoid opacity and the SH colour
//                 (coefficients and view direction); the SH rows and their
//                 gradients move through shared memory in coalesced sweeps.
#include "internal.h"
#include "raster_common.cuh"

namespace hg {

namespace {

constexpr int BW = 8;
constexpr int BT = BW * 32;
constexpr int NG = 9;  // d mean2d x,y, d conic A,B,C, d opacity, d rgb

// Sum 16 per-lane values over the warp; lane l receives the total of value
// index (l >> 1) & 15 (recursive halving: 8 + 4 + 2 + 1 + 1 shuffles).
__device__ __forceinline__ float reduce_scatter16(float (&v)[16], int lane) {
  float w8[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const bool up = lane & 16;
    const float mine = up ? v[8 + k] : v[k];
    const float other = up ? v[k] : v[8 + k];
    w8[k] = mine + __shfl_xor_sync(0xffffffffu, other, 16);
  }
  float w4[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool up = lane & 8;
    const float mine = up ? w8[4 + k] : w8[k];
    const float other = up ? w8[k] : w8[4 + k];
    w4[k] = mine + __shfl_xor_sync(0xffffffffu, other, 8);
  }
  float w2[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool up = lane & 4;
    const float mine = up ? w4[2 + k] : w4[k];
    const float other = up ? w4[k] : w4[2 + k];
    w2[k] = mine + __shfl_xor_sync(0xffffffffu, other, 4);
  }
  const bool up = lane & 2;
  const float mine = up ? w2[1] : w2[0];
  const float other = up ? w2[0] : w2[1];
  float w1 = mine + __shfl_xor_sync(0xffffffffu, other, 2);
  w1 += __shfl_xor_sync(0xffffffffu, w1, 1);
  return w1;
}

// One gaussian at one pixel, walking back to front: T is the transmittance
// behind the gaussian (after it), S the colour behind it.  When the gaussian
// contributed (alpha > 0; the caller only passes gaussians up to the pixel's
// last contributor) its terms are added into g, T becomes the transmittance
// in front of it and S grows by its colour.
__device__ __forceinline__ void bwd_pixel(float& T, float3& S, float ub, float dx, float dy, const float4& g0,
                                          const float4& g1, const float4& g2, float cA, float cB, float cC,
                                          const float3& vv, float (&g)[16], bool& contrib) {
  float raw, ex;
  const float a = alpha_terms(ub, dy, g0, g1, g2, raw, ex);
  contrib = a > 0.f;
  if (!contrib) return;
  // 1 - a >= 0.01: the fast reciprocal's 2-ulp error, compounded over a
  // batch's walk, stays orders below the gradients' 1e-3 bound (the
  // correctly rounded division cost 12% of the backward)
  const float inv = __fdividef(1.f, 1.f - a);
  const float tb = T * inv;  // transmittance entering the gaussian
  const float wt = a * tb;
  g[6] += vv.x * wt;
  g[7] += vv.y * wt;
  g[8] += vv.z * wt;
  const float dal = vv.x * (g2.x * tb - S.x * inv) + vv.y * (g2.y * tb - S.y * inv) + vv.z * (g2.z * tb - S.z * inv);
  S.x = fmaf(g2.x, wt, S.x);
  S.y = fmaf(g2.y, wt, S.y);
  S.z = fmaf(g2.z, wt, S.z);
  T = tb;
  if (!(raw < ALPHA_MAX)) return;  // clamped alpha: no derivative
  g[5] += dal * ex;
  const float dq = dal * raw * -0.5f;
  g[2] += dq * dx * dx;
  g[3] += dq * 2.f * dx * dy;
  g[4] += dq * dy * dy;
  g[0] += dq * -2.f * (cA * dx + cB * dy);
  g[1] += dq * -2.f * (cB * dx + cC * dy);
}

__device__ __forceinline__ int find_view_tile(const ViewDesc* views, int n_views, int tile) {
  int v = 0;
  while (v + 1 < n_views && views[v + 1].tile_base <= tile) ++v;
  return v;
}

template <int MW, int MH>
__global__ void __launch_bounds__(256) k_bwd_suffix(SuffixArgs a) {
  constexpr int M = MW * MH;
  if (read_status(a.fc)) return;
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int tile = wg; tile < a.total_tiles; tile += nwarps) {
    const int v = find_view_tile(a.views, a.n_views, tile);
    const ViewDesc& V = a.views[v];
    const int lt = tile - V.tile_base;
    const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
    const int seg = V.seg_base + (ty / MH) * V.mgx + (tx / MW);
    const int tl = (ty % MH) * MW + (tx % MW);
    const uint32_t r0 = a.first_batch[seg], r1 = a.first_batch[seg + 1];
    bool first = true;
    float3 B0 = make_float3(0.f, 0.f, 0.f), B1 = B0;
    for (uint32_t r = r1; r-- > r0;) {
      if (!((a.active[r] >> tl) & 1ull)) continue;
      float4* ex = a.exitrec + ((size_t)r * M + tl) * TILE_PX;
      const float4 e0 = ex[lane], e1 = ex[lane + 32];
      if (first) {
        // the last batch that blended the tile leaves the final transmittance
        B0 = make_float3(e0.w * a.bg[0], e0.w * a.bg[1], e0.w * a.bg[2]);
        B1 = make_float3(e1.w * a.bg[0], e1.w * a.bg[1], e1.w * a.bg[2]);
        first = false;
      }
      ex[lane] = make_float4(B0.x, B0.y, B0.z, e0.w);
      ex[lane + 32] = make_float4(B1.x, B1.y, B1.z, e1.w);
      B0 = make_float3(B0.x + e0.x, B0.y + e0.y, B0.z + e0.z);
      B1 = make_float3(B1.x + e1.x, B1.y + e1.y, B1.z + e1.z);
    }
  }
}

template <int MW, int MH>
__global__ void __launch_bounds__(BT) k_raster_bwd(BackwardArgs a, int cap) {
  constexpr int M = MW * MH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s_rec = reinterpret_cast<float4*>(smem_raw);
  uint32_t* s_top = reinterpret_cast<uint32_t*>(s_rec + (size_t)cap * 3);
  uint32_t* s_bot = s_top + (size_t)((cap + 31) / 32) * M;
  float* s_grad = reinterpret_cast<float*>(s_bot + (size_t)((cap + 31) / 32) * M);
  __shared__ uint64_t bar;
  __shared__ uint32_t s_unit, s_qn, s_qhead;
  __shared__ uint8_t s_q[64];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (read_status(a.fc)) return;
  const uint32_t n_units = a.fc->n_batches;
  uint32_t phase = 0;
  const float k2 = 1.f / (CHOL_PRESCALE * CHOL_PRESCALE);
  while (true) {
    __syncthreads();  // every thread has read the previous unit's index
    if (tid == 0) {
      // a failed wait anywhere invalidates the pass: stop claiming units
      s_unit = read_status(a.fc) ? 0xffffffffu : atomicAdd(&a.fc->raster_claim, 1u);
      s_qhead = 0;
    }
    __syncthreads();
    const uint32_t u = s_unit;
    if (u >= n_units) break;
    const uint32_t r = a.batch_order[u];
    const unsigned long long act = a.active[r];
    if (act == 0) continue;  // uniform: the unit blended no tile
    const uint4 bt = a.batches[r];
    const uint32_t seg = bt.x, start = bt.y, count = bt.z;
    const int v = find_view(a.views, a.n_views, (int)seg);
    const ViewDesc& V = a.views[v];
    const int mloc = (int)seg - V.seg_base;
    const int mtx0 = (mloc % V.mgx) * MW, mty0 = (mloc / V.mgx) * MH;
    const float4* rec_v = a.rec + (size_t)v * a.n * REC_F4;
    if (tid == 0) mbar_arrive_expect_tx(&bar, count * 48u);
    __syncthreads();
    for (uint32_t j = tid; j < count; j += BT) {
      const uint32_t id = a.vals[start + j];
      tma_load_1d(s_rec + (size_t)j * 3, rec_v + (size_t)id * REC_F4, 48u, &bar);
    }
    for (uint32_t j = tid; j < count * NG; j += BT) s_grad[j] = 0.f;
    if (!mbar_wait_bounded(&bar, phase, a.wait_polls)) {
      set_status(a.fc, HG_ERR_DEVICE_TIMEOUT);
      atomicOr(&a.fc->timeout_where, 8u);
      mbar_wait_bounded(&bar, phase);  // the copies in flight land before the CTA exits
      return;
    }
    phase ^= 1u;
    build_tile_masks<MW, MH>(s_rec, s_top, s_bot, count, V, mtx0, mty0, BW);
    if (warp == 0) {
      int qn = 0;
#pragma unroll
      for (int h = 0; h < (M + 31) / 32; ++h) {
        const int t = h * 32 + lane;
        const bool hit = t < M && ((act >> t) & 1ull);
        const uint32_t bal = __ballot_sync(0xffffffffu, hit);
        if (hit) s_q[qn + __popc(bal & lanemask_lt())] = (uint8_t)t;
        qn += __popc(bal);
      }
      if (lane == 0) s_qn = (uint32_t)qn;
    }
    __syncthreads();
    const uint32_t qn = s_qn;
    while (true) {
      uint32_t qi = 0;
      if (lane == 0) qi = atomicAdd(&s_qhead, 1u);
      qi = __shfl_sync(0xffffffffu, qi, 0);
      if (qi >= qn) break;
      const int t = s_q[qi];
      const int gtx = mtx0 + t % MW, gty = mty0 + t / MW;
      const int px = gtx * TILE + (lane & 7), py = gty * TILE + (lane >> 3);
      const bool in0 = px < V.W && py < V.H, in1 = px < V.W && py + 4 < V.H;
      // {colour behind the batch, T after its last contributor} per pixel
      const size_t eo = ((size_t)r * M + t) * TILE_PX;
      const float4 e0 = a.exitrec[eo + lane], e1 = a.exitrec[eo + lane + 32];
      const uint32_t la0 = a.exitlast[eo + lane], la1 = a.exitlast[eo + lane + 32];
      const int l0 = la0 == NO_LAST ? -1 : (int)la0, l1 = la1 == NO_LAST ? -1 : (int)la1;
      float T0 = e0.w, T1 = e1.w;
      float3 S0 = make_float3(e0.x, e0.y, e0.z), S1 = make_float3(e1.x, e1.y, e1.z);
      float3 v0 = make_float3(0.f, 0.f, 0.f), v1 = v0;
      if (in0 && l0 >= 0) {
        const long long o = V.pix_base + (long long)py * V.W + px;
        v0 = make_float3(a.dl_drgb[o * 3 + 0], a.dl_drgb[o * 3 + 1], a.dl_drgb[o * 3 + 2]);
      }
      if (in1 && l1 >= 0) {
        const long long o = V.pix_base + (long long)(py + 4) * V.W + px;
        v1 = make_float3(a.dl_drgb[o * 3 + 0], a.dl_drgb[o * 3 + 1], a.dl_drgb[o * 3 + 2]);
      }
      const float fpx = (float)px, fpy = (float)py, fpy1 = (float)(py + 4);
      // the tile's gaussians back to front, from the warp's latest last
      // contributor: set bits of its mini-batch masks, highest first
      const int lm = __reduce_max_sync(0xffffffffu, max(l0, l1));
      for (int k = lm >> 5; k >= 0; --k) {
        const uint32_t mt = s_top[k * M + t], mb = s_bot[k * M + t];
        uint32_t m = mt | mb;
        if (k == (lm >> 5)) m &= 0xffffffffu >> (31 - (lm & 31));  // bits <= lm
        while (m) {
          const int b = 31 - __clz(m);
          const uint32_t bit = 1u << b;
          m ^= bit;
          const int j = k * 32 + b;
          const float4 g0 = s_rec[j * 3 + 0], g1 = s_rec[j * 3 + 1], g2 = s_rec[j * 3 + 2];
          const float cA = g0.z * g0.z * k2, cB = g0.z * g0.w * k2, cC = (g0.w * g0.w + g1.x * g1.x) * k2;
          const float dx = fpx - g0.x;
          const float ub = g0.z * dx;
          float gs[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) gs[q] = 0.f;
          // a half the gaussian cannot reach is skipped, as in the forward
          bool c0 = false, c1 = false;
          if ((mt & bit) && j <= l0) bwd_pixel(T0, S0, ub, dx, fpy - g0.y, g0, g1, g2, cA, cB, cC, v0, gs, c0);
          if ((mb & bit) && j <= l1) bwd_pixel(T1, S1, ub, dx, fpy1 - g0.y, g0, g1, g2, cA, cB, cC, v1, gs, c1);
          if (__any_sync(0xffffffffu, c0 || c1)) {
            const float tot = reduce_scatter16(gs, lane);
            const int idx = (lane >> 1) & 15;
            if ((lane & 1) == 0 && idx < NG && tot != 0.f) atomicAdd(&s_grad[j * NG + idx], tot);
          }
        }
      }
    }
    __syncthreads();
    float* g2d = a.g2d + (size_t)v * a.n * NG;
    for (uint32_t j = tid; j < count * NG; j += BT) {
      const float val = s_grad[j];
      if (val != 0.f) atomicAdd(&g2d[(size_t)a.vals[start + j / NG] * NG + j % NG], val);
    }
  }
}

// SH basis values and their derivatives with respect to the unit direction
// (the polynomials of the forward, differentiated term by term).
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float* Y, float* Yx, float* Yy, float* Yz) {
  const float C0 = 0.28209479177387814f;
  Y[0] = C0;
  Yx[0] = Yy[0] = Yz[0] = 0.f;
  if (DEG >= 1) {
    const float C1 = 0.48860251190291992f;
    Y[1] = -C1 * y, Yx[1] = 0.f, Yy[1] = -C1, Yz[1] = 0.f;
    Y[2] = C1 * z, Yx[2] = 0.f, Yy[2] = 0.f, Yz[2] = C1;
    Y[3] = -C1 * x, Yx[3] = -C1, Yy[3] = 0.f, Yz[3] = 0.f;
  }
  if (DEG >= 2) {
    const float C2a = 1.0925484305920792f, C2b = 0.31539156525252005f, C2c = 0.54627421529603959f;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = C2a * x * y, Yx[4] = C2a * y, Yy[4] = C2a * x, Yz[4] = 0.f;
    Y[5] = -C2a * y * z, Yx[5] = 0.f, Yy[5] = -C2a * z, Yz[5] = -C2a * y;
    Y[6] = C2b * (2.f * zz - xx - yy), Yx[6] = -2.f * C2b * x, Yy[6] = -2.f * C2b * y, Yz[6] = 4.f * C2b * z;
    Y[7] = -C2a * x * z, Yx[7] = -C2a * z, Yy[7] = 0.f, Yz[7] = -C2a * x;
    Y[8] = C2c * (xx - yy), Yx[8] = 2.f * C2c * x, Yy[8] = -2.f * C2c * y, Yz[8] = 0.f;
    if (DEG >= 3) {
      const float C3a = 0.59004358992664352f, C3b = 2.8906114426405538f, C3c = 0.45704579946446577f;
      const float C3d = 0.3731763325901154f, C3e = 1.4453057213202769f;
      const float t4 = 4.f * zz - xx - yy;
      Y[9] = -C3a * y * (3.f * xx - yy), Yx[9] = -6.f * C3a * x * y, Yy[9] = -3.f * C3a * (xx - yy), Yz[9] = 0.f;
      Y[10] = C3b * x * y * z, Yx[10] = C3b * y * z, Yy[10] = C3b * x * z, Yz[10] = C3b * x * y;
      Y[11] = -C3c * y * t4, Yx[11] = 2.f * C3c * x * y, Yy[11] = -C3c * (t4 - 2.f * yy), Yz[11] = -8.f * C3c * y * z;
      Y[12] = C3d * z * (2.f * zz - 3.f * xx - 3.f * yy), Yx[12] = -6.f * C3d * x * z, Yy[12] = -6.f * C3d * y * z,
      Yz[12] = C3d * (6.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = -C3c * x * t4, Yx[13] = -C3c * (t4 - 2.f * xx), Yy[13] = 2.f * C3c * x * y, Yz[13] = -8.f * C3c * x * z;
      Y[14] = C3e * z * (xx - yy), Yx[14] = 2.f * C3e * x * z, Yy[14] = -2.f * C3e * y * z, Yz[14] = C3e * (xx - yy);
      Y[15] = -C3a * x * (xx - 3.f * yy), Yx[15] = -3.f * C3a * (xx - yy), Yy[15] = 6.f * C3a * x * y, Yz[15] = 0.f;
    }
  }
}

// Chain rule of one gaussian i through all views: writes the gradients of
// its mean, log-scales, quaternion and opacity logit, and adds the SH
// gradient to dsh.  shr is the gaussian's SH row (K x 3 floats).
template <int DEG>
__device__ __forceinline__ void project_bwd_gaussian(const ProjectBackwardArgs& a, long long i, const float* shr,
                                                     float (&dsh)[(DEG + 1) * (DEG + 1) * 3]) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  const float px = a.means[i * 3 + 0], py = a.means[i * 3 + 1], pz = a.means[i * 3 + 2];
  const float sx = expf(a.log_scales[i * 3 + 0]), sy = expf(a.log_scales[i * 3 + 1]), sz = expf(a.log_scales[i * 3 + 2]);
  const float4 q = reinterpret_cast<const float4*>(a.quats)[i];
  const float op = 1.f / (1.f + expf(-a.opacity_logits[i]));
  const float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  const float qn = rsqrtf(qn2);
  const float w = q.x * qn, x = q.y * qn, y = q.z * qn, z = q.w * qn;
  const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                         {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                         {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
  const float S[3] = {sx, sy, sz};
  float M[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) M[r][c] = R[r][c] * S[c];
  float sig3[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) sig3[r][c] = M[r][0] * M[c][0] + M[r][1] * M[c][1] + M[r][2] * M[c][2];
  float dmu[3] = {0.f, 0.f, 0.f}, dM[3][3] = {}, dlogit = 0.f;
  for (int v = 0; v < a.n_views; ++v) {
    const float* g = a.g2d + ((size_t)v * a.n + i) * NG;
    float gv[NG];
    bool any = false;
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      gv[k] = g[k];
      any = any || gv[k] != 0.f;
    }
    if (!any) continue;
    const ViewDesc& V = a.views[v];
    const float tz = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(V.vm[8], px), __fmul_rn(V.vm[9], py)),
                                         __fmul_rn(V.vm[10], pz)),
                               V.vm[11]);
    if (!(tz > 0.2f)) continue;
    const float tx = fmaf(V.vm[0], px, fmaf(V.vm[1], py, fmaf(V.vm[2], pz, V.vm[3])));
    const float ty = fmaf(V.vm[4], px, fmaf(V.vm[5], py, fmaf(V.vm[6], pz, V.vm[7])));
    const float itz = 1.f / tz;
    const float limx = 1.3f * V.tan_x, limy = 1.3f * V.tan_y;
    const float uxr = tx * itz, uyr = ty * itz;
    const bool cx_ok = uxr > -limx && uxr < limx, cy_ok = uyr > -limy && uyr < limy;
    const float ux = fminf(fmaxf(uxr, -limx), limx), uy = fminf(fmaxf(uyr, -limy), limy);
    const float j00 = V.fx * itz, j02 = -V.fx * ux * itz, j11 = V.fy * itz, j12 = -V.fy * uy * itz;
    const float W[3][3] = {{V.vm[0], V.vm[1], V.vm[2]}, {V.vm[4], V.vm[5], V.vm[6]}, {V.vm[8], V.vm[9], V.vm[10]}};
    float T[2][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T[0][k] = j00 * W[0][k] + j02 * W[2][k];
      T[1][k] = j11 * W[1][k] + j12 * W[2][k];
    }
    // Sigma2 = T Sigma3 T^T + 0.3 I
    float TS[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) TS[r][c] = T[r][0] * sig3[0][c] + T[r][1] * sig3[1][c] + T[r][2] * sig3[2][c];
    const float ca = TS[0][0] * T[0][0] + TS[0][1] * T[0][1] + TS[0][2] * T[0][2] + 0.3f;
    const float cb = TS[0][0] * T[1][0] + TS[0][1] * T[1][1] + TS[0][2] * T[1][2];
    const float cc = TS[1][0] * T[1][0] + TS[1][1] * T[1][1] + TS[1][2] * T[1][2] + 0.3f;
    const float idet = 1.f / (ca * cc - cb * cb);
    const float A = cc * idet, B = -cb * idet, Cc = ca * idet;
    // dL/dSigma2 = -Ainv G Ainv, G = [[dA, dB/2], [dB/2, dC]]
    const float G00 = gv[2], G01 = 0.5f * gv[3], G11 = gv[4];
    const float P00 = A * G00 + B * G01, P01 = A * G01 + B * G11, P10 = B * G00 + Cc * G01, P11 = B * G01 + Cc * G11;
    const float D00 = -(P00 * A + P01 * B), D01 = -(P00 * B + P01 * Cc), D11 = -(P10 * B + P11 * Cc);
    const float D[2][2] = {{D00, D01}, {D01, D11}};
    // dT = 2 D T Sigma3 = 2 D TS
    float dT[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) dT[r][c] = 2.f * (D[r][0] * TS[0][c] + D[r][1] * TS[1][c]);
    // dSigma3 = T^T D T
    float dS3[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        dS3[r][c] = T[0][r] * (D00 * T[0][c] + D01 * T[1][c]) + T[1][r] * (D01 * T[0][c] + D11 * T[1][c]);
    // dM += 2 dSigma3 M
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) dM[r][c] += 2.f * (dS3[r][0] * M[0][c] + dS3[r][1] * M[1][c] + dS3[r][2] * M[2][c]);
    // dJ = dT W^T (entries J00, J02, J11, J12)
    const float dj00 = dT[0][0] * W[0][0] + dT[0][1] * W[0][1] + dT[0][2] * W[0][2];
    const float dj02 = dT[0][0] * W[2][0] + dT[0][1] * W[2][1] + dT[0][2] * W[2][2];
    const float dj11 = dT[1][0] * W[1][0] + dT[1][1] * W[1][1] + dT[1][2] * W[1][2];
    const float dj12 = dT[1][0] * W[2][0] + dT[1][1] * W[2][1] + dT[1][2] * W[2][2];
    float dt[3] = {0.f, 0.f, 0.f};
    const float itz2 = itz * itz;
    dt[2] += dj00 * (-V.fx * itz2) + dj11 * (-V.fy * itz2);
    if (cx_ok) {
      dt[0] += dj02 * (-V.fx * itz2);
      dt[2] += dj02 * (2.f * V.fx * tx * itz2 * itz);
    } else {
      dt[2] += dj02 * (V.fx * ux * itz2);
    }
    if (cy_ok) {
      dt[1] += dj12 * (-V.fy * itz2);
      dt[2] += dj12 * (2.f * V.fy * ty * itz2 * itz);
    } else {
      dt[2] += dj12 * (V.fy * uy * itz2);
    }
    // mean2d = (fx tx / tz + cx - 0.5, fy ty / tz + cy - 0.5)
    dt[0] += gv[0] * V.fx * itz;
    dt[1] += gv[1] * V.fy * itz;
    dt[2] += -(gv[0] * V.fx * tx + gv[1] * V.fy * ty) * itz2;
#pragma unroll
    for (int k = 0; k < 3; ++k) dmu[k] += W[0][k] * dt[0] + W[1][k] * dt[1] + W[2][k] * dt[2];
    // opacity
    dlogit += gv[5] * op * (1.f - op);
    // colour
    const float ddx = px - V.campos[0], ddy = py - V.campos[1], ddz = pz - V.campos[2];
    const float dist = sqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
    const float idn = 1.f / dist;
    const float ex = ddx * idn, ey = ddy * idn, ez = ddz * idn;
    float Y[16], Yx[16], Yy[16], Yz[16];
    sh_basis_grad<DEG>(ex, ey, ez, Y, Yx, Yy, Yz);
    float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) raw[c] = fmaf(Y[k], shr[k * 3 + c], raw[c]);
    float gc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) gc[c] = raw[c] > 0.f ? gv[6 + c] : 0.f;
    float gdx = 0.f, gdy = 0.f, gdz = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dsh[k * 3 + c] += Y[k] * gc[c];
        s = fmaf(shr[k * 3 + c], gc[c], s);
      }
      gdx = fmaf(Yx[k], s, gdx);
      gdy = fmaf(Yy[k], s, gdy);
      gdz = fmaf(Yz[k], s, gdz);
    }
    const float dot = ex * gdx + ey * gdy + ez * gdz;
    dmu[0] += (gdx - ex * dot) * idn;
    dmu[1] += (gdy - ey * dot) * idn;
    dmu[2] += (gdz - ez * dot) * idn;
  }
  // scales and rotation from dM (M = R diag(s))
  float ds[3], dR[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ds[c] = dM[0][c] * R[0][c] + dM[1][c] * R[1][c] + dM[2][c] * R[2][c];
#pragma unroll
    for (int r = 0; r < 3; ++r) dR[r][c] = dM[r][c] * S[c];
  }
  const float gw = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
  const float gx = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] - w * dR[1][2] + z * dR[2][0] +
                          w * dR[2][1] - 2.f * x * dR[2][2]);
  const float gy = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] - w * dR[2][0] +
                          z * dR[2][1] - 2.f * y * dR[2][2]);
  const float gz = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2.f * z * dR[1][1] +
                          y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
  const float qd = w * gw + x * gx + y * gy + z * gz;
  a.d_quats[i * 4 + 0] = (gw - w * qd) * qn;
  a.d_quats[i * 4 + 1] = (gx - x * qd) * qn;
  a.d_quats[i * 4 + 2] = (gy - y * qd) * qn;
  a.d_quats[i * 4 + 3] = (gz - z * qd) * qn;
  for (int k = 0; k < 3; ++k) {
    a.d_means[i * 3 + k] = dmu[k];
    a.d_log_scales[i * 3 + k] = ds[k] * S[k];
  }
  a.d_opacity_logits[i] = dlogit;
}

// One thread per gaussian.  The CTA's SH rows are read from and the SH
// gradient rows written to global memory by coalesced row-major sweeps
// through shared memory (rows padded to an odd stride, so the per-thread
// row accesses of a warp fall in distinct banks).
constexpr int PB_THREADS = 128;

template <int DEG>
__global__ void __launch_bounds__(PB_THREADS) k_project_bwd(ProjectBackwardArgs a) {
  constexpr int KS = (DEG + 1) * (DEG + 1) * 3;
  constexpr int ST = KS | 1;
  __shared__ float s_sh[PB_THREADS * ST];
  const int t = threadIdx.x;
  const long long base = (long long)blockIdx.x * PB_THREADS;
  const int rows = (int)min((long long)PB_THREADS, a.n - base);
  const float* src = a.sh + base * KS;
  for (int e = t; e < rows * KS; e += PB_THREADS) s_sh[(e / KS) * ST + e % KS] = src[e];
  __syncthreads();
  float dsh[KS];
#pragma unroll
  for (int k = 0; k < KS; ++k) dsh[k] = 0.f;
  if (t < rows) project_bwd_gaussian<DEG>(a, base + t, s_sh + t * ST, dsh);
  __syncthreads();
  if (t < rows) {
#pragma unroll
    for (int k = 0; k < KS; ++k) s_sh[t * ST + k] = dsh[k];
  }
  __syncthreads();
  float* dst = a.d_sh + base * KS;
  for (int e = t; e < rows * KS; e += PB_THREADS) dst[e] = s_sh[(e / KS) * ST + e % KS];
}

template <int MW, int MH>
cudaError_t launch_bwd_shape(const BackwardArgs& a, cudaStream_t st) {
  constexpr int M = MW * MH;
  const int cap = a.batch_cap;
  const size_t sm = (size_t)cap * 48 + (size_t)((cap + 31) / 32) * M * 8 + (size_t)cap * NG * 4;
  cudaError_t e = cudaFuncSetAttribute(k_raster_bwd<MW, MH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int occ = 1, dev = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_raster_bwd<MW, MH>, BT, sm);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_raster_bwd<MW, MH><<<sms * (occ < 1 ? 1 : occ), BT, sm, st>>>(a, cap);
  note_launch();
  return cudaGetLastError();
}

template <int DEG>
cudaError_t launch_pbwd_deg(const ProjectBackwardArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  k_project_bwd<DEG><<<(unsigned)((a.n + PB_THREADS - 1) / PB_THREADS), PB_THREADS, 0, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

template <int MW, int MH>
cudaError_t launch_suffix_shape(const SuffixArgs& a, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = min((a.total_tiles + 7) / 8, sms * 8);
  if (blocks < 1) blocks = 1;
  k_bwd_suffix<MW, MH><<<blocks, 256, 0, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bwd_suffix(const SuffixArgs& a, cudaStream_t st) {
  if (a.macro_w == 8 && a.macro_h == 4) return launch_suffix_shape<8, 4>(a, st);
  if (a.macro_w == 4 && a.macro_h == 4) return launch_suffix_shape<4, 4>(a, st);
  if (a.macro_w == 8 && a.macro_h == 8) return launch_suffix_shape<8, 8>(a, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_raster_backward(const BackwardArgs& a, cudaStream_t st) {
  if (a.macro_w == 8 && a.macro_h == 4) return launch_bwd_shape<8, 4>(a, st);
  if (a.macro_w == 4 && a.macro_h == 4) return launch_bwd_shape<4, 4>(a, st);
  if (a.macro_w == 8 && a.macro_h == 8) return launch_bwd_shape<8, 8>(a, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_project_backward(const ProjectBackwardArgs& a, cudaStream_t st) {
  switch (a.sh_degree) {
    case 0: return launch_pbwd_deg<0>(a, st);
    case 1: return launch_pbwd_deg<1>(a, st);
    case 2: return launch_pbwd_deg<2>(a, st);
    default: return launch_pbwd_deg<3>(a, st);
  }
}

}  // namespace hg

using namespace hg;

extern "C" hg_status hg_render_backward(hg_state* s, const float* dL_drgb, float* d_means, float* d_log_scales,
                                        float* d_quats, float* d_opacity_logits, float* d_sh, void* stream) {
  if (!s || !s->has_frame || !dL_drgb || !d_means || !d_log_scales || !d_quats || !d_opacity_logits || !d_sh) {
    hg_set_error("hg_render_backward: bad arguments");
    return HG_ERR_INVALID_ARG;
  }
  if (!s->opts.save_for_backward || s->opts.path != HG_PATH_HIGS || !s->scene) {
    hg_set_error("hg_render_backward: the frame was not rendered on the HiGS path with save_for_backward");
    return HG_ERR_INVALID_ARG;
  }
  if (s->scene->sh_storage != HG_SH_F32) {
    hg_set_error("hg_render_backward: the scene stores its SH in half precision (training needs float32)");
    return HG_ERR_INVALID_ARG;
  }
  cudaSetDevice(s->ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const FrameGeom& g = s->geom;
  const long long n = s->n;
  hg_status r = ws_ensure(s, G_DMEANS2, sizeof(float) * NG * (size_t)n * g.V + 16, st);
  if (r != HG_OK) return r;
  float* g2d = (float*)s->bufs[G_DMEANS2].p;
  FrameCounters* fc = (FrameCounters*)s->bufs[B_FC].p;
  // the pass starts with a clean status word (the forward completed with
  // HG_OK; a failed earlier backward of this frame leaves nothing behind)
  cudaError_t e = cudaMemsetAsync(g2d, 0, sizeof(float) * NG * (size_t)n * g.V, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(&fc->raster_claim, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(&fc->status, 0, sizeof(int), st);
  if (e != cudaSuccess) return hg_cuda_status(e, "backward clear");
  if (s->bwd_suffix_done != s->frame_id && n > 0) {
    // colour behind every batch, once per saved frame (in place)
    SuffixArgs sa{};
    sa.active = (const unsigned long long*)s->bufs[B_ACTIVE].p;
    sa.first_batch = (const uint32_t*)s->bufs[B_FIRSTB].p;
    sa.exitrec = (float4*)s->bufs[B_EXIT].p;
    sa.views = (const ViewDesc*)s->bufs[B_VIEWS].p;
    sa.n_views = g.V;
    sa.total_tiles = g.total_tiles;
    sa.macro_w = s->opts.macro_w;
    sa.macro_h = s->opts.macro_h;
    for (int c = 0; c < 3; ++c) sa.bg[c] = s->opts.bg[c];
    sa.fc = fc;
    if ((e = launch_bwd_suffix(sa, st)) != cudaSuccess) return hg_cuda_status(e, "backward suffix");
    s->bwd_suffix_done = s->frame_id;
  }
  if (n > 0) {
    BackwardArgs ba{};
    ba.rec = (const float4*)s->bufs[B_REC].p;
    ba.n = n;
    ba.views = (const ViewDesc*)s->bufs[B_VIEWS].p;
    ba.n_views = g.V;
    ba.vals = (const uint32_t*)s->bufs[B_VALS].p;
    ba.batches = (const uint4*)s->bufs[B_BATCHES].p;
    ba.batch_order = (const uint32_t*)s->bufs[B_BORDER].p;
    ba.active = (const unsigned long long*)s->bufs[B_ACTIVE].p;
    ba.exitrec = (float4*)s->bufs[B_EXIT].p;
    ba.exitlast = (const uint16_t*)s->bufs[B_EXITLAST].p;
    ba.dl_drgb = dL_drgb;
    ba.g2d = g2d;
    ba.batch_cap = s->opts.batch_cap;
    ba.macro_w = s->opts.macro_w;
    ba.macro_h = s->opts.macro_h;
    ba.wait_polls = s->ctx->wait_polls;
    ba.fc = fc;
    if ((e = launch_raster_backward(ba, st)) != cudaSuccess) return hg_cuda_status(e, "raster backward");
  }
  ProjectBackwardArgs pa{};
  const hg_scene* sc = s->scene;
  pa.means = sc->arr[0];
  pa.log_scales = sc->arr[1];
  pa.quats = sc->arr[2];
  pa.opacity_logits = sc->arr[3];
  pa.sh = sc->arr[4];
  pa.n = n;
  pa.sh_degree = sc->deg;
  pa.views = (const ViewDesc*)s->bufs[B_VIEWS].p;
  pa.n_views = g.V;
  pa.g2d = g2d;
  pa.d_means = d_means;
  pa.d_log_scales = d_log_scales;
  pa.d_quats = d_quats;
  pa.d_opacity_logits = d_opacity_logits;
  pa.d_sh = d_sh;
  if ((e = launch_project_backward(pa, st)) != cudaSuccess) return hg_cuda_status(e, "projection backward");
  // the device status of the pass, for hg_state_sync
  if ((e = cudaMemcpyAsync(s->fc_host, fc, sizeof(FrameCounters), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return hg_cuda_status(e, "backward status");
  s->last_stream = st;
  s->has_grad2d = true;
  return HG_OK;
}
