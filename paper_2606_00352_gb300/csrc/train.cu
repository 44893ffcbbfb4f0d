// Loss and optimiser of the differentiable path (Sec. 6): the fused L2 loss
// with its gradient, and one fused Adam step over every parameter array of a
// scene.  Together with hg_render (save_for_backward) and hg_render_backward
// they make a densification-free optimisation step that runs entirely in
// this library's kernels.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"
#include "kernels.cuh"

namespace hg {

namespace {

constexpr int LOSS_THREADS = 1024;  // 2 blocks per SM (the block count is fixed): enough loads in flight

// dL/dC = C - C* per element; L = 1/2 sum (C - C*)^2.  Elements are taken
// four at a time (16-byte vectors when the three arrays allow it): the four
// squares are summed in float32, (d0^2 + d1^2) + (d2^2 + d3^2), and the
// group sums in double (FP64 arithmetic is slow on this part, so one double
// add per four elements).  The grid is fixed and so is the summation order
// (deterministic): per-block partials, which the last block to finish adds
// with a fixed reduction tree.
__device__ __forceinline__ float sq4(float a, float b, float c, float d) { return (a * a + b * b) + (c * c + d * d); }

__global__ void __launch_bounds__(LOSS_THREADS) k_l2_loss(const float* __restrict__ rgb,
                                                          const float* __restrict__ target, long long n,
                                                          float* __restrict__ dl, double* partial,
                                                          unsigned int* counter, double* loss) {
  __shared__ double red[LOSS_THREADS / 32];
  __shared__ bool last;
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * LOSS_THREADS;
  const bool vec = ((reinterpret_cast<uintptr_t>(rgb) | reinterpret_cast<uintptr_t>(target) |
                     reinterpret_cast<uintptr_t>(dl)) & 15u) == 0;
  const long long groups = n / 4;
  for (long long q = (long long)blockIdx.x * LOSS_THREADS + threadIdx.x; q < groups; q += stride) {
    float4 d;
    if (vec) {
      const float4 a = reinterpret_cast<const float4*>(rgb)[q], b = reinterpret_cast<const float4*>(target)[q];
      d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
      reinterpret_cast<float4*>(dl)[q] = d;
    } else {
      const long long i = q * 4;
      d = make_float4(rgb[i] - target[i], rgb[i + 1] - target[i + 1], rgb[i + 2] - target[i + 2],
                      rgb[i + 3] - target[i + 3]);
      dl[i] = d.x;
      dl[i + 1] = d.y;
      dl[i + 2] = d.z;
      dl[i + 3] = d.w;
    }
    acc += (double)sq4(d.x, d.y, d.z, d.w);
  }
  // the last n mod 4 elements: block 0, one thread each
  if (blockIdx.x == 0 && threadIdx.x < (int)(n - groups * 4)) {
    const long long i = groups * 4 + threadIdx.x;
    const float d = rgb[i] - target[i];
    dl[i] = d;
    acc += (double)(d * d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < LOSS_THREADS / 32; ++w) s += red[w];
    partial[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;  // block-uniform
  // the last block adds the partials with a fixed tree (one per thread, then
  // the warp and block reductions above), so the order is fixed and the
  // partials are read in parallel
  __threadfence();
  double v = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += LOSS_THREADS) v += __ldcg(&partial[b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < LOSS_THREADS / 32; ++w) s += red[w];
    *loss = 0.5 * s;
    *counter = 0;
  }
}

struct AdamGroup {
  float* p;
  const float* g;
  float* m;
  float* v;
  long long n;
  long long nv;  // 4-element vector units (0 when an array is not 16-byte aligned)
  float lr;
};

struct AdamArgs {
  AdamGroup grp[5];
  long long end[5];  // exclusive prefix ends of the groups, in units
  float b1, b2, c1, c2, eps;
};

__device__ __forceinline__ float adam_one(const AdamArgs& a, const AdamGroup& G, float g, float& m, float& v,
                                          float p) {
  m = fmaf(a.b1, m, (1.f - a.b1) * g);
  v = fmaf(a.b2, v, (1.f - a.b2) * g * g);
  return p - G.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
}

// One thread per unit of all five groups; a unit is four consecutive
// elements of a group (16-byte vectors) for the first nv units of the
// group, then single elements for the rest (the last count mod 4, or all of
// them when one of the group's arrays is not 16-byte aligned).
__global__ void __launch_bounds__(256) k_adam(AdamArgs a) {
  const long long total = a.end[4];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int k = 0;
    while (i >= a.end[k]) ++k;
    const long long u = i - (k ? a.end[k - 1] : 0);
    const AdamGroup& G = a.grp[k];
    const long long nv = G.nv;
    if (u < nv) {
      const float4 g = reinterpret_cast<const float4*>(G.g)[u];
      float4 m = reinterpret_cast<const float4*>(G.m)[u], v = reinterpret_cast<const float4*>(G.v)[u];
      float4 p = reinterpret_cast<const float4*>(G.p)[u];
      p.x = adam_one(a, G, g.x, m.x, v.x, p.x);
      p.y = adam_one(a, G, g.y, m.y, v.y, p.y);
      p.z = adam_one(a, G, g.z, m.z, v.z, p.z);
      p.w = adam_one(a, G, g.w, m.w, v.w, p.w);
      reinterpret_cast<float4*>(G.m)[u] = m;
      reinterpret_cast<float4*>(G.v)[u] = v;
      reinterpret_cast<float4*>(G.p)[u] = p;
    } else {
      const long long j = nv * 4 + (u - nv);
      float m = G.m[j], v = G.v[j];
      G.p[j] = adam_one(a, G, G.g[j], m, v, G.p[j]);
      G.m[j] = m;
      G.v[j] = v;
    }
  }
}

}  // namespace

}  // namespace hg

using namespace hg;

extern "C" hg_status hg_l2_loss(hg_ctx* ctx, const float* rgb, const float* target, int64_t n, float* dL_drgb,
                                double* loss, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!rgb || !target || !dL_drgb)) || !loss) {
    hg_set_error("hg_l2_loss: bad arguments");
    return HG_ERR_INVALID_ARG;
  }
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (!ctx->loss_scratch) {
    ctx->loss_scratch = ctx_alloc(ctx, LOSS_SCRATCH_BYTES, st);
    if (!ctx->loss_scratch) {
      hg_set_error("hg_l2_loss: scratch allocation failed");
      return HG_ERR_OOM;
    }
    if (cudaMemsetAsync(ctx->loss_scratch, 0, LOSS_SCRATCH_BYTES, st) != cudaSuccess) {
      hg_set_error("hg_l2_loss: scratch clear failed");
      return HG_ERR_CUDA;
    }
  }
  double* partial = (double*)ctx->loss_scratch;
  unsigned int* counter = (unsigned int*)(partial + LOSS_BLOCKS);
  k_l2_loss<<<LOSS_BLOCKS, LOSS_THREADS, 0, st>>>(rgb, target, (long long)n, dL_drgb, partial, counter, loss);
  note_launch();
  if (cudaGetLastError() != cudaSuccess) {
    hg_set_error("hg_l2_loss: launch failed");
    return HG_ERR_CUDA;
  }
  return HG_OK;
}

extern "C" hg_status hg_adam_step(hg_scene* scene, const float* const grads[5], float* const m[5],
                                  float* const v[5], const hg_adam_opts* o, void* stream) {
  if (!scene || !grads || !m || !v || !o || o->step < 1 || !(o->beta1 >= 0.f && o->beta1 < 1.f) ||
      !(o->beta2 >= 0.f && o->beta2 < 1.f) || !(o->eps >= 0.f)) {
    hg_set_error("hg_adam_step: bad arguments");
    return HG_ERR_INVALID_ARG;
  }
  if (scene->sh_storage != HG_SH_F32) {
    hg_set_error("hg_adam_step: the scene stores its SH in half precision (training needs float32)");
    return HG_ERR_INVALID_ARG;
  }
  AdamArgs a{};
  const long long k3 = (long long)(scene->deg + 1) * (scene->deg + 1) * 3;
  const long long counts[5] = {scene->n * 3, scene->n * 3, scene->n * 4, scene->n, scene->n * k3};
  long long end = 0;
  for (int k = 0; k < 5; ++k) {
    if (counts[k] > 0 && (!grads[k] || !m[k] || !v[k])) {
      hg_set_error("hg_adam_step: missing buffer");
      return HG_ERR_INVALID_ARG;
    }
    const bool aligned = ((reinterpret_cast<uintptr_t>(scene->arr[k]) | reinterpret_cast<uintptr_t>(grads[k]) |
                           reinterpret_cast<uintptr_t>(m[k]) | reinterpret_cast<uintptr_t>(v[k])) & 15u) == 0;
    const long long nv = aligned ? counts[k] / 4 : 0;
    a.grp[k] = AdamGroup{scene->arr[k], grads[k], m[k], v[k], counts[k], nv, o->lr[k]};
    end += nv + (counts[k] - 4 * nv);
    a.end[k] = end;
  }
  a.b1 = o->beta1;
  a.b2 = o->beta2;
  a.c1 = (float)(1.0 / (1.0 - std::pow((double)o->beta1, (double)o->step)));
  a.c2 = (float)(1.0 / (1.0 - std::pow((double)o->beta2, (double)o->step)));
  a.eps = o->eps;
  if (end == 0) return HG_OK;
  cudaSetDevice(scene->ctx->device);
  const long long blocks = std::min<long long>((end + 255) / 256, (long long)scene->ctx->sms * 16);
  k_adam<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(a);
  note_launch();
  if (cudaGetLastError() != cudaSuccess) {
    hg_set_error("hg_adam_step: launch failed");
    return HG_ERR_CUDA;
  }
  return HG_OK;
}
