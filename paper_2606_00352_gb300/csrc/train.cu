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

constexpr int LOSS_THREADS = 256;

// dL/dC = C - C* per element; L = 1/2 sum (C - C*)^2 accumulated in double
// with a fixed grid and a fixed summation order (deterministic): per-block
// partials, the last block to finish adds them in block order.
__global__ void __launch_bounds__(LOSS_THREADS) k_l2_loss(const float* __restrict__ rgb,
                                                          const float* __restrict__ target, long long n,
                                                          float* __restrict__ dl, double* partial,
                                                          unsigned int* counter, double* loss) {
  __shared__ double red[LOSS_THREADS / 32];
  __shared__ bool last;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * LOSS_THREADS + threadIdx.x; i < n;
       i += (long long)gridDim.x * LOSS_THREADS) {
    const float d = rgb[i] - target[i];
    dl[i] = d;
    acc += (double)d * (double)d;
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
  if (last && threadIdx.x == 0) {
    __threadfence();
    double s = 0.0;
    for (unsigned int b = 0; b < gridDim.x; ++b) s += ((volatile double*)partial)[b];
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
  float lr;
};

struct AdamArgs {
  AdamGroup grp[5];
  long long end[5];  // exclusive prefix ends of the groups in the flat index
  float b1, b2, c1, c2, eps;
};

// One thread per parameter element of all five groups.
__global__ void __launch_bounds__(256) k_adam(AdamArgs a) {
  const long long total = a.end[4];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int k = 0;
    while (i >= a.end[k]) ++k;
    const long long j = i - (k ? a.end[k - 1] : 0);
    const AdamGroup& G = a.grp[k];
    const float g = G.g[j];
    const float m = fmaf(a.b1, G.m[j], (1.f - a.b1) * g);
    const float v = fmaf(a.b2, G.v[j], (1.f - a.b2) * g * g);
    G.m[j] = m;
    G.v[j] = v;
    G.p[j] -= G.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
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
    a.grp[k] = AdamGroup{scene->arr[k], grads[k], m[k], v[k], counts[k], o->lr[k]};
    end += counts[k];
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
