// Spatial storage order of a scene (a memory layout, not part of the
// paper's method): gaussians sorted by the 30-bit Morton code of their means,
// so that gaussians near in space, which land in the same macro-tiles, are
// near in memory.  The projection then writes the records of one screen
// region close together and the partition's fill writes its (key, id) pairs
// into few cache lines.
//   bounds  min / max of the finite coordinates per axis (order-preserving
//           integer images of the floats, atomics)
//   morton  q_a = min(1023, floor((x_a - lo_a) * s_a)), s_a = 1024 / (hi_a - lo_a)
//           (1 when the extent is 0), float32 round-to-nearest operations;
//           code bit 3 b + a = bit b of q_a; value = the gaussian's index
//   sort    single-segment onesweep over four 8-bit digits (stable: ties
//           keep index order)
//   gather  rows of a scene array by the permutation
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.cuh"

namespace hg {

namespace {

constexpr int ORDER_THREADS = 256;

// order-preserving map of floats to unsigned integers (total order of the
// finite values; -0 below +0)
__device__ __forceinline__ uint32_t float_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// mm[0..2] = min keys, mm[3..5] = max keys (initialised to ~0 / 0)
__global__ void __launch_bounds__(ORDER_THREADS) k_bounds(const float* means, long long n, uint32_t* mm) {
  uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float x = means[i * 3 + a];
      if (isfinite(x)) {
        const uint32_t k = float_key(x);
        lo[a] = min(lo[a], k);
        hi[a] = max(hi[a], k);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMin(&mm[a], lo[a]);
      atomicMax(&mm[3 + a], hi[a]);
    }
  }
}

// 10 bits of q spread to bit positions 0, 3, 6, ..., 27
__device__ __forceinline__ uint32_t spread3(uint32_t q) {
  q &= 0x3ffu;
  q = (q | (q << 16)) & 0x030000ffu;
  q = (q | (q << 8)) & 0x0300f00fu;
  q = (q | (q << 4)) & 0x030c30c3u;
  q = (q | (q << 2)) & 0x09249249u;
  return q;
}

__global__ void __launch_bounds__(ORDER_THREADS) k_morton(const float* means, long long n, const uint32_t* mm,
                                                          uint32_t* keys, uint32_t* vals) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t code = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const bool any = mm[a] <= mm[3 + a];  // some finite coordinate on this axis
    const float lo = any ? key_float(mm[a]) : 0.f, hi = any ? key_float(mm[3 + a]) : 0.f;
    const float ext = __fsub_rn(hi, lo);
    const float s = ext > 0.f ? __fdiv_rn(1024.f, ext) : 1.f;
    const float x = means[i * 3 + a];
    const float t = isfinite(x) ? __fmul_rn(__fsub_rn(x, lo), s) : 0.f;
    const int q = min(max((int)floorf(t), 0), 1023);
    code |= spread3((uint32_t)q) << a;
  }
  keys[i] = code;
  vals[i] = (uint32_t)i;
}

// onesweep tiles of one segment [0, n)
__global__ void k_order_tiles(long long n, uint4* tiles, FrameCounters* fc) {
  const uint32_t nt = (uint32_t)((n + OS_TILE - 1) / OS_TILE);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nt; k += gridDim.x * blockDim.x)
    tiles[k] = make_uint4(0u, k * OS_TILE, (uint32_t)min((long long)OS_TILE, n - (long long)k * OS_TILE), k);
  if (blockIdx.x == 0 && threadIdx.x == 0) fc->n_big_tiles = nt;
}

// dst row i = src row perm[i], rows of `words` 32-bit words
__global__ void __launch_bounds__(ORDER_THREADS) k_gather_rows(const uint32_t* src, uint32_t* dst,
                                                               const int32_t* perm, long long n, int words) {
  const long long total = n * words;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / words;
    const int w = (int)(e - i * words);
    dst[e] = src[(long long)perm[i] * words + w];
  }
}

// 16-byte rows variant (quaternions, packed SH, float32 SH rows of 48 words
// as 12 vectors)
__global__ void __launch_bounds__(ORDER_THREADS) k_gather_rows16(const uint4* src, uint4* dst, const int32_t* perm,
                                                                 long long n, int vecs) {
  const long long total = n * vecs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / vecs;
    const int w = (int)(e - i * vecs);
    dst[e] = src[(long long)perm[i] * vecs + w];
  }
}

}  // namespace

hg_status spatial_order(hg_ctx* ctx, const float* means, long long n, int32_t* perm, cudaStream_t st) {
  if (n == 0) return HG_OK;
  const long long nt = (n + OS_TILE - 1) / OS_TILE;
  // scratch: counters | min/max | tiles | digit histogram | look-back | keys, vals, alternates
  const size_t fc_b = 256, mm_b = 256, tiles_b = sizeof(uint4) * (size_t)nt, hist_b = sizeof(uint32_t) * 4 * 256,
               lb_b = sizeof(uint32_t) * 4 * 256 * (size_t)nt, kv_b = sizeof(uint32_t) * (size_t)n;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t total = fc_b + mm_b + up(tiles_b) + hist_b + up(lb_b) + 4 * up(kv_b);
  unsigned char* base = (unsigned char*)ctx_alloc(ctx, total, st);
  if (!base) return HG_ERR_OOM;
  unsigned char* p = base;
  FrameCounters* fc = (FrameCounters*)p;
  p += fc_b;
  uint32_t* mm = (uint32_t*)p;
  p += mm_b;
  uint4* tiles = (uint4*)p;
  p += up(tiles_b);
  uint32_t* hist = (uint32_t*)p;
  p += hist_b;
  uint32_t* lb = (uint32_t*)p;
  p += up(lb_b);
  uint32_t* keys = (uint32_t*)p;
  p += up(kv_b);
  uint32_t* vals = (uint32_t*)p;
  p += up(kv_b);
  uint32_t* keys2 = (uint32_t*)p;
  p += up(kv_b);
  uint32_t* vals2 = (uint32_t*)p;
  static_assert(sizeof(FrameCounters) <= 256, "counter block");
  const uint32_t mm_init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
  cudaError_t e = cudaMemsetAsync(fc, 0, fc_b, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mm, mm_init, sizeof(mm_init), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    const int grid = ctx->sms * 4;
    k_bounds<<<grid, ORDER_THREADS, 0, st>>>(means, n, mm);
    note_launch();
    k_morton<<<(unsigned)((n + ORDER_THREADS - 1) / ORDER_THREADS), ORDER_THREADS, 0, st>>>(means, n, mm, keys, vals);
    note_launch();
    k_order_tiles<<<(unsigned)min((nt + 255) / 256, 1024ll), 256, 0, st>>>(n, tiles, fc);
    note_launch();
    e = cudaGetLastError();
  }
  bool alt = false;
  if (e == cudaSuccess) {
    OsTileView tv{tiles, &fc->n_big_tiles, hist, nullptr, nullptr, nullptr};
    e = launch_onesweep<uint32_t, 4>(tv, keys, vals, keys2, vals2, hist, 4 * 256, true, lb, (size_t)nt * 256,
                                     fc->os_claim, 0, 4, ctx->wait_polls, fc, st, &alt);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(perm, alt ? vals2 : vals, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &fc->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  ctx_free(ctx, base, total, st);
  if (e != cudaSuccess) return hg_cuda_status(e, "spatial order");
  return (hg_status)status;
}

cudaError_t gather_rows(const void* src, void* dst, const int32_t* perm, long long n, size_t row_bytes,
                        cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const bool v16 = row_bytes % 16 == 0 && ((uintptr_t)src & 15) == 0 && ((uintptr_t)dst & 15) == 0;
  const long long units = n * (long long)(row_bytes / (v16 ? 16 : 4));
  const unsigned grid = (unsigned)min((units + ORDER_THREADS - 1) / ORDER_THREADS, 65536ll);
  if (v16)
    k_gather_rows16<<<grid, ORDER_THREADS, 0, st>>>((const uint4*)src, (uint4*)dst, perm, n, (int)(row_bytes / 16));
  else
    k_gather_rows<<<grid, ORDER_THREADS, 0, st>>>((const uint32_t*)src, (uint32_t*)dst, perm, n,
                                                  (int)(row_bytes / 4));
  note_launch();
  return cudaGetLastError();
}

}  // namespace hg

extern "C" hg_status hg_spatial_order(hg_ctx* ctx, const float* means, int64_t n, int32_t* perm, void* stream) {
  if (!ctx || n < 0 || n > (int64_t)0x3fffffff || (n > 0 && (!means || !perm))) {
    hg_set_error("hg_spatial_order: bad arguments");
    return HG_ERR_INVALID_ARG;
  }
  cudaSetDevice(ctx->device);
  return hg::spatial_order(ctx, means, n, perm, (cudaStream_t)stream);
}
