// Device-side building blocks shared by the render kernels: frame layout,
// status word, TMA bulk copies with bounded mbarrier waits, warp scans.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/higs.h"

namespace hg {

constexpr int TILE = 8;            // render tile edge in pixels (Sec. 3.1)
constexpr int TILE_SHIFT = 3;      // floor(a / TILE) = a >> TILE_SHIFT (arithmetic shift)
constexpr int TILE_PX = TILE * TILE;
constexpr int BP = 8192;           // partitioning batch B_p (Sec. 3.2)
constexpr float T_EPS = 1e-4f;     // termination threshold
constexpr float ALPHA_MIN = 1.0f / 255.0f;
constexpr float ALPHA_MAX = 0.99f;
// sqrt(log2(e) / 2): Cholesky factors of the conic are prescaled by this so
// that alpha = o * exp2(-e) with e = q log2(e) / 2 (Sec. 4.5, numerical format)
constexpr float CHOL_PRESCALE = 0.84932180028801906868f;
// q <= 9 in prescaled units: 9 log2(e) / 2
constexpr float SUPPORT_E = 6.49212768400033546357f;
constexpr int MAX_VIEWS = 64;
// Raster records: 48 bytes of data at a 64-byte stride in global memory, so
// that a record never straddles two 64-byte DRAM access chunks.
constexpr int REC_F4 = 4;
constexpr int RADIUS_MAX = 1 << 20;
constexpr uint32_t SPIN_LIMIT = 1u << 24;  // bounded device waits (polls), default
constexpr uint32_t CHAIN_SPIN = 200000;    // batch-chain polls (~0.1 s) before a unit renders unchained

// Per-view geometry, uploaded once per frame.
struct ViewDesc {
  float vm[12];          // rows 0..2 of the world->camera matrix
  float fx, fy, cx, cy;
  float campos[3];
  float tan_x, tan_y;    // W / (2 fx), H / (2 fy)
  int W, H;
  int tiles_x, tiles_y;  // render-tile grid
  int mgx, mgy;          // macro-tile grid
  int seg_base;          // first global segment (macro-tile) of the view
  int tile_base;         // first global render tile of the view
  long long pix_base;    // first pixel of the view in the packed outputs
};

// Device counters of one frame (zeroed at frame start).
struct FrameCounters {
  int status;              // hg_status of the first device failure
  uint32_t n_pairs;
  uint32_t n_batches;
  uint32_t n_big_tiles;
  uint32_t n_big_segs;
  uint32_t max_seg;
  uint32_t tier_count[6];
  uint32_t n_visible;
  uint32_t raster_claim;
  uint32_t merge_claim;
  uint32_t os_claim[8];
  uint32_t tier_claim[6];  // next list entry of each SMEM sort tier (dynamic claiming)
  uint32_t timeout_where;
  uint32_t sort_resorts;   // shared-memory sort segments sorted again (a long run in one bucket)
  unsigned long long replays;
  unsigned long long raster_evals;
  // HG_FLAG_PROFILE: the intrinsic per-pixel work of the frame (support
  // evaluations of live pixels up to their stop; contributing ones)
  unsigned long long pixel_support_evals;
  unsigned long long pixel_contrib_evals;
  unsigned long long pixel_live_evals;  // evaluations of pixels still live
  // rasteriser phase cycles summed over units (HG_FLAG_PROFILE): load, masks,
  // chain wait, blend (per warp, summed), end barrier (per warp, summed), units
  unsigned long long raster_cycles[6];
};

__device__ __forceinline__ void set_status(FrameCounters* fc, int code) {
  atomicCAS(&fc->status, 0, code);
}

__device__ __forceinline__ int read_status(const FrameCounters* fc) {
  return *((volatile const int*)&fc->status);
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the previous kernel of its stream is still
// finishing; it calls pdl_wait() before it reads anything that kernel
// wrote (the previous grid has then completed and its writes are visible).
// Without that launch attribute the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ------------------------------------------------------------ mbarrier + TMA
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of `bar` with at most `polls` polls (0: give up at
// once); returns false on timeout (the caller records HG_ERR_DEVICE_TIMEOUT
// and then waits, with the default limit, for its copies still in flight).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t polls = SPIN_LIMIT) {
  for (uint32_t it = 0; it < polls; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// 1-D bulk copy global -> shared completing on `bar` (both addresses 16-byte
// aligned, bytes a multiple of 16).
__device__ __forceinline__ void tma_load_1d(void* smem_dst, const void* gmem_src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(smem_dst)),
      "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// 1-D bulk copy shared -> global (bulk-group completion).
__device__ __forceinline__ void tma_store_1d(void* gmem_dst, const void* smem_src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gmem_dst),
               "r"(smem_u32(smem_src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void tma_store_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void tma_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// streaming (evict-first) 16-byte store
__device__ __forceinline__ void st_cs(float4* p, float4 v) {
  asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

// ------------------------------------------------------------------ scans
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) >= o) v += n;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Exclusive block scan of one value per thread; `tmp` holds >= 33 entries.
// Returns the exclusive prefix; *total receives the block sum.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* tmp, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? tmp[lane] : T(0);
    T wi = warp_incl_scan(w);
    if (lane < nw) tmp[lane] = wi - w;
    if (lane == nw - 1) tmp[32] = wi;
  }
  __syncthreads();
  T res = tmp[warp] + inc - v;
  if (total) *total = tmp[32];
  __syncthreads();
  return res;
}

__device__ __forceinline__ int find_view(const ViewDesc* views, int n_views, int seg) {
  int v = 0;
  while (v + 1 < n_views && views[v + 1].seg_base <= seg) ++v;
  return v;
}

}  // namespace hg
