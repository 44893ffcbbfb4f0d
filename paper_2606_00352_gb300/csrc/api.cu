// C ABI: contexts, scenes, frame workspaces and the render pipeline driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "binning.cuh"
#include "internal.h"
#include "sh_codec.cuh"

using namespace hg;

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

namespace hg {
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_issued() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace hg

void hg_set_error(const std::string& s) { g_last_error = s; }

hg_status hg_cuda_status(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return HG_OK;
  hg_set_error(std::string(where) + ": " + cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return HG_ERR_OOM;
  return HG_ERR_CUDA;
}

#define HG_TRY(expr, where)                                   \
  do {                                                        \
    cudaError_t e__ = (expr);                                 \
    if (e__ != cudaSuccess) return hg_cuda_status(e__, where); \
  } while (0)

extern "C" const char* hg_status_str(hg_status s) {
  switch (s) {
    case HG_OK: return "ok";
    case HG_ERR_INVALID_ARG: return "invalid argument";
    case HG_ERR_OOM: return "out of device memory";
    case HG_ERR_CUDA: return "CUDA error";
    case HG_ERR_CAPACITY: return "workspace capacity exceeded";
    case HG_ERR_DEVICE_TIMEOUT: return "bounded device wait timed out";
    case HG_ERR_BUSY: return "busy";
    case HG_ERR_NOT_FOUND: return "not found";
    case HG_ERR_CANCELLED: return "cancelled";
    case HG_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

extern "C" const char* hg_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* hg_version(void) { return "higs-gb300 0.1 (sm_103a)"; }
extern "C" int64_t hg_kernel_launches(void) { return hg::launches_issued(); }

// Stage timing events: inside a stream capture an event record must be an
// external node to be recorded when the graph runs.
static cudaError_t record_stage(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    return cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
  return cudaEventRecord(ev, st);
}

// ---------------------------------------------------------------- memory
void* ctx_alloc(hg_ctx* ctx, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 256;
  if (ctx->has_alloc) return ctx->alloc.alloc(bytes, (void*)st, ctx->alloc.user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void ctx_free(hg_ctx* ctx, void* p, size_t bytes, cudaStream_t st) {
  if (!p) return;
  if (ctx->has_alloc)
    ctx->alloc.free(p, bytes, (void*)st, ctx->alloc.user);
  else
    cudaFree(p);
}

hg_status ws_ensure(hg_state* s, int id, size_t bytes, cudaStream_t st) {
  Buf& b = s->bufs[id];
  if (b.bytes >= bytes && b.p) return HG_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    hg_set_error("workspace buffer " + std::to_string(id) + " must grow to " + std::to_string(bytes) +
                 " bytes during graph capture");
    return HG_ERR_CAPACITY;
  }
  if (b.p) {
    // the old buffer may still be read by work queued earlier on any stream
    cudaDeviceSynchronize();
    ctx_free(s->ctx, b.p, b.bytes, st);
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t want = bytes + bytes / 8 + 256;
  want = (want + 255) & ~size_t(255);
  b.p = ctx_alloc(s->ctx, want, st);
  if (!b.p) {
    hg_set_error("workspace allocation of " + std::to_string(want) + " bytes failed");
    return HG_ERR_OOM;
  }
  b.bytes = want;
  return HG_OK;
}

// ---------------------------------------------------------------- context
extern "C" hg_status hg_ctx_create(int device, const hg_allocator* alloc, hg_ctx** out) {
  if (!out) return HG_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  HG_TRY(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) {
    hg_set_error("device index out of range");
    return HG_ERR_INVALID_ARG;
  }
  HG_TRY(cudaSetDevice(device), "cudaSetDevice");
  hg_ctx* c = new hg_ctx();
  c->device = device;
  if (alloc && alloc->alloc && alloc->free) {
    c->alloc = *alloc;
    c->has_alloc = true;
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  *out = c;
  return HG_OK;
}

extern "C" void hg_ctx_destroy(hg_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->internal) hg_state_free(ctx->internal);
  if (ctx->loss_scratch) {
    cudaDeviceSynchronize();
    ctx_free(ctx, ctx->loss_scratch, LOSS_SCRATCH_BYTES, nullptr);
  }
  delete ctx;
}

extern "C" hg_status hg_ctx_set_wait_limits(hg_ctx* ctx, int64_t wait_polls, int64_t chain_polls) {
  if (!ctx || wait_polls > (int64_t)0xffffffffu || chain_polls > (int64_t)0xffffffffu) {
    hg_set_error("hg_ctx_set_wait_limits: bad arguments");
    return HG_ERR_INVALID_ARG;
  }
  ctx->wait_polls = wait_polls < 0 ? SPIN_LIMIT : (uint32_t)wait_polls;
  ctx->chain_polls = chain_polls < 0 ? CHAIN_SPIN : (uint32_t)chain_polls;
  return HG_OK;
}

// ---------------------------------------------------------------- scenes
extern "C" hg_status hg_create_scene(hg_ctx* ctx, const hg_scene_desc* d, hg_scene** out) {
  if (!ctx || !d || !out || d->n < 0 || d->sh_degree < 0 || d->sh_degree > 3 || d->sh_storage < HG_SH_F32 ||
      d->sh_storage > HG_SH_CODEC32 || (d->sh_storage == HG_SH_CODEC32 && d->sh_degree != 3) ||
      (d->order != HG_ORDER_INPUT && d->order != HG_ORDER_SPATIAL) || (d->order == HG_ORDER_SPATIAL && d->borrow)) {
    hg_set_error("hg_create_scene: bad arguments");
    return HG_ERR_INVALID_ARG;
  }
  if (d->n > (int64_t)0x3fffffff) {
    hg_set_error("hg_create_scene: more than 2^30 gaussians");
    return HG_ERR_INVALID_ARG;
  }
  if (d->n > 0 && (!d->means || !d->log_scales || !d->quats || !d->opacity_logits || !d->sh)) {
    hg_set_error("hg_create_scene: null array");
    return HG_ERR_INVALID_ARG;
  }
  cudaSetDevice(ctx->device);
  hg_scene* s = new hg_scene();
  s->ctx = ctx;
  s->n = d->n;
  s->deg = d->sh_degree;
  const int K = (d->sh_degree + 1) * (d->sh_degree + 1);
  s->sh_storage = d->sh_storage;
  const void* src[5] = {d->means, d->log_scales, d->quats, d->opacity_logits, d->sh};
  const size_t per[5] = {3, 3, 4, 1, (size_t)K * 3};
  const bool codec = d->sh_storage == HG_SH_CODEC32;
  const size_t esz[5] = {4, 4, 4, 4, d->sh_storage == HG_SH_F32 ? 4u : 2u};
  bool aligned = true;
  for (int i = 0; i < 5; ++i) aligned = aligned && (((uintptr_t)src[i]) & 15) == 0;
  s->owned = !(d->borrow && aligned) || codec;
  for (int i = 0; i < 5; ++i) {
    s->bytes[i] = codec && i == 4 ? sizeof(uint32_t) * SH_CODEC_WORDS * (size_t)d->n : per[i] * esz[i] * (size_t)d->n;
    if (codec && i == 4) {
      // packed SH: encoded here from the float32 coefficients
      s->arr[i] = (float*)ctx_alloc(ctx, s->bytes[i], nullptr);
      s->sh_scale = (float*)ctx_alloc(ctx, sizeof(float) * 2 * SH_CODEC_CH, nullptr);
      if (!s->arr[i] || !s->sh_scale) {
        hg_destroy_scene(s);
        hg_set_error("hg_create_scene: allocation failed");
        return HG_ERR_OOM;
      }
      const hg_status r = sh_codec_encode(ctx, (const float*)src[i], d->n, (uint32_t*)s->arr[i], s->sh_scale,
                                          s->sh_scale + SH_CODEC_CH);
      if (r != HG_OK) {
        hg_destroy_scene(s);
        return r;
      }
      continue;
    }
    if (s->owned) {
      s->arr[i] = (float*)ctx_alloc(ctx, s->bytes[i], nullptr);
      if (!s->arr[i]) {
        hg_destroy_scene(s);
        hg_set_error("hg_create_scene: allocation failed");
        return HG_ERR_OOM;
      }
      if (d->n) {
        cudaError_t e = cudaMemcpy(s->arr[i], src[i], s->bytes[i], cudaMemcpyDefault);
        if (e != cudaSuccess) {
          hg_destroy_scene(s);
          return hg_cuda_status(e, "hg_create_scene copy");
        }
      }
    } else {
      s->arr[i] = (float*)const_cast<void*>(src[i]);
    }
  }
  if (d->order == HG_ORDER_SPATIAL && d->n > 0) {
    // store the gaussians in spatial order: permutation, then each array
    // gathered into a new buffer that replaces the copy
    s->perm = (int32_t*)ctx_alloc(ctx, sizeof(int32_t) * (size_t)d->n, nullptr);
    if (!s->perm) {
      hg_destroy_scene(s);
      hg_set_error("hg_create_scene: allocation failed");
      return HG_ERR_OOM;
    }
    hg_status r = spatial_order(ctx, s->arr[0], d->n, s->perm, nullptr);
    for (int i = 0; i < 5 && r == HG_OK; ++i) {
      void* dst = ctx_alloc(ctx, s->bytes[i], nullptr);
      if (!dst) {
        r = HG_ERR_OOM;
        hg_set_error("hg_create_scene: allocation failed");
        break;
      }
      cudaError_t e = gather_rows(s->arr[i], dst, s->perm, d->n, s->bytes[i] / (size_t)d->n, nullptr);
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      if (e != cudaSuccess) {
        ctx_free(ctx, dst, s->bytes[i], nullptr);
        r = hg_cuda_status(e, "hg_create_scene reorder");
        break;
      }
      ctx_free(ctx, s->arr[i], s->bytes[i], nullptr);
      s->arr[i] = (float*)dst;
    }
    if (r != HG_OK) {
      hg_destroy_scene(s);
      return r;
    }
  }
  *out = s;
  return HG_OK;
}

extern "C" void hg_destroy_scene(hg_scene* s) {
  if (!s) return;
  if (s->owned)
    for (int i = 0; i < 5; ++i) ctx_free(s->ctx, s->arr[i], s->bytes[i], nullptr);
  if (s->sh_scale) ctx_free(s->ctx, s->sh_scale, sizeof(float) * 2 * SH_CODEC_CH, nullptr);
  if (s->perm) ctx_free(s->ctx, s->perm, sizeof(int32_t) * (size_t)s->n, nullptr);
  delete s;
}

extern "C" hg_status hg_scene_order(const hg_scene* s, int32_t* perm_host) {
  if (!s || (s->n > 0 && !perm_host)) {
    hg_set_error("hg_scene_order: bad arguments");
    return HG_ERR_INVALID_ARG;
  }
  if (!s->perm) {
    for (int64_t i = 0; i < s->n; ++i) perm_host[i] = (int32_t)i;
    return HG_OK;
  }
  cudaSetDevice(s->ctx->device);
  const cudaError_t e = cudaMemcpy(perm_host, s->perm, sizeof(int32_t) * (size_t)s->n, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? HG_OK : hg_cuda_status(e, "hg_scene_order");
}

extern "C" hg_status hg_scene_sh_codec(const hg_scene* s, float* scales_host, uint32_t* codes_host) {
  if (!s || !scales_host || s->sh_storage != HG_SH_CODEC32 || !s->sh_scale) {
    hg_set_error("hg_scene_sh_codec: not a packed-SH scene");
    return HG_ERR_INVALID_ARG;
  }
  cudaSetDevice(s->ctx->device);
  cudaError_t e = cudaMemcpy(scales_host, s->sh_scale, sizeof(float) * SH_CODEC_CH, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && codes_host && s->n > 0)
    e = cudaMemcpy(codes_host, s->arr[4], s->bytes[4], cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? HG_OK : hg_cuda_status(e, "hg_scene_sh_codec");
}

extern "C" int64_t hg_scene_size(const hg_scene* s) { return s ? s->n : 0; }

// ---------------------------------------------------------------- states
hg_status state_create(hg_ctx* ctx, hg_state** out) {
  hg_state* s = new hg_state();
  s->ctx = ctx;
  cudaError_t e = cudaMallocHost((void**)&s->fc_host, sizeof(FrameCounters));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s->views_host, sizeof(ViewDesc) * MAX_VIEWS);
  if (e != cudaSuccess) {
    delete s;
    return hg_cuda_status(e, "pinned host allocation");
  }
  memset(s->fc_host, 0, sizeof(FrameCounters));
  for (int i = 0; i < N_EVENTS; ++i) cudaEventCreate(&s->ev[i]);
  cudaEventCreateWithFlags(&s->frame_done, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&s->views_uploaded, cudaEventDisableTiming);
  {
    SortStreams& ss = s->sort_streams;
    bool ok = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < 3; ++i) {
      ok = ok && cudaStreamCreateWithFlags(&ss.aux[i], cudaStreamNonBlocking) == cudaSuccess;
      ok = ok && cudaEventCreateWithFlags(&ss.join[i], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
      hg_state_free(s);
      return hg_cuda_status(cudaGetLastError(), "sort streams");
    }
    s->has_sort_streams = true;
  }
  *out = s;
  return HG_OK;
}

extern "C" void hg_state_free(hg_state* s) {
  if (!s) return;
  cudaSetDevice(s->ctx->device);
  cudaDeviceSynchronize();
  for (int i = 0; i < BUF_COUNT; ++i) ctx_free(s->ctx, s->bufs[i].p, s->bufs[i].bytes, nullptr);
  for (int i = 0; i < N_EVENTS; ++i) cudaEventDestroy(s->ev[i]);
  if (s->frame_done) cudaEventDestroy(s->frame_done);
  if (s->views_uploaded) cudaEventDestroy(s->views_uploaded);
  {
    SortStreams& ss = s->sort_streams;
    if (ss.fork) cudaEventDestroy(ss.fork);
    for (int i = 0; i < 3; ++i) {
      if (ss.aux[i]) cudaStreamDestroy(ss.aux[i]);
      if (ss.join[i]) cudaEventDestroy(ss.join[i]);
    }
  }
  cudaFreeHost(s->fc_host);
  cudaFreeHost(s->views_host);
  delete s;
}

cudaError_t state_wait(hg_state* s) {
  if (s->frame_in_graph && s->frame_done) return cudaEventSynchronize(s->frame_done);
  return cudaStreamSynchronize(s->last_stream);
}

extern "C" hg_status hg_state_sync(hg_state* s) {
  if (!s) return HG_ERR_INVALID_ARG;
  cudaSetDevice(s->ctx->device);
  HG_TRY(state_wait(s), "hg_state_sync");
  return (hg_status)s->fc_host->status;
}

// ---------------------------------------------------------------- frames
static bool valid_opts(const hg_render_opts* o, std::string& why) {
  if (o->path != HG_PATH_HIGS && o->path != HG_PATH_PLAIN) return why = "path", false;
  const bool shape_ok = (o->macro_w == 8 && o->macro_h == 4) || (o->macro_w == 4 && o->macro_h == 4) ||
                        (o->macro_w == 8 && o->macro_h == 8);
  if (!shape_ok) return why = "macro shape must be 8x4, 4x4 or 8x8", false;
  if (o->batch_cap < 32 || o->batch_cap > 2048 || (o->batch_cap & 31)) return why = "batch_cap", false;
  if (o->bin_test != HG_BIN_RECT && o->bin_test != HG_BIN_ELLIPSE) return why = "bin_test", false;
  if ((o->flags & HG_FLAG_FP16) && o->save_for_backward)
    return why = "HG_FLAG_FP16 does not save for the backward (float32 only)", false;
  if ((o->flags & HG_FLAG_INDEPENDENT) && o->save_for_backward)
    return why = "save_for_backward needs the chained schedule (not HG_FLAG_INDEPENDENT)", false;
  return true;
}

hg_status build_views(hg_state* s, const hg_camera* cams, int V, const hg_render_opts* o, FrameGeom& g) {
  g = FrameGeom();
  g.V = V;
  long long pix = 0;
  int seg = 0, tiles = 0, max_nm = 0;
  for (int v = 0; v < V; ++v) {
    const hg_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width > 16384 || c.height > 16384 || !(c.fx > 0) || !(c.fy > 0)) {
      hg_set_error("camera " + std::to_string(v) + ": bad image size or focal length");
      return HG_ERR_INVALID_ARG;
    }
    ViewDesc& d = s->views_host[v];
    memset(&d, 0, sizeof(d));
    for (int k = 0; k < 12; ++k) d.vm[k] = c.viewmat[k];
    d.fx = c.fx;
    d.fy = c.fy;
    d.cx = c.cx;
    d.cy = c.cy;
    // camera centre -R^T t
    for (int k = 0; k < 3; ++k)
      d.campos[k] = -(c.viewmat[0 * 4 + k] * c.viewmat[3] + c.viewmat[1 * 4 + k] * c.viewmat[7] +
                      c.viewmat[2 * 4 + k] * c.viewmat[11]);
    d.tan_x = 0.5f * (float)c.width / c.fx;
    d.tan_y = 0.5f * (float)c.height / c.fy;
    d.W = c.width;
    d.H = c.height;
    d.tiles_x = (c.width + TILE - 1) / TILE;
    d.tiles_y = (c.height + TILE - 1) / TILE;
    d.mgx = (d.tiles_x + o->macro_w - 1) / o->macro_w;
    d.mgy = (d.tiles_y + o->macro_h - 1) / o->macro_h;
    d.seg_base = seg;
    d.tile_base = tiles;
    d.pix_base = pix;
    seg += d.mgx * d.mgy;
    tiles += d.tiles_x * d.tiles_y;
    pix += (long long)c.width * c.height;
    max_nm = std::max(max_nm, d.mgx * d.mgy);
  }
  g.S = seg;
  g.total_tiles = tiles;
  g.pixels = pix;
  g.max_nm = max_nm;
  return HG_OK;
}

static void sizes_from_counters(hg_state* s, const FrameGeom& g, const hg_render_opts* o) {
  const FrameCounters& f = *s->fc_host;
  const size_t need_pairs = (size_t)f.n_pairs;
  if (o->path == HG_PATH_HIGS) {
    s->cap_pairs = std::max(s->cap_pairs, need_pairs + need_pairs / 8 + 1024);
    s->cap_batches = std::max(s->cap_batches, (size_t)f.n_batches + f.n_batches / 8 + 64);
    s->cap_tiles = std::max(s->cap_tiles, (size_t)f.n_big_tiles + f.n_big_tiles / 8 + 16);
    s->cap_big_segs = std::max(s->cap_big_segs, (size_t)f.n_big_segs + 16);
  } else {
    s->cap_plain_pairs = std::max(s->cap_plain_pairs, need_pairs + need_pairs / 8 + 1024);
    s->cap_plain_tiles = s->cap_plain_pairs / OS_TILE + 16;
  }
  (void)g;
}

hg_status ensure_workspace(hg_state* s, long long n, const FrameGeom& g, const hg_render_opts* o,
                           cudaStream_t st) {
  const int V = g.V;
  hg_status r;
  // capacities (first frame: estimates; later frames: measured + slack)
  if (s->cap_pairs == 0) s->cap_pairs = (size_t)std::max<long long>(1 << 20, 2 * n * V);
  if (s->cap_batches == 0) s->cap_batches = s->cap_pairs / o->batch_cap + g.S + 64;
  s->cap_batches = std::max(s->cap_batches, (size_t)g.S + 64);
  if (s->cap_tiles == 0) s->cap_tiles = s->cap_pairs / OS_TILE + 16;
  if (s->cap_big_segs == 0) s->cap_big_segs = std::min<size_t>((size_t)g.S, s->cap_pairs / TIER3_MAX + 16);
  s->cap_big_segs = std::max<size_t>(s->cap_big_segs, 16);
  if (s->cap_plain_pairs == 0) s->cap_plain_pairs = (size_t)std::max<long long>(1 << 20, 8 * n * V);
  if (s->cap_plain_tiles == 0) s->cap_plain_tiles = s->cap_plain_pairs / OS_TILE + 16;

  const size_t vis_words = (size_t)((n + 31) / 32);
  const int M = o->macro_w * o->macro_h;
  const int n_pb = (int)((n + BP - 1) / BP);
#define ENS(id, bytes) \
  if ((r = ws_ensure(s, id, (bytes), st)) != HG_OK) return r;
  ENS(B_FC, sizeof(FrameCounters));
  ENS(B_VIEWS, sizeof(ViewDesc) * MAX_VIEWS);
  ENS(B_BIN, sizeof(uint4) * n * V);
  ENS(B_DKEY, sizeof(uint32_t) * n * V);
  ENS(B_REC, sizeof(float4) * REC_F4 * n * V);
  ENS(B_VIS, sizeof(uint32_t) * vis_words * V);
  if (o->flags & HG_FLAG_KEEP_SPLATS) ENS(B_SPLATS, sizeof(hg_splat) * n * V);
  if (o->path == HG_PATH_PLAIN) {
    ENS(P_COUNTS, sizeof(uint32_t) * n * V);
    ENS(P_OFFS, sizeof(uint32_t) * (n * V + 1));
    const size_t nblk = (size_t)((n * V + 4095) / 4096);
    ENS(P_SCAN, sizeof(uint32_t) * ((nblk + 3) & ~size_t(3)) + sizeof(uint4) * s->cap_plain_tiles);
    ENS(P_KEYS, sizeof(unsigned long long) * s->cap_plain_pairs);
    ENS(P_KEYS2, sizeof(unsigned long long) * s->cap_plain_pairs);
    ENS(P_VALS, sizeof(uint32_t) * s->cap_plain_pairs);
    ENS(P_VALS2, sizeof(uint32_t) * s->cap_plain_pairs);
    ENS(P_RANGES, sizeof(uint2) * g.total_tiles);
    ENS(P_LOOKBACK, sizeof(uint32_t) * 8 * 256 * s->cap_plain_tiles);  // one region per digit pass
    ENS(P_DHIST, sizeof(uint32_t) * 8 * 256);
  } else {
    ENS(B_HIST, sizeof(uint16_t) * (size_t)n_pb * g.S + 16);
    ENS(B_COLPRE, sizeof(uint32_t) * (size_t)n_pb * g.S + 16);
    ENS(B_SEGTOT, sizeof(uint32_t) * g.S);
    ENS(B_SEGOFF, sizeof(uint32_t) * (g.S + 1));
    ENS(B_FIRSTB, sizeof(uint32_t) * (g.S + 1));
    ENS(B_TIERLIST, sizeof(uint32_t) * N_TIERS * (size_t)g.S);
    ENS(B_BIGTILES, sizeof(uint4) * s->cap_tiles);
    ENS(B_BIGSEGS, sizeof(uint32_t) * s->cap_big_segs);
    ENS(B_BIGTF, sizeof(uint32_t) * s->cap_big_segs);
    ENS(B_KEYS, sizeof(uint32_t) * s->cap_pairs);
    ENS(B_VALS, sizeof(uint32_t) * s->cap_pairs);
    ENS(B_KEYS2, sizeof(uint32_t) * s->cap_pairs);
    ENS(B_VALS2, sizeof(uint32_t) * s->cap_pairs);
    ENS(B_BATCHES, sizeof(uint4) * s->cap_batches);
    ENS(B_BORDER, sizeof(uint32_t) * s->cap_batches);
    ENS(B_RANKC, sizeof(uint32_t) * (MAX_RANKS + 1));
    ENS(B_PARTIAL, sizeof(float4) * TILE_PX * M * s->cap_batches);
    ENS(B_ACTIVE, sizeof(unsigned long long) * s->cap_batches);
    ENS(B_CHAIN, sizeof(uint32_t) * g.S);
    ENS(B_MODE, sizeof(uint32_t) * s->cap_batches);
    ENS(B_TSTATE, sizeof(float4) * TILE_PX * (size_t)g.total_tiles);
    ENS(B_TRANK, sizeof(uint32_t) * g.total_tiles);
    ENS(B_SEGHIST, sizeof(uint32_t) * 8 * 256 * s->cap_big_segs);
    ENS(B_LOOKBACK, sizeof(uint32_t) * 8 * 256 * s->cap_tiles);  // one region per digit pass
    if (o->save_for_backward) {
      ENS(B_EXIT, sizeof(float4) * TILE_PX * M * s->cap_batches);
      ENS(B_EXITLAST, sizeof(uint16_t) * TILE_PX * M * s->cap_batches);
    }
  }
#undef ENS
  return HG_OK;
}

hg_status enqueue_frame(hg_state* s, const FrameInputs& in, const hg_render_opts* o, const FrameGeom& g,
                               float* out_rgb, float* out_T, cudaStream_t st) {
  const long long n = in.n;
  const int V = g.V;
  const bool timing = (o->flags & HG_FLAG_TIMING) != 0;
  hg_status r = ensure_workspace(s, n, g, o, st);
  if (r != HG_OK) return r;
  const size_t vis_words = (size_t)((n + 31) / 32);
  const int M = o->macro_w * o->macro_h;
  const int n_pb = (int)((n + BP - 1) / BP);
  FrameCounters* fc = (FrameCounters*)s->bufs[B_FC].p;
  ViewDesc* views = (ViewDesc*)s->bufs[B_VIEWS].p;
  if (timing) HG_TRY(record_stage(s->ev[0], st), "stage event 0");
  HG_TRY(cudaMemsetAsync(fc, 0, sizeof(FrameCounters), st), "memset counters");
  HG_TRY(cudaMemcpyAsync(views, s->views_host, sizeof(ViewDesc) * V, cudaMemcpyHostToDevice, st), "upload views");
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HG_TRY(cudaStreamIsCapturing(st, &cs), "capture status");
    if (cs == cudaStreamCaptureStatusNone) HG_TRY(cudaEventRecord(s->views_uploaded, st), "views uploaded");
  }
  ProjectArgs pj{};
  pj.n = n;
  pj.views = views;
  pj.n_views = V;
  pj.vis_words = (long long)vis_words;
  pj.bin = (uint4*)s->bufs[B_BIN].p;
  pj.dkeys = (uint32_t*)s->bufs[B_DKEY].p;
  pj.rec = (float4*)s->bufs[B_REC].p;
  pj.vis = (uint32_t*)s->bufs[B_VIS].p;
  pj.bin_mode = o->path == HG_PATH_PLAIN ? BIN_CLASSIC
                                         : (o->bin_test == HG_BIN_ELLIPSE ? BIN_CELLS_ELLIPSE : BIN_CELLS_RECT);
  pj.macro_w = o->macro_w;
  pj.macro_h = o->macro_h;
  pj.wait_polls = s->ctx->wait_polls;
  pj.fc = fc;
  if (in.splats) {
    HG_TRY(launch_splats_to_records(in.splats, n, V, (long long)vis_words, pj, st), "splats to records");
  } else {
    pj.means = in.scene->arr[0];
    pj.log_scales = in.scene->arr[1];
    pj.quats = in.scene->arr[2];
    pj.opacity_logits = in.scene->arr[3];
    pj.sh = in.scene->arr[4];
    pj.sh_storage = in.scene->sh_storage;
    pj.sh_scale2 = in.scene->sh_scale ? in.scene->sh_scale + SH_CODEC_CH : nullptr;
    pj.splats = (o->flags & HG_FLAG_KEEP_SPLATS) ? (hg_splat*)s->bufs[B_SPLATS].p : nullptr;
    HG_TRY(launch_project(pj, in.scene->deg, st), "project");
  }
  if (timing) HG_TRY(record_stage(s->ev[1], st), "stage event 1");

  if (o->path == HG_PATH_PLAIN) {
    PlainArgs pa{};
    pa.bin = (const uint4*)s->bufs[B_BIN].p;
    pa.rec = (const float4*)s->bufs[B_REC].p;
    pa.n = n;
    pa.vis = (const uint32_t*)s->bufs[B_VIS].p;
    pa.vis_words = vis_words;
    pa.views = views;
    pa.n_views = V;
    pa.total_tiles = g.total_tiles;
    pa.counts = (uint32_t*)s->bufs[P_COUNTS].p;
    pa.offsets = (uint32_t*)s->bufs[P_OFFS].p;
    pa.scan_tmp = (uint32_t*)s->bufs[P_SCAN].p;
    pa.keys = (unsigned long long*)s->bufs[P_KEYS].p;
    pa.vals = (uint32_t*)s->bufs[P_VALS].p;
    pa.keys_alt = (unsigned long long*)s->bufs[P_KEYS2].p;
    pa.vals_alt = (uint32_t*)s->bufs[P_VALS2].p;
    pa.ranges = (uint2*)s->bufs[P_RANGES].p;
    pa.lookback = (uint32_t*)s->bufs[P_LOOKBACK].p;
    pa.digit_hist = (uint32_t*)s->bufs[P_DHIST].p;
    pa.cap_pairs = (uint32_t)std::min<size_t>(s->cap_plain_pairs, 0xffffffffu);
    pa.cap_tiles = (uint32_t)s->cap_plain_tiles;
    pa.wait_polls = s->ctx->wait_polls;
    for (int k = 0; k < 3; ++k) pa.bg[k] = o->bg[k];
    pa.out_rgb = out_rgb;
    pa.out_T = out_T;
    pa.fc = fc;
    unsigned long long* sk = nullptr;
    uint32_t* sv = nullptr;
    HG_TRY(launch_plain(pa, st, &sk, &sv), "plain path");
    s->plain_keys = sk;
    s->plain_vals = sv;
    if (timing)
      for (int k = 2; k < 6; ++k) HG_TRY(record_stage(s->ev[k], st), "stage event");
  } else {
    PartitionArgs pa{};
    pa.bin = (const uint4*)s->bufs[B_BIN].p;
    pa.dkeys = (const uint32_t*)s->bufs[B_DKEY].p;
    pa.vis = (const uint32_t*)s->bufs[B_VIS].p;
    pa.n = n;
    pa.vis_words = (long long)vis_words;
    pa.views = views;
    pa.n_views = V;
    pa.n_seg = g.S;
    pa.n_pb = n_pb;
    pa.macro_w = o->macro_w;
    pa.macro_h = o->macro_h;
    pa.max_nm = g.max_nm;
    pa.hist = (uint16_t*)s->bufs[B_HIST].p;
    pa.colpre = (uint32_t*)s->bufs[B_COLPRE].p;
    pa.seg_tot = (uint32_t*)s->bufs[B_SEGTOT].p;
    pa.seg_off = (uint32_t*)s->bufs[B_SEGOFF].p;
    pa.first_batch = (uint32_t*)s->bufs[B_FIRSTB].p;
    pa.tier_list = (uint32_t*)s->bufs[B_TIERLIST].p;
    pa.big_tiles = (uint4*)s->bufs[B_BIGTILES].p;
    pa.big_segs = (uint32_t*)s->bufs[B_BIGSEGS].p;
    pa.big_tile_first = (uint32_t*)s->bufs[B_BIGTF].p;
    pa.keys = (uint32_t*)s->bufs[B_KEYS].p;
    pa.vals = (uint32_t*)s->bufs[B_VALS].p;
    pa.batches = (uint4*)s->bufs[B_BATCHES].p;
    pa.batch_order = (uint32_t*)s->bufs[B_BORDER].p;
    pa.rank_count = (uint32_t*)s->bufs[B_RANKC].p;
    pa.batch_cap = o->batch_cap;
    pa.cap_pairs = (uint32_t)std::min<size_t>(s->cap_pairs, 0xffffffffu);
    pa.cap_batches = (uint32_t)s->cap_batches;
    pa.cap_tiles = (uint32_t)s->cap_tiles;
    pa.cap_big_segs = (uint32_t)s->cap_big_segs;
    pa.seg_hist = (uint32_t*)s->bufs[B_SEGHIST].p;
    pa.fc = fc;
    if (n > 0) HG_TRY(launch_partition(pa, st), "partition");
    if (timing) HG_TRY(record_stage(s->ev[2], st), "stage event 2");

    SortArgs sa{};
    sa.keys = pa.keys;
    sa.vals = pa.vals;
    sa.keys_alt = (uint32_t*)s->bufs[B_KEYS2].p;
    sa.vals_alt = (uint32_t*)s->bufs[B_VALS2].p;
    sa.seg_off = pa.seg_off;
    sa.tier_list = pa.tier_list;
    sa.n_seg = g.S;
    sa.big_tiles = pa.big_tiles;
    sa.big_segs = pa.big_segs;
    sa.big_tile_first = pa.big_tile_first;
    sa.seg_hist = (uint32_t*)s->bufs[B_SEGHIST].p;
    sa.lookback = (uint32_t*)s->bufs[B_LOOKBACK].p;
    sa.cap_tiles = pa.cap_tiles;
    sa.cap_big_segs = pa.cap_big_segs;
    sa.wait_polls = s->ctx->wait_polls;
    // the last completed frame of this state had no segment above the
    // shared-memory tiers: a small onesweep grid (still correct if this one has)
    sa.os_ctas = s->fc_host->n_big_tiles == 0 ? 8 : 0;
    sa.fc = fc;
    if (n > 0) HG_TRY(launch_sort(sa, st, s->has_sort_streams ? &s->sort_streams : nullptr), "sort");
    if (timing) HG_TRY(record_stage(s->ev[3], st), "stage event 3");

    HG_TRY(cudaMemsetAsync(s->bufs[B_CHAIN].p, 0, sizeof(uint32_t) * g.S, st), "memset chain");
    HG_TRY(cudaMemsetAsync(s->bufs[B_TRANK].p, 0, sizeof(uint32_t) * g.total_tiles, st), "memset tile rank");
    RasterArgs ra{};
    ra.rec = (const float4*)s->bufs[B_REC].p;
    ra.n = n;
    ra.views = views;
    ra.n_views = V;
    ra.n_seg = g.S;
    ra.keys = pa.keys;
    ra.vals = pa.vals;
    ra.batches = pa.batches;
    ra.batch_order = pa.batch_order;
    ra.cap_batches = pa.cap_batches;
    ra.batch_cap = o->batch_cap;
    ra.macro_w = o->macro_w;
    ra.macro_h = o->macro_h;
    ra.partial = (float4*)s->bufs[B_PARTIAL].p;
    ra.active = (unsigned long long*)s->bufs[B_ACTIVE].p;
    ra.chain = (uint32_t*)s->bufs[B_CHAIN].p;
    ra.mode = (uint32_t*)s->bufs[B_MODE].p;
    ra.tile_state = (float4*)s->bufs[B_TSTATE].p;
    ra.tile_rank = (uint32_t*)s->bufs[B_TRANK].p;
    ra.exitrec = o->save_for_backward ? (float4*)s->bufs[B_EXIT].p : nullptr;
    ra.exitlast = o->save_for_backward ? (uint16_t*)s->bufs[B_EXITLAST].p : nullptr;
    ra.persistent_ctas = 0;
    ra.independent = (o->flags & HG_FLAG_INDEPENDENT) ? 1 : 0;
    ra.fp16 = (o->flags & HG_FLAG_FP16) ? 1 : 0;
    ra.direct_out = o->save_for_backward ? 0 : 1;
    ra.first_batch = pa.first_batch;
    ra.out_rgb = out_rgb;
    ra.out_T = out_T;
    for (int c = 0; c < 3; ++c) ra.bg[c] = o->bg[c];
    ra.profile = (o->flags & HG_FLAG_PROFILE) ? 1 : 0;
    ra.wait_polls = s->ctx->wait_polls;
    ra.chain_polls = s->ctx->chain_polls;
    ra.fc = fc;
    if (n > 0) HG_TRY(launch_raster(ra, st), "raster");
    if (timing) HG_TRY(record_stage(s->ev[4], st), "stage event 4");

    MergeArgs ma{};
    ma.partial = ra.partial;
    ma.active = ra.active;
    ma.mode = ra.mode;
    ma.tile_state = ra.tile_state;
    ma.tile_rank = ra.tile_rank;
    ma.first_batch = pa.first_batch;
    ma.chain = ra.chain;
    ma.batches = pa.batches;
    ma.vals = pa.vals;
    ma.rec = ra.rec;
    ma.n = n;
    ma.views = views;
    ma.n_views = V;
    ma.total_tiles = g.total_tiles;
    ma.macro_w = o->macro_w;
    ma.macro_h = o->macro_h;
    for (int k = 0; k < 3; ++k) ma.bg[k] = o->bg[k];
    ma.out_rgb = out_rgb;
    ma.out_T = out_T;
    ma.fc = fc;
    if (n == 0) {
      // empty scene: the first batch table is all zero, merge writes background
      HG_TRY(cudaMemsetAsync(pa.first_batch, 0, sizeof(uint32_t) * (g.S + 1), st), "memset first_batch");
    }
    HG_TRY(launch_merge(ma, st), "merge");
    if (timing) HG_TRY(record_stage(s->ev[5], st), "stage event 5");
  }
  HG_TRY(cudaMemcpyAsync(s->fc_host, fc, sizeof(FrameCounters), cudaMemcpyDeviceToHost, st), "read counters");
  return HG_OK;
}

hg_status run_frame(hg_state* s, const FrameInputs& in, const hg_render_opts* o, const hg_camera* cams, int V,
                    float* out_rgb, float* out_T, cudaStream_t st) {
  // the previous frame's view table must have been uploaded before it is
  // overwritten (an asynchronous frame may still wait in its stream)
  HG_TRY(cudaEventSynchronize(s->views_uploaded), "view table in use");
  FrameGeom g;
  hg_status r = build_views(s, cams, V, o, g);
  if (r != HG_OK) return r;
  s->geom = g;
  s->opts = *o;
  s->n = in.n;
  s->scene = in.scene;
  s->last_stream = st;
  s->has_frame = true;
  s->frame_in_graph = false;
  s->has_grad2d = false;
  ++s->frame_id;
  const bool async = (o->flags & HG_FLAG_ASYNC) != 0;
  for (int attempt = 0; attempt < 4; ++attempt) {
    r = enqueue_frame(s, in, o, g, out_rgb, out_T, st);
    if (r != HG_OK) return r;
    if (async) return HG_OK;
    HG_TRY(cudaStreamSynchronize(st), "frame");
    const int status = s->fc_host->status;
    if (status == HG_ERR_CAPACITY) {
      sizes_from_counters(s, g, o);
      continue;
    }
    if (status != HG_OK) {
      hg_set_error(std::string("device status: ") + hg_status_str((hg_status)status));
      return (hg_status)status;
    }
    return HG_OK;
  }
  hg_set_error("workspace did not converge");
  return HG_ERR_CAPACITY;
}

static hg_status resolve_state(hg_ctx* ctx, hg_state** state, hg_state** out) {
  if (state) {
    if (!*state) {
      hg_status r = state_create(ctx, state);
      if (r != HG_OK) return r;
    }
    *out = *state;
    return HG_OK;
  }
  if (!ctx->internal) {
    hg_status r = state_create(ctx, &ctx->internal);
    if (r != HG_OK) return r;
  }
  *out = ctx->internal;
  return HG_OK;
}

static hg_status check_render_args(const hg_camera* cams, int n_views, const hg_render_opts* opts, float* out_rgb) {
  std::string why;
  if (!cams || n_views <= 0 || n_views > MAX_VIEWS || !opts || !out_rgb) {
    hg_set_error("render: null argument or view count outside 1..64");
    return HG_ERR_INVALID_ARG;
  }
  if (!valid_opts(opts, why)) {
    hg_set_error("render options: " + why);
    return HG_ERR_INVALID_ARG;
  }
  return HG_OK;
}

extern "C" hg_status hg_render(hg_scene* scene, const hg_camera* cams, int n_views, const hg_render_opts* opts,
                               float* out_rgb, float* out_T, hg_state** state, void* stream) {
  if (!scene) return HG_ERR_INVALID_ARG;
  hg_status r = check_render_args(cams, n_views, opts, out_rgb);
  if (r != HG_OK) return r;
  cudaSetDevice(scene->ctx->device);
  hg_state* s;
  if ((r = resolve_state(scene->ctx, state, &s)) != HG_OK) return r;
  FrameInputs in{scene, nullptr, scene->n};
  return run_frame(s, in, opts, cams, n_views, out_rgb, out_T, (cudaStream_t)stream);
}

extern "C" hg_status hg_render_splats(hg_ctx* ctx, const hg_splat* d_splats, int64_t n, const hg_camera* cams,
                                      int n_views, const hg_render_opts* opts, float* out_rgb, float* out_T,
                                      hg_state** state, void* stream) {
  if (!ctx || n < 0 || (n > 0 && !d_splats)) return HG_ERR_INVALID_ARG;
  if (opts && opts->save_for_backward) {
    hg_set_error("hg_render_splats: no scene parameters to differentiate");
    return HG_ERR_INVALID_ARG;
  }
  hg_status r = check_render_args(cams, n_views, opts, out_rgb);
  if (r != HG_OK) return r;
  cudaSetDevice(ctx->device);
  hg_state* s;
  if ((r = resolve_state(ctx, state, &s)) != HG_OK) return r;
  FrameInputs in{nullptr, d_splats, n};
  return run_frame(s, in, opts, cams, n_views, out_rgb, out_T, (cudaStream_t)stream);
}

extern "C" hg_status hg_render_stats(hg_state* s, hg_frame_stats* out) {
  if (!s || !out || !s->has_frame) return HG_ERR_INVALID_ARG;
  cudaSetDevice(s->ctx->device);
  HG_TRY(state_wait(s), "stats");
  const FrameCounters& f = *s->fc_host;
  memset(out, 0, sizeof(*out));
  out->n_views = s->geom.V;
  out->n_gaussians = s->n;
  out->n_visible = f.n_visible;
  out->n_pairs = f.n_pairs;
  out->n_segments = s->geom.S;
  out->n_batches = f.n_batches;
  out->max_segment = f.max_seg;
  for (int t = 0; t < N_TIERS; ++t) out->seg_by_tier[t] = f.tier_count[t];
  out->n_sort_tiles = f.n_big_tiles;
  out->n_replays = (int64_t)f.replays;
  out->raster_evals = (int64_t)f.raster_evals;
  out->status = f.status;
  out->sort_resorts = (int32_t)f.sort_resorts;
  for (int k = 0; k < 6; ++k) out->raster_cycles[k] = (int64_t)f.raster_cycles[k];
  out->pixel_support_evals = (int64_t)f.pixel_support_evals;
  out->pixel_contrib_evals = (int64_t)f.pixel_contrib_evals;
  out->pixel_live_evals = (int64_t)f.pixel_live_evals;
  if (s->opts.flags & HG_FLAG_TIMING) {
    float ms[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 5; ++k) cudaEventElapsedTime(&ms[k], s->ev[k], s->ev[k + 1]);
    out->ms_project = ms[0];
    out->ms_partition = ms[1];
    out->ms_sort = ms[2];
    out->ms_raster = ms[3];
    out->ms_merge = ms[4];
    cudaEventElapsedTime(&out->ms_total, s->ev[0], s->ev[5]);
  }
  return HG_OK;
}

extern "C" hg_status hg_state_read(hg_state* s, int which, void* dst, size_t dst_bytes, size_t* needed) {
  if (!s || !s->has_frame) return HG_ERR_INVALID_ARG;
  cudaSetDevice(s->ctx->device);
  HG_TRY(cudaStreamSynchronize(s->last_stream), "state read");
  const FrameCounters& f = *s->fc_host;
  const FrameGeom& g = s->geom;
  const bool higs = s->opts.path == HG_PATH_HIGS;
  size_t bytes = 0;
  const void* src = nullptr;
  std::vector<uint32_t> tmp;
  switch (which) {
    case HG_BUF_SEG_OFF:
      if (!higs) return HG_ERR_UNSUPPORTED;
      bytes = sizeof(uint32_t) * (g.S + 1);
      src = s->bufs[B_SEGOFF].p;
      break;
    case HG_BUF_PAIR_KEYS:
    case HG_BUF_PAIR_IDS:
      if (!higs) return HG_ERR_UNSUPPORTED;
      bytes = sizeof(uint32_t) * f.n_pairs;
      src = s->bufs[which == HG_BUF_PAIR_KEYS ? B_KEYS : B_VALS].p;
      break;
    case HG_BUF_BATCHES: {
      if (!higs) return HG_ERR_UNSUPPORTED;
      bytes = sizeof(uint32_t) * 3 * f.n_batches;
      if (needed) *needed = bytes;
      if (!dst) return HG_OK;
      if (dst_bytes < bytes) return HG_ERR_INVALID_ARG;
      std::vector<uint4> b(f.n_batches);
      if (f.n_batches)
        HG_TRY(cudaMemcpy(b.data(), s->bufs[B_BATCHES].p, sizeof(uint4) * f.n_batches, cudaMemcpyDeviceToHost),
               "read batches");
      uint32_t* o = (uint32_t*)dst;
      for (size_t i = 0; i < b.size(); ++i) {
        o[3 * i + 0] = b[i].x;
        o[3 * i + 1] = b[i].y;
        o[3 * i + 2] = b[i].z;
      }
      return HG_OK;
    }
    case HG_BUF_SPLATS:
      if (!(s->opts.flags & HG_FLAG_KEEP_SPLATS)) return HG_ERR_UNSUPPORTED;
      bytes = sizeof(hg_splat) * s->n * g.V;
      src = s->bufs[B_SPLATS].p;
      break;
    case HG_BUF_PLAIN_KEYS:
    case HG_BUF_PLAIN_IDS:
      if (higs) return HG_ERR_UNSUPPORTED;
      bytes = (which == HG_BUF_PLAIN_KEYS ? sizeof(unsigned long long) : sizeof(uint32_t)) * f.n_pairs;
      src = which == HG_BUF_PLAIN_KEYS ? (const void*)s->plain_keys : (const void*)s->plain_vals;
      break;
    case HG_BUF_TILE_RANGES:
      if (higs) return HG_ERR_UNSUPPORTED;
      bytes = sizeof(uint32_t) * 2 * (size_t)g.total_tiles;
      src = s->bufs[P_RANGES].p;
      break;
    case HG_BUF_RECORDS:
      bytes = sizeof(float4) * REC_F4 * (size_t)s->n * g.V;
      src = s->bufs[B_REC].p;
      break;
    case HG_BUF_VISIBILITY:
      bytes = sizeof(uint32_t) * (size_t)((s->n + 31) / 32) * g.V;
      src = s->bufs[B_VIS].p;
      break;
    case HG_BUF_GRAD2D:
      if (!s->has_grad2d) return HG_ERR_UNSUPPORTED;
      bytes = sizeof(float) * 9 * (size_t)s->n * g.V;
      src = s->bufs[G_DMEANS2].p;
      break;
    case HG_BUF_VIEW_SEG_BASE: {
      bytes = sizeof(uint32_t) * (g.V + 1);
      if (needed) *needed = bytes;
      if (!dst) return HG_OK;
      if (dst_bytes < bytes) return HG_ERR_INVALID_ARG;
      uint32_t* o = (uint32_t*)dst;
      for (int v = 0; v < g.V; ++v) o[v] = (uint32_t)s->views_host[v].seg_base;
      o[g.V] = (uint32_t)g.S;
      return HG_OK;
    }
    default:
      return HG_ERR_INVALID_ARG;
  }
  if (needed) *needed = bytes;
  if (!dst) return HG_OK;
  if (dst_bytes < bytes) return HG_ERR_INVALID_ARG;
  if (bytes) HG_TRY(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost), "state read copy");
  return HG_OK;
}
