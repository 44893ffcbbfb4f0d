// Host-side objects behind the opaque C ABI handles.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "kernels.cuh"

struct hg_ctx {
  int device = 0;
  hg_allocator alloc{};
  bool has_alloc = false;
  int sms = 0;
  hg_state* internal = nullptr;  // workspace used when the caller passes no state
  void* loss_scratch = nullptr;   // hg_l2_loss block partials + counter (allocated on first use)
  // bounded device waits (hg_ctx_set_wait_limits): polls of an mbarrier or a
  // look-back word before the wait gives up, and of the batch chain before a
  // unit renders unchained
  uint32_t wait_polls = hg::SPIN_LIMIT;
  uint32_t chain_polls = hg::CHAIN_SPIN;
};

struct hg_scene {
  hg_ctx* ctx = nullptr;
  int64_t n = 0;
  int deg = 0;
  bool owned = true;
  int sh_storage = HG_SH_F32;  // element type of arr[4]
  float* sh_scale = nullptr;   // packed SH: device [2][48] (s, s / Q^2)
  float* arr[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // means, log_scales, quats, logits, sh
  size_t bytes[5] = {0, 0, 0, 0, 0};
  int32_t* perm = nullptr;  // HG_ORDER_SPATIAL: device [n], caller's index of each stored gaussian
};

namespace hg {

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

enum BufId {
  B_FC, B_VIEWS, B_BIN, B_DKEY, B_REC, B_VIS, B_SPLATS,
  B_HIST, B_COLPRE, B_SEGTOT, B_SEGOFF, B_FIRSTB, B_TIERLIST, B_BIGTILES, B_BIGSEGS, B_BIGTF,
  B_KEYS, B_VALS, B_KEYS2, B_VALS2, B_BATCHES, B_BORDER, B_RANKC,
  B_PARTIAL, B_ACTIVE, B_CHAIN, B_MODE, B_TSTATE, B_TRANK, B_STOPPOS, B_EXIT, B_EXITLAST, B_SEGHIST, B_LOOKBACK,
  P_COUNTS, P_OFFS, P_SCAN, P_KEYS, P_KEYS2, P_VALS, P_VALS2, P_RANGES, P_LOOKBACK, P_DHIST,
  G_DMEANS2, G_AUX,
  BUF_COUNT
};

struct FrameGeom {
  int V = 0;
  int S = 0;
  int total_tiles = 0;
  long long pixels = 0;
  int max_nm = 0;
};

struct FrameInputs {
  const hg_scene* scene;
  const hg_splat* splats;
  long long n;
};

constexpr int N_EVENTS = 8;

}  // namespace hg

struct hg_state {
  hg_ctx* ctx = nullptr;
  hg::Buf bufs[hg::BUF_COUNT];
  hg::FrameCounters* fc_host = nullptr;  // pinned
  hg::ViewDesc* views_host = nullptr;    // pinned, MAX_VIEWS entries
  // recorded after the view table's upload of the last frame enqueued
  // outside a capture: the next frame writes views_host only once that
  // upload has run (asynchronous frames queue behind one another)
  cudaEvent_t views_uploaded = nullptr;
  cudaEvent_t ev[hg::N_EVENTS] = {};
  hg::SortStreams sort_streams{};  // side streams of the sort tiers
  bool has_sort_streams = false;
  cudaStream_t last_stream = nullptr;
  bool has_frame = false;
  hg::FrameGeom geom;
  hg_render_opts opts{};
  long long n = 0;
  const hg_scene* scene = nullptr;
  size_t cap_pairs = 0, cap_batches = 0, cap_tiles = 0, cap_big_segs = 0;
  size_t cap_plain_pairs = 0, cap_plain_tiles = 0;
  // plain path: the buffers holding the sorted (64-bit key, record) pairs
  unsigned long long* plain_keys = nullptr;
  uint32_t* plain_vals = nullptr;
  // frames rendered into this state, and the frame whose saved batch colours
  // the backward already turned into colours behind the batches
  uint64_t frame_id = 0, bwd_suffix_done = 0;
  bool has_grad2d = false;  // a backward of the current frame wrote G_DMEANS2
  // set by hg_graph_launch: the replay's completion event (waiting on it
  // waits for this frame only, not for later work queued on the stream)
  cudaEvent_t frame_done = nullptr;
  bool frame_in_graph = false;
};

void hg_set_error(const std::string& s);
hg_status hg_cuda_status(cudaError_t e, const char* where);
void* ctx_alloc(hg_ctx* ctx, size_t bytes, cudaStream_t st);
void ctx_free(hg_ctx* ctx, void* p, size_t bytes, cudaStream_t st);

// hg_l2_loss: fixed grid and its scratch (block partials + finish counter)
constexpr int LOSS_BLOCKS = 304;
constexpr size_t LOSS_SCRATCH_BYTES = sizeof(double) * LOSS_BLOCKS + 256;
hg_status ws_ensure(hg_state* s, int id, size_t bytes, cudaStream_t st);
namespace hg {
// hg_spatial_order on a stream (synchronises it); gather of scene rows by a permutation
hg_status spatial_order(hg_ctx* ctx, const float* means, long long n, int32_t* perm, cudaStream_t st);
cudaError_t gather_rows(const void* src, void* dst, const int32_t* perm, long long n, size_t row_bytes,
                        cudaStream_t st);
}  // namespace hg
hg_status state_create(hg_ctx* ctx, hg_state** out);
hg_status build_views(hg_state* s, const hg_camera* cams, int V, const hg_render_opts* o, hg::FrameGeom& g);
// Grows the frame workspace of `s` to n gaussians and the views of `g`
// (capacities: the state's, or first-frame estimates); nothing is launched.
hg_status ensure_workspace(hg_state* s, long long n, const hg::FrameGeom& g, const hg_render_opts* o,
                           cudaStream_t st);
hg_status enqueue_frame(hg_state* s, const hg::FrameInputs& in, const hg_render_opts* o, const hg::FrameGeom& g,
                        float* out_rgb, float* out_T, cudaStream_t st);
// Waits for the last frame of `s` (its replay event after a graph launch,
// else its stream).
cudaError_t state_wait(hg_state* s);
hg_status run_frame(hg_state* s, const hg::FrameInputs& in, const hg_render_opts* o, const hg_camera* cams, int V,
                    float* out_rgb, float* out_T, cudaStream_t st);
