/*
 * higs.h - C ABI of the hierarchically tiled 3D Gaussian Splatting renderer
 * (HiGS, arxiv 2606.00352) for sm_103a GPUs.
 *
 * One call renders V views of a device-resident gaussian scene through the
 * paper's pipeline (Fig. 2; Sec. 3-4):
 *   projection + SH colour (Sec. 4.2) -> macro-tile count / two-level scan /
 *   fill (Sec. 3.2, 4.3) -> segmented depth sort (Sec. 3.3, 4.4) -> batch split
 *   (Sec. 3.1) -> macro-tile rasterisation (Alg. 1, Alg. 2, Sec. 4.5) ->
 *   ordered merge of the batch partials (Eq. 1, Sec. 3.4).
 * A plain one-block-per-8x8-tile path with a global 64-bit radix sort (the
 * baseline of Sec. 5) renders the same image for comparison.
 *
 * Conventions for every function below:
 *  - Pointers named d_* or documented as "device" are CUDA device pointers of
 *    the context's device; all other pointers are host pointers.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Render calls are stream-ordered: they enqueue work and,
 *    unless stated otherwise, return before the GPU finishes.
 *  - Every function returns an hg_status; nothing aborts.  Device-side
 *    failures (capacity exceeded, a bounded wait that gave up) are written to
 *    a device status word and reported by the call that synchronises
 *    (hg_render in synchronous mode, hg_state_sync, hg_graph_launch with a
 *    check).  hg_last_error() returns a thread-local message for the last
 *    failure of the calling thread.
 *  - Image outputs of a multi-view call are packed back to back: view v
 *    starts at pixel offset sum_{u<v} W_u H_u; RGB is [H][W][3] float32 per
 *    view and transmittance [H][W] float32.
 */
#ifndef HIGS_H
#define HIGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HG_OK = 0,
  HG_ERR_INVALID_ARG = -1,
  HG_ERR_OOM = -2,
  HG_ERR_CUDA = -3,
  HG_ERR_CAPACITY = -4,       /* a preallocated buffer was too small (frame invalid) */
  HG_ERR_DEVICE_TIMEOUT = -5, /* a bounded device wait gave up (frame invalid) */
  HG_ERR_BUSY = -6,
  HG_ERR_NOT_FOUND = -7,
  HG_ERR_CANCELLED = -8,
  HG_ERR_UNSUPPORTED = -9
} hg_status;

typedef struct hg_ctx hg_ctx;
typedef struct hg_scene hg_scene;
typedef struct hg_state hg_state;
typedef struct hg_graph hg_graph;
typedef struct hg_server hg_server;

/* Device memory provider.  alloc returns a device pointer of at least
 * `bytes` (aligned to 256 bytes) or NULL; free releases it.  When the
 * allocator passed to hg_ctx_create is NULL the library uses cudaMalloc /
 * cudaFree.  Workspace buffers are requested only when a frame needs more
 * than the buffers it already holds. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, size_t bytes, void* stream, void* user);
  void* user;
} hg_allocator;

/* Gaussian scene, structure of arrays, float32, device pointers:
 *   means [n][3], log_scales [n][3], quats [n][4] (w, x, y, z, any norm),
 *   opacity_logits [n], sh [n][(sh_degree+1)^2][3] (coefficient k = l*l+l+m).
 * borrow = 0: the library copies the arrays into memory it owns.
 * borrow = 1: the library keeps the pointers; the caller keeps them alive
 * and unchanged while the scene exists.
 * order: HG_ORDER_INPUT keeps the caller's gaussian order; HG_ORDER_SPATIAL
 * (borrow = 0 only) stores the gaussians in hg_spatial_order, so gaussians
 * that are near in space are near in memory and the projection's writes and
 * the partition's pair writes of one screen region are close together; the
 * image is that of the reordered set (hg_scene_order gives the order). */
typedef struct {
  int64_t n;
  int32_t sh_degree; /* 0..3 */
  int32_t borrow;
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logits;
  const void* sh;     /* [n][(deg+1)^2][3] of the element type sh_storage */
  int32_t sh_storage; /* HG_SH_F32, HG_SH_F16, HG_SH_BF16 or HG_SH_CODEC32 */
  int32_t order;      /* HG_ORDER_INPUT or HG_ORDER_SPATIAL */
} hg_scene_desc;

enum { HG_ORDER_INPUT = 0, HG_ORDER_SPATIAL = 1 };

/* Storage type of the SH coefficients (the projection computes in float32
 * either way; half storage halves the bytes the projection reads per
 * gaussian at degree 3, 236 -> 140).  HG_SH_CODEC32 is the 32-byte packed
 * representation of Sec. 4.2 (degree 3 only; YCoCg-R; the DC basis as a
 * float16 luma and 13-bit linear chroma, the others square-root gamma with
 * 6/4/4 bits; per-channel 99.5th-percentile scales): `sh` then points to float32 coefficients in
 * device memory, which hg_create_scene encodes (the scene always owns the
 * codes; 236 -> 76 bytes per gaussian).  Scenes with half or packed SH
 * render and serve; hg_render_backward and hg_adam_step need float32 SH. */
enum { HG_SH_F32 = 0, HG_SH_F16 = 1, HG_SH_BF16 = 2, HG_SH_CODEC32 = 3 };

/* The packed SH of a HG_SH_CODEC32 scene: scales_host[16][3] receives the
 * per-channel scales s (Y, Co, Cg per basis), codes_host (may be NULL)
 * n * 8 uint32 code words.  Synchronous.
 * Errors: HG_ERR_INVALID_ARG (not a packed-SH scene), HG_ERR_CUDA. */
hg_status hg_scene_sh_codec(const hg_scene* scene, float* scales_host, uint32_t* codes_host);

/* Spatial storage order of n gaussians (not part of the paper's method: a
 * memory layout for the front end's bandwidth, Sec. 4.2-4.3).  perm[i] is
 * the index of the i-th gaussian in ascending 30-bit Morton code of its
 * mean, ties by index.  The code quantises each axis a over the bounding
 * box [lo_a, hi_a] of the finite coordinates: q_a = min(1023,
 * floor((x_a - lo_a) * s_a)) with s_a = 1024 / (hi_a - lo_a) (1 when
 * hi_a = lo_a), every operation float32 round-to-nearest, a non-finite
 * coordinate counting as lo_a; bit 3 b + a of the code is bit b of q_a
 * (a = 0, 1, 2 for x, y, z).
 *   means  device float32 [n][3]
 *   perm   device int32 [n], written
 * Stream-ordered on `stream`; scratch (24 n bytes and the sort's tile
 * buffers) comes from the context's allocator and is released before the
 * call returns, which synchronises the stream.
 * Errors: HG_ERR_INVALID_ARG (n < 0, n > 2^30, null pointers), HG_ERR_OOM,
 * HG_ERR_CUDA. */
hg_status hg_spatial_order(hg_ctx* ctx, const float* means, int64_t n, int32_t* perm, void* stream);

/* Storage order of a scene: perm_host[i] = the caller's index of the
 * scene's i-th gaussian (the identity for HG_ORDER_INPUT).  Synchronous.
 * Errors: HG_ERR_INVALID_ARG, HG_ERR_CUDA. */
hg_status hg_scene_order(const hg_scene* scene, int32_t* perm_host);

/* Pinhole camera: world->camera 4x4 row-major (x right, y down, z forward),
 * focal lengths and principal point in pixels; pixel (i, j) has its centre
 * at (i, j) + (0.5, 0.5) in the (cx, cy) frame. */
typedef struct {
  float viewmat[16];
  float fx, fy, cx, cy;
  int32_t width, height;
} hg_camera;

/* Projected gaussian ("splat"), the record the projection front end hands to
 * partitioning and rasterisation (Sec. 4.2 outputs).  48 bytes. */
typedef struct {
  float mean2d[2];   /* pixel-centre convention: centre of pixel (i, j) is (i, j) */
  float conic[3];    /* (A, B, C): q = A dx^2 + 2 B dx dy + C dy^2 */
  float opacity;     /* sigmoid(logit) */
  float rgb[3];      /* max(0, SH + 0.5) */
  uint32_t depth_key;/* float32 bits of the camera-space depth */
  int32_t radius;    /* ceil(3 sqrt(lambda_max)), 0 = culled */
  float depth;
} hg_splat;

enum { HG_PATH_HIGS = 0, HG_PATH_PLAIN = 1 };
/* Gaussian-to-macro-tile test of the partitioning (Sec. 3.2, 4.3):
   HG_BIN_RECT     the 3-sigma rectangle in integers,
   HG_BIN_ELLIPSE  the rectangle refined per macro row band by the ellipse at
                   the opacity-aware level of the blend test (float32 with a
                   fixed operation order and margins; conservative, so the
                   image is the same, with fewer pairs).
   The plain per-tile path always uses the rectangle. */
enum { HG_BIN_RECT = 0, HG_BIN_ELLIPSE = 1 };
enum {
  HG_FLAG_ASYNC = 1,       /* do not synchronise or check the status word */
  HG_FLAG_TIMING = 2,      /* record per-stage CUDA events (hg_render_stats) */
  HG_FLAG_KEEP_SPLATS = 4, /* also write hg_splat records (hg_state_read) */
  HG_FLAG_INDEPENDENT = 8, /* render every batch independently from T = 1 and
                              composite the partials by Eq. 1 with exact-termination
                              replay (the paper's schedule) instead of chaining the
                              batches of a macro-tile in depth order */
  HG_FLAG_PROFILE = 16,    /* count rasteriser phase cycles (hg_frame_stats) */
  HG_FLAG_FP16 = 32        /* half-precision rasterisation (Sec. 3.5, 4.5): alpha of
                              the two pixels a thread owns in half2 arithmetic from
                              prescaled Cholesky factors and macro-tile-centred
                              coordinates; transmittance and colour stay float32 with
                              exact per-pixel termination.  Its own tolerance (PSNR,
                              not the float32 bounds); not with save_for_backward */
};

typedef struct {
  int32_t path;        /* HG_PATH_HIGS or HG_PATH_PLAIN */
  int32_t macro_w;     /* render tiles per macro-tile in x: 4 or 8 (default 8) */
  int32_t macro_h;     /* render tiles per macro-tile in y: 4 or 8 (default 4) */
  int32_t batch_cap;   /* B_r, 32..2048 multiple of 32 (default 1024) */
  int32_t bin_test;    /* HG_BIN_RECT or HG_BIN_ELLIPSE */
  float bg[3];         /* background colour added as C + T bg */
  int32_t save_for_backward;
  int32_t flags;       /* HG_FLAG_* */
} hg_render_opts;

/* Per-frame statistics (filled after the frame completed). */
typedef struct {
  int64_t n_views, n_gaussians, n_visible;
  int64_t n_pairs;        /* macro-tile pairs (HiGS) or tile pairs (plain) */
  int64_t n_segments;     /* macro-tiles over all views */
  int64_t n_batches;      /* N_R */
  int64_t max_segment;    /* largest segment (HiGS: macro-tile; plain path: 8x8 tile) */
  int64_t seg_by_tier[6]; /* segments sorted by tier: <=1K, <=4K, <=8K, <=16K, onesweep, empty/1 */
  int64_t n_sort_tiles;   /* onesweep tiles */
  int64_t n_replays;      /* merge replays (exact termination across batches) */
  int64_t raster_evals;   /* (gaussian, pixel) evaluations in the rasteriser */
  int32_t status;         /* device status word (hg_status) */
  int32_t sort_resorts;   /* shared-memory sort segments sorted again by the bitonic
                           * network (a run of more than 32 pairs in one bucket) */
  float ms_project, ms_partition, ms_sort, ms_raster, ms_merge, ms_total;
  /* with HG_FLAG_PROFILE: SM clock cycles summed over processing units of
   * [0] record gather, [1] tile masks + queue, [2] chain wait, and over warps
   * of [3] tile blending, [4] end-of-unit barrier; [5] units */
  int64_t raster_cycles[6];
  /* with HG_FLAG_PROFILE (float32 rasteriser): the intrinsic per-pixel work,
   * the (pixel, gaussian) evaluations a per-pixel renderer cannot skip
   * (support q <= 9 while the pixel is live, up to and including its stop),
   * and those of them that contributed a colour; and the rasteriser's
   * evaluations of pixels still live, in or out of the support (its other
   * evaluations are of pixels that had stopped) */
  int64_t pixel_support_evals, pixel_contrib_evals, pixel_live_evals;
} hg_frame_stats;

/* ---------------------------------------------------------------- context */
const char* hg_status_str(hg_status s);
const char* hg_last_error(void);
const char* hg_version(void);

/* Create a context on `device`; `alloc` may be NULL (cudaMalloc).  An
 * allocator whose alloc returns NULL makes the call that needed the memory
 * return HG_ERR_OOM (nothing is left half-built). */
hg_status hg_ctx_create(int device, const hg_allocator* alloc, hg_ctx** out);
void hg_ctx_destroy(hg_ctx* ctx);

/* Limits of the bounded device waits of frames enqueued on this context
 * after the call (failure detection, not part of the paper).
 *  wait_polls   polls of an mbarrier (the TMA stagings of the projection,
 *               the rasteriser and the backward) or of a onesweep look-back
 *               word before the wait gives up: the frame stops with
 *               HG_ERR_DEVICE_TIMEOUT (the CTA still waits, with the
 *               default limit, for the copies it issued, so nothing is left
 *               in flight) and later kernels of the frame return at once;
 *               default 2^24.
 *  chain_polls  polls of the batch chain (Sec. 3.4 ordered merge: the unit of
 *               rank k waiting for rank k-1 of its macro-tile) before the
 *               unit renders unchained from T = 1 and the merge composites
 *               it by Eq. 1 with replay (same image); default 200000
 *               (about 0.1 s).  A frame saved for the backward cannot
 *               render unchained: there a chain wait that gives up ends the
 *               frame with HG_ERR_DEVICE_TIMEOUT.  The backward's waits (its
 *               staged copies, and batch j waiting for batches j+1.. of its
 *               macro-tile) use wait_polls.
 * 0 gives up at once (tests of the failure paths); a negative value
 * restores the default.  Errors: HG_ERR_INVALID_ARG (NULL context, a value
 * above 2^32 - 1). */
hg_status hg_ctx_set_wait_limits(hg_ctx* ctx, int64_t wait_polls, int64_t chain_polls);

/* ------------------------------------------------------------------ scene */
/* Sec. 4.2 inputs.  Copies (borrow = 0) are enqueued on the legacy stream and
 * complete before the call returns. */
hg_status hg_create_scene(hg_ctx* ctx, const hg_scene_desc* desc, hg_scene** out);
void hg_destroy_scene(hg_scene* scene);
int64_t hg_scene_size(const hg_scene* scene);

/* ----------------------------------------------------------------- render */
/* Render `n_views` cameras of `scene` (the whole pipeline of Sec. 3-4).
 *  out_rgb: device, sum_v W_v H_v * 3 floats; out_T: device, sum_v W_v H_v
 *  floats or NULL.
 *  state: NULL -> the context's internal workspace is used (calls on the
 *  same context must then be stream-serialised); non-NULL -> *state (created
 *  on first use when *state == NULL) holds this frame's workspace, its
 *  statistics and, with save_for_backward, what hg_render_backward needs.
 *  Unless HG_FLAG_ASYNC is set the call synchronises `stream` and returns
 *  the device status; when a workspace buffer was too small it grows it and
 *  renders again, so HG_ERR_CAPACITY is only seen in asynchronous use.
 *  Asynchronous frames may follow one another on one state and stream (the
 *  call waits, on the host, only until the previous frame's camera table has
 *  been uploaded); hg_state_sync then returns the last frame's status.
 * Errors: HG_ERR_INVALID_ARG (bad sizes or options), HG_ERR_OOM,
 *  HG_ERR_CUDA, HG_ERR_DEVICE_TIMEOUT. */
hg_status hg_render(hg_scene* scene, const hg_camera* cams, int n_views,
                    const hg_render_opts* opts, float* out_rgb, float* out_T,
                    hg_state** state, void* stream);

/* Same pipeline starting from precomputed splats (skips the projection):
 * d_splats is device [n_views][n] hg_splat.  Used to run the discrete stages
 * on records computed elsewhere. */
hg_status hg_render_splats(hg_ctx* ctx, const hg_splat* d_splats, int64_t n,
                           const hg_camera* cams, int n_views, const hg_render_opts* opts,
                           float* out_rgb, float* out_T, hg_state** state, void* stream);

/* Backward of 0.5 ||C - C*||^2-style losses (the differentiable render that
 * Sec. 6 sketches): given dL/dC (device, same layout as out_rgb) of the frame
 * saved in `state` (rendered with save_for_backward), write dL/d(parameter)
 * into the device arrays (same shapes as the scene arrays, in the scene's
 * stored order (hg_scene_order); they are overwritten, not accumulated).
 * The forward rendered every batch chained (save_for_backward refuses
 * HG_FLAG_INDEPENDENT, and a chain wait that gives up ends that frame with
 * HG_ERR_DEVICE_TIMEOUT) and saved, per pixel of every (batch, tile) it
 * blended, the transmittance after the pixel's last contributing gaussian
 * of the batch and that gaussian's index.  The backward walks the batches
 * of each macro-tile from the last to the first and each batch back to
 * front, recovering T_i = T_{i+1} / (1 - alpha_i) and accumulating the
 * colour behind every gaussian from the back (starting at T_final bg), so
 * no difference of pixel-sized colours enters a gradient.  Stream-ordered;
 * its device status (a bounded wait that gave up: HG_ERR_DEVICE_TIMEOUT)
 * is returned by the next hg_state_sync.  Errors: HG_ERR_INVALID_ARG (no
 * saved frame, half or packed SH), HG_ERR_OOM, HG_ERR_CUDA. */
hg_status hg_render_backward(hg_state* state, const float* dL_drgb,
                             float* d_means, float* d_log_scales, float* d_quats,
                             float* d_opacity_logits, float* d_sh, void* stream);

/* ---------------------------------------------------------- optimisation
 * One densification-free optimisation step of the differentiable path
 * (Sec. 6) is: hg_render with save_for_backward, hg_l2_loss, then
 * hg_render_backward with its dL/dC, then hg_adam_step.  All four are
 * stream-ordered and run only this library's kernels. */

/* L2 photometric loss L = 1/2 sum_i (rgb_i - target_i)^2 over n floats and
 * its gradient dL/d rgb_i = rgb_i - target_i (float32).  rgb, target and
 * dL_drgb are device arrays of n floats (dL_drgb may alias neither input);
 * *loss (device double) receives L.  The squares are summed in float32
 * four consecutive elements at a time and those sums in double, in a fixed
 * order, so the result is deterministic.  Scratch for the reduction
 * is allocated through the context's allocator on the first call: make that
 * call outside CUDA graph capture.  Calls on one context must be
 * stream-serialised (they share the scratch).
 * Errors: HG_ERR_INVALID_ARG, HG_ERR_OOM, HG_ERR_CUDA. */
hg_status hg_l2_loss(hg_ctx* ctx, const float* rgb, const float* target, int64_t n,
                     float* dL_drgb, double* loss, void* stream);

typedef struct {
  float lr[5];        /* learning rate per group: means, log_scales, quats,
                         opacity_logits, sh */
  float beta1, beta2; /* moment decay rates, in [0, 1) */
  float eps;          /* denominator guard, >= 0 */
  int32_t step;       /* 1-based step count t of this update */
} hg_adam_opts;

/* One Adam step (Kingma and Ba) on every parameter array of `scene`, in
 * place: m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
 * p <- p - lr m / (1 - b1^t) / (sqrt(v / (1 - b2^t)) + eps), all five groups
 * in one kernel.  grads / m / v are device arrays with the shapes of the
 * scene arrays (float32, [n][3], [n][3], [n][4], [n], [n][K][3]); m and v are
 * updated in place and start at zero.  With a borrowed scene the caller's
 * parameter tensors are updated.
 * Errors: HG_ERR_INVALID_ARG (null buffer, step < 1, beta outside [0, 1)),
 *  HG_ERR_CUDA. */
hg_status hg_adam_step(hg_scene* scene, const float* const grads[5], float* const m[5],
                       float* const v[5], const hg_adam_opts* opts, void* stream);

void hg_state_free(hg_state* state);

/* Wait for the frame of `state` and return its device status. */
hg_status hg_state_sync(hg_state* state);

/* Statistics of the last frame rendered into `state` (synchronises). */
hg_status hg_render_stats(hg_state* state, hg_frame_stats* out);

/* Copy an intermediate buffer of the last frame to host memory (synchronises).
 * HiGS path: HG_BUF_SEG_OFF (uint32 [S+1]), HG_BUF_PAIR_KEYS (uint32 [P]),
 * HG_BUF_PAIR_IDS (uint32 [P]), HG_BUF_BATCHES (uint32 [N_R][3]: segment,
 * start, count).  Plain path (Sec. 2 / 5 baseline): HG_BUF_PLAIN_KEYS (uint64
 * [P] sorted keys, global render tile << 32 | depth key), HG_BUF_PLAIN_IDS
 * (uint32 [P] record index v n + i), HG_BUF_TILE_RANGES (uint32 [tiles][2]
 * [start, end) of every global render tile, 0 0 for an empty tile).  Both:
 * HG_BUF_SPLATS (hg_splat [V][n], needs HG_FLAG_KEEP_SPLATS),
 * HG_BUF_VIEW_SEG_BASE (uint32 [V+1]).  After hg_render_backward:
 * HG_BUF_GRAD2D (float32 [V][n][9], the gradient with respect to each
 * view's projected record: d mean2d x, y, d conic A, B, C of q = A dx^2 +
 * 2 B dx dy + C dy^2, d opacity, d rgb).  Both paths, the projection's
 * outputs: HG_BUF_RECORDS (float32 [V][n][16], the raster record of every
 * (view, gaussian): {mx, my, l0', l1'} {l2', o, radius bits, depth key
 * bits} {r, g, b, blend level} {0}, l' the Cholesky factors of the conic
 * prescaled by sqrt(log2(e) / 2); the records of culled entries are
 * unspecified) and HG_BUF_VISIBILITY (uint32 [V][ceil(n / 32)], bit i % 32
 * of word i / 32 set when gaussian i is visible in the view).  A buffer of
 * the other path (or a gradient before any backward) is
 * HG_ERR_UNSUPPORTED.  *bytes_needed receives the size; dst may be NULL to
 * query it. */
enum { HG_BUF_SEG_OFF = 0, HG_BUF_PAIR_KEYS = 1, HG_BUF_PAIR_IDS = 2, HG_BUF_BATCHES = 3,
       HG_BUF_SPLATS = 4, HG_BUF_VIEW_SEG_BASE = 5, HG_BUF_PLAIN_KEYS = 6, HG_BUF_PLAIN_IDS = 7,
       HG_BUF_TILE_RANGES = 8, HG_BUF_GRAD2D = 9, HG_BUF_RECORDS = 10, HG_BUF_VISIBILITY = 11 };
hg_status hg_state_read(hg_state* state, int which, void* dst, size_t dst_bytes,
                        size_t* bytes_needed);

/* ------------------------------------------------------------ CUDA graphs */
/* Multi-view frames in one captured CUDA graph (the batching of several
 * views per launch).  hg_graph_create renders one sizing frame
 * synchronously on `stream` (non-default stream required), grows `state`'s
 * workspace with headroom, then captures the whole pipeline for these views
 * into a graph that writes out_rgb / out_T.  `state` must stay alive and must
 * not be used by other calls while the graph exists. */
hg_status hg_graph_create(hg_scene* scene, const hg_camera* cams, int n_views, const hg_render_opts* opts,
                          float* out_rgb, float* out_T, hg_state* state, void* stream, hg_graph** out);
/* Enqueue one replay on `stream` (NULL = the capture stream). */
hg_status hg_graph_launch(hg_graph* graph, void* stream);
/* New poses with the captured count and resolutions for the next replay;
 * call only when no replay is pending (after hg_graph_sync). */
hg_status hg_graph_set_cameras(hg_graph* graph, const hg_camera* cams, int n_views);
/* Wait for the last replay (its own completion, not later work queued on
 * the same stream: two graphs over two states can be kept in flight on one
 * stream, each synchronised on its own) and return its device status;
 * HG_ERR_CAPACITY means a pose binned more pairs than the capture allows:
 * create the graph again from that pose. */
hg_status hg_graph_sync(hg_graph* graph);
/* Kernels one replay launches. */
int64_t hg_graph_kernels(const hg_graph* graph);
void hg_graph_destroy(hg_graph* graph);

/* ---------------------------------------------------------------- serving */
/* Continuous-batching render server over device-resident scenes (not in the
 * paper).  A dispatcher thread keeps up to max_inflight launches on the
 * device, each on its own stream with its own workspace; whenever a launch
 * slot is free it packs up to max_views_per_launch pending requests of the
 * scene of the oldest pending request (any mix of resolutions) into one
 * multi-view launch, if the memory the slots then hold stays within
 * mem_budget_bytes (0 = no limit).  Requests arriving meanwhile are admitted
 * as slots and memory free up, so their work overlaps on the device.  A
 * slot's workspace grows on demand: a launch that binned more pairs than it
 * holds is re-run after the slot reallocates (25% headroom), which delays
 * that launch and the device by the allocation; latency-sensitive callers
 * warm every slot with the largest launches they expect (max_views_per_launch
 * views at the largest resolution) before serving, or set presize_width /
 * presize_height: registering a scene then sizes every slot for
 * max_views_per_launch views of that resolution over the largest scene
 * registered so far (pair capacity 3 n V, which covers the macro-tile pairs
 * of the configs' scenes at 4K with headroom), so launches up to that size
 * never grow a workspace on the request path. */
typedef struct {
  int32_t max_inflight;          /* 1..64 launches on the device at once */
  int32_t max_views_per_launch;  /* 1..64 */
  int64_t mem_budget_bytes;
  int32_t batch_window_us;       /* hold the oldest request up to this long while fewer than
                                    max_views_per_launch requests of its scene are pending
                                    (0: launch as soon as a slot is free) */
  int32_t presize_width;         /* largest request resolution to size the slots for at */
  int32_t presize_height;        /* hg_serve_add_scene (0 0: grow on demand) */
  int32_t pad;
  hg_render_opts opts;           /* render options of every launch (path HiGS) */
} hg_serve_config;

typedef struct {
  int64_t submitted, completed, rejected, cancelled, failed, launches, queued, inflight_launches,
      max_inflight_seen, held_bytes;
  double p50_ms, p99_ms, mean_ms, max_ms; /* submit -> completion, completed requests */
  double req_per_s;                       /* completed requests per second since the last reset */
  double mean_views_per_launch;
} hg_serve_counters;

hg_status hg_serve_create(hg_ctx* ctx, const hg_serve_config* cfg, hg_server** out);
/* Register a scene (kept alive by the caller while the server exists). */
hg_status hg_serve_add_scene(hg_server* server, hg_scene* scene, int* scene_id);
/* Queue one view; returns at once.  out_rgb receives H*W*3 floats: device
 * memory (out_on_host = 0) or page-locked host memory (out_on_host = 1;
 * pageable memory would stall the dispatcher).  HG_ERR_NOT_FOUND for an
 * unknown scene, HG_ERR_OOM when the request alone exceeds the budget. */
hg_status hg_serve_submit(hg_server* server, int scene_id, const hg_camera* cam, float* out_rgb, int out_on_host,
                          uint64_t* req_id);
/* *done = 1 once the request finished; returns its status when done. */
hg_status hg_serve_poll(hg_server* server, uint64_t req_id, int* done);
/* Wait up to timeout_ms (< 0: forever) and release the request; returns its
 * status, HG_ERR_BUSY on timeout. */
hg_status hg_serve_wait(hg_server* server, uint64_t req_id, int timeout_ms);
/* Cancel a request that has not been launched (HG_ERR_BUSY if it has). */
hg_status hg_serve_cancel(hg_server* server, uint64_t req_id);
hg_status hg_serve_stats(hg_server* server, hg_serve_counters* out);
hg_status hg_serve_reset_stats(hg_server* server);
/* Stops the dispatcher after the launches in flight complete. */
void hg_serve_destroy(hg_server* server);

/* ----------------------------------------------------------------- tuning */
typedef struct {
  int32_t macro_w, macro_h, batch_cap;
  float ms; /* median frame time of the candidate */
} hg_tune_result;

/* Pick the macro-tile shape (4x4, 8x4, 8x8 render tiles; the partitioning
 * scale of Sec. 3.1) and the batch cap B_r (256, 512, 1024, 2048) that
 * render `cams` of `scene` fastest: every candidate renders the views
 * 1 + `iters` times on `stream` (synchronously) and is scored by the median
 * frame time.  *best receives `base` with the winning shape and cap (path
 * HiGS).  results (may be NULL) receives up to max_results candidates,
 * *n_results their count.  cache_path (may be NULL): a text file of
 * "key macro_w macro_h batch_cap ms" lines; a hit returns without rendering,
 * a sweep appends its winner.  Allocates a temporary workspace. */
hg_status hg_autotune(hg_scene* scene, const hg_camera* cams, int n_views, const hg_render_opts* base, int iters,
                      const char* cache_path, hg_render_opts* best, hg_tune_result* results, int max_results,
                      int* n_results, void* stream);

/* ---------------------------------------------------- allocation-free sort */
/* Segmented sort of (uint32 key, uint32 value) pairs, ascending by (key,
 * value) inside each segment, with no device allocation at all.  This is an
 * extra entry point with no counterpart in the paper: it exists for callers
 * that cannot call cudaMalloc where they sort (code running inside another
 * allocator's callback, or a host process that must not touch the device
 * heap while other work is in flight).  Its scratch (look-back words, digit
 * histograms, tile descriptors and a ping-pong copy of the pairs, about
 * 13 MB) is one fixed device array inside the library that every GPU which
 * loads the library holds until the process exits.  Four stable radix passes
 * over the values, then four over the keys, give the (key, value) order for
 * any input (all keys equal included) in time linear in n_pairs.
 *  d_seg_off: device [n_seg + 1], non-decreasing, d_seg_off[0] = 0,
 *             d_seg_off[n_seg] = n_pairs (copied to the host and checked).
 *  d_keys_in / d_vals_in: device [n_pairs], not modified unless they are
 *             the outputs (in place: d_keys_out == d_keys_in and
 *             d_vals_out == d_vals_in; every other overlap of the four
 *             ranges is rejected with HG_ERR_INVALID_ARG).
 *  d_keys_out / d_vals_out: device [n_pairs], the sorted pairs.
 * Limits: n_pairs <= 524288 and n_seg <= 512; larger inputs are rejected
 * with HG_ERR_INVALID_ARG and a message, before any device work.
 * The first call on a device looks up the scratch array's device address
 * (with that device current).  Every call clears the parts of the array
 * that must start at zero; all calls share the array, so calls whose GPU
 * work overlaps (other threads, other streams) race and must be serialised
 * by the caller.  The call synchronises `stream` (it reads d_seg_off and
 * the device status back), so it cannot be recorded into a stream capture:
 * on a capturing stream it returns HG_ERR_INVALID_ARG without enqueueing
 * anything.  It returns the device status. */
hg_status hg_segmented_sort_noalloc(const uint32_t* d_seg_off, int n_seg, int64_t n_pairs,
                                    const uint32_t* d_keys_in, const uint32_t* d_vals_in,
                                    uint32_t* d_keys_out, uint32_t* d_vals_out, void* stream);

/* Kernel launches issued by the library so far (all contexts). */
int64_t hg_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* HIGS_H */
