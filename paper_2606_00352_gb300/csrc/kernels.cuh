// Launch interface of the render kernels (host <-> device layouts).
#pragma once
#include "common.cuh"

namespace hg {

struct ProjectArgs {
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logits;
  const void* sh;         // element type sh_storage (HG_SH_*)
  int sh_storage;
  const float* sh_scale2; // packed SH: s / Q^2 per channel (device, 48), else null
  long long n;
  const ViewDesc* views;  // device
  int n_views;
  long long vis_words;    // ceil(n / 32)
  uint4* bin;             // [V][n] binning records (visible entries)
  float4* rec;            // [V][n][REC_F4]
  uint32_t* vis;          // [V][vis_words]
  uint32_t* dkeys;        // [V][n] depth keys (cell binning records)
  int bin_mode;           // BIN_CLASSIC, BIN_CELLS_RECT or BIN_CELLS_ELLIPSE
  int macro_w, macro_h;   // render tiles per macro cell (cell binning records)
  hg_splat* splats;       // optional [V][n]
  uint32_t wait_polls;    // mbarrier polls before a wait gives up (HG_ERR_DEVICE_TIMEOUT)
  FrameCounters* fc;
};

// Partition (count -> scan -> fill) and batch split of one frame.
struct PartitionArgs {
  const uint4* bin;        // [V][n] cell binning records
  const uint32_t* dkeys;   // [V][n] depth keys
  const uint32_t* vis;
  long long n;
  long long vis_words;
  const ViewDesc* views;
  int n_views;
  int n_seg;              // S = sum of macro-tiles
  int n_pb;               // N_B = ceil(n / B_p)
  int macro_w, macro_h;   // render tiles per macro-tile
  int max_nm;             // largest per-view macro-tile count
  uint16_t* hist;         // [N_B][S] (view v occupies columns [seg_base_v, seg_base_v + N_M_v))
  uint32_t* colpre;       // [N_B][S] exclusive prefix over partition batches
  uint32_t* seg_tot;      // [S]
  uint32_t* seg_off;      // [S + 1]
  uint32_t* first_batch;  // [S + 1]
  uint32_t* tier_list;    // [N_TIERS][S] segment ids per sort tier
  uint4* big_tiles;       // onesweep tiles {seg, start, count, tile index in segment}
  uint32_t* big_segs;     // [S] big segment ids
  uint32_t* big_tile_first; // [S] first tile of each big segment
  uint32_t* keys;         // pair keys [cap_pairs]
  uint32_t* vals;         // pair ids  [cap_pairs]
  uint4* batches;         // [cap_batches] {seg, start, count, j}
  uint32_t* batch_order;  // [cap_batches] raster schedule: batch ids, batch rank major
  uint32_t* rank_count;   // [MAX_RANKS + 1] scratch for the schedule
  int batch_cap;
  uint32_t cap_pairs, cap_batches, cap_tiles, cap_big_segs;
  uint32_t* seg_hist;     // [cap_big_segs][8][256] onesweep digit histograms, zeroed here for the big segments
  FrameCounters* fc;
};

// Sort tiers: segment-size limits handled by one CTA in shared memory.
constexpr int TIER0_MAX = 1024;    // 128 threads x 8 pairs, 2^12 buckets
constexpr int TIER1_MAX = 4096;    // 256 threads x 16, 2^13 buckets
constexpr int TIER2_MAX = 8192;    // 512 threads x 16, 2^14 buckets
constexpr int TIER3_MAX = 16384;   // 1024 threads x 16, 2^15 buckets
// tiers: <= 1K, <= 4K, <= 8K, <= 16K (shared memory), onesweep, empty / one pair
constexpr int N_TIERS = 6;
constexpr int TIER_OS = 4, TIER_NONE = 5;
constexpr int OS_THREADS = 512;    // onesweep tile: 512 threads x 16 items
constexpr int OS_ITEMS = 16;
constexpr int OS_TILE = OS_THREADS * OS_ITEMS;
constexpr int MAX_RANKS = 4096;    // batch ranks tracked by the raster schedule

struct SortArgs {
  uint32_t* keys;
  uint32_t* vals;
  uint32_t* keys_alt;
  uint32_t* vals_alt;
  const uint32_t* seg_off;
  const uint32_t* tier_list;  // [N_TIERS][S]
  int n_seg;
  const uint4* big_tiles;
  const uint32_t* big_segs;
  const uint32_t* big_tile_first;
  uint32_t* seg_hist;         // [cap_big_segs][8][256], zero on entry
  uint32_t* lookback;         // [8][cap_tiles][256]
  uint32_t cap_tiles, cap_big_segs;
  uint32_t wait_polls;        // look-back polls before a wait gives up
  int os_ctas;                // cap of the onesweep grids (0: one full wave)
  FrameCounters* fc;
};

struct RasterArgs {
  const float4* rec;          // [V][n][REC_F4]
  long long n;
  const ViewDesc* views;
  int n_views;
  int n_seg;
  const uint32_t* keys;       // sorted pair keys
  const uint32_t* vals;       // sorted pair ids
  const uint4* batches;       // {seg, start, count, j}
  const uint32_t* batch_order;
  uint32_t cap_batches;
  int batch_cap;              // B_r
  int macro_w, macro_h;
  float4* partial;            // [cap_batches][M][64] (r, g, b, +-T) of batches rendered unchained
  unsigned long long* active; // [cap_batches] tiles the batch blended
  uint32_t* chain;            // [S] batches of the segment composited in order so far; bit 31: chain broken
  uint32_t* mode;             // [cap_batches] BATCH_CHAINED or BATCH_LOCAL
  float4* tile_state;         // [total tiles][64] (r, g, b, +-T) after the chained batches
  uint32_t* tile_rank;        // [total tiles] rank + 1 of the last chained batch that blended the tile, 0 = none
  // optional [cap_batches][M][64], saved for the backward: per pixel of every
  // tile the batch blended, {the batch's own colour (r, g, b), the
  // transmittance after its last contributor in the batch} and the index in
  // the batch of that contributor (NO_LAST16: none)
  float4* exitrec;
  uint16_t* exitlast;
  int persistent_ctas;
  int independent;            // never wait: every batch after the first renders from T = 1
  int fp16;                   // half2 alpha (HG_FLAG_FP16)
  // direct output: the last chained batch of a macro-tile writes the image
  // (C + T bg, T) itself and marks the segment CHAIN_DONE for the merge
  int direct_out;
  const uint32_t* first_batch;  // [S + 1]
  float* out_rgb;
  float* out_T;
  float bg[3];
  int profile;                // accumulate phase cycles into FrameCounters::raster_cycles
  uint32_t wait_polls;        // mbarrier polls before a wait gives up (HG_ERR_DEVICE_TIMEOUT)
  uint32_t chain_polls;       // polls of the batch chain before a unit renders unchained
  FrameCounters* fc;
};

constexpr uint32_t NO_LAST = 0xffffu;  // exitlast: no gaussian of the batch contributed to the pixel (B_r <= 2048)
constexpr uint32_t BATCH_CHAINED = 1;  // rendered from the exact transmittance entering it
constexpr uint32_t BATCH_LOCAL = 2;    // rendered from T = 1; composited by the merge
constexpr uint32_t CHAIN_BROKEN = 0x80000000u;
constexpr uint32_t CHAIN_DONE = 0x40000000u;  // the raster wrote the segment's output

struct MergeArgs {
  const uint32_t* chain;      // [S]: CHAIN_DONE segments were written by the rasteriser
  const float4* partial;
  const unsigned long long* active;
  const uint32_t* mode;
  const float4* tile_state;
  const uint32_t* tile_rank;
  const uint32_t* first_batch;
  const uint4* batches;
  const uint32_t* vals;
  const float4* rec;
  long long n;
  const ViewDesc* views;
  int n_views;
  int total_tiles;
  int macro_w, macro_h;
  float bg[3];
  float* out_rgb;
  float* out_T;
  FrameCounters* fc;
};

struct BackwardArgs {
  const float4* rec;          // forward records [V][n][REC_F4]
  long long n;
  const ViewDesc* views;
  int n_views;
  const uint32_t* vals;       // sorted pair ids
  const uint4* batches;
  const uint32_t* batch_order;
  const unsigned long long* active;
  // [cap_batches][M][64] per blended (batch, tile, pixel), written by the
  // forward as {the batch's colour, T after its last contributor} and turned
  // by the suffix pass into {the colour behind the batch, T}
  float4* exitrec;
  const uint16_t* exitlast;   // [cap_batches][M][64] index of the last contributor, NO_LAST: none
  const float* dl_drgb;       // [pixels][3]
  float* g2d;                 // [V][n][9]: d mean2d (2), d conic A B C (3), d opacity, d rgb (3)
  int batch_cap;
  int macro_w, macro_h;
  uint32_t wait_polls;        // mbarrier polls before a wait gives up (HG_ERR_DEVICE_TIMEOUT)
  FrameCounters* fc;
};

// Colour behind every batch (the backward's suffix over a macro-tile's
// batches): one warp per render tile.
struct SuffixArgs {
  const unsigned long long* active;
  const uint32_t* first_batch;  // [S + 1]
  float4* exitrec;
  const ViewDesc* views;
  int n_views;
  int total_tiles;
  int macro_w, macro_h;
  float bg[3];
  FrameCounters* fc;
};

struct ProjectBackwardArgs {
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logits;
  const float* sh;
  long long n;
  int sh_degree;
  const ViewDesc* views;
  int n_views;
  const float* g2d;
  float* d_means;
  float* d_log_scales;
  float* d_quats;
  float* d_opacity_logits;
  float* d_sh;
};

struct PlainArgs {
  const uint4* bin;           // valid where the visibility bit is set
  const float4* rec;
  const uint32_t* vis;        // [V][vis_words]
  long long vis_words;
  long long n;
  const ViewDesc* views;
  int n_views;
  int total_tiles;
  uint32_t* counts;           // [V n]
  uint32_t* offsets;          // [V n + 1]
  uint32_t* scan_tmp;
  unsigned long long* keys;   // [cap] (global tile << 32) | depth key
  uint32_t* vals;             // [cap] record index v n + i
  unsigned long long* keys_alt;
  uint32_t* vals_alt;
  uint2* ranges;              // [total tiles]
  uint32_t* lookback;         // [8][cap_tiles][256]
  uint32_t* digit_hist;       // [8][256]
  uint32_t cap_pairs, cap_tiles;
  uint32_t wait_polls;        // look-back polls before a wait gives up
  float bg[3];
  float* out_rgb;
  float* out_T;
  FrameCounters* fc;
};

// Tiles of the segments sorted by the onesweep: {big segment index, start,
// count, tile index inside the segment}; a segment's tiles are consecutive.
struct OsTileView {
  const uint4* tiles;
  const uint32_t* tile_count;     // device
  const uint32_t* seg_hist;       // [big segments][npass][256]
  const uint32_t* seg_off;        // segment offsets, or NULL for one segment at 0
  const uint32_t* big_segs;       // big segment index -> segment id
  const uint32_t* big_tile_first;
};

// Onesweep LSD radix sort of the tiles' segments over digit passes
// [first_pass, first_pass + npass) of K keys with uint32 values; the result
// is in (keys, vals) for an even pass count, else in the alternates.
// seg_hist: [segments][NPASS][256] words (zeroed here when zero_hist, else
// zero on entry); lookback: [NPASS][lb_stride] words, lb_stride >= 256 x
// tiles (cleared by the histogram kernel).
template <typename K, int NPASS>
cudaError_t launch_onesweep(const OsTileView& tv, K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt,
                            uint32_t* seg_hist, size_t seg_hist_words, bool zero_hist, uint32_t* lookback,
                            size_t lb_stride, uint32_t* claims, int first_pass, int npass, uint32_t wait_polls,
                            FrameCounters* fc, cudaStream_t st, bool* result_in_alt);

// Host-side count of kernel launches issued by this library (all threads).
void note_launch(int n = 1);
long long launches_issued();

// Launch with programmatic stream serialization: the kernel's CTAs may be
// scheduled while the stream's previous kernel drains; the kernel must call
// pdl_wait() before reading that kernel's results.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t launch_project(const ProjectArgs& a, int deg, cudaStream_t st);
cudaError_t launch_splats_to_records(const hg_splat* sp, long long n, int n_views, long long vis_words,
                                     const ProjectArgs& out, cudaStream_t st);
cudaError_t launch_partition(const PartitionArgs& a, cudaStream_t st);
// Side streams of a frame's sort: the SMEM tiers sort disjoint segments, so
// three of them run on their own streams (forked from and joined back into
// the frame's stream with events, which stream capture turns into graph
// branches) while the smallest tier and the onesweep run on the frame's.
struct SortStreams {
  cudaStream_t aux[3];
  cudaEvent_t fork;
  cudaEvent_t join[3];
};
cudaError_t launch_sort(const SortArgs& a, cudaStream_t st, const SortStreams* ss);
cudaError_t launch_raster(const RasterArgs& a, cudaStream_t st);
cudaError_t launch_merge(const MergeArgs& a, cudaStream_t st);
cudaError_t launch_bwd_suffix(const SuffixArgs& a, cudaStream_t st);
cudaError_t launch_raster_backward(const BackwardArgs& a, cudaStream_t st);
cudaError_t launch_project_backward(const ProjectBackwardArgs& a, cudaStream_t st);
// returns the key pointer that holds the sorted result through *sorted_keys / *sorted_vals
cudaError_t launch_plain(PlainArgs& a, cudaStream_t st, unsigned long long** sorted_keys, uint32_t** sorted_vals);

}  // namespace hg
