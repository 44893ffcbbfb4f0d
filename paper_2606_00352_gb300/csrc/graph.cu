// Multi-view frames captured once into a CUDA graph and replayed (the
// "views in one captured graph" batching).  The capture records the whole
// pipeline with fixed workspace capacities; the per-frame camera upload is a
// memcpy node reading the state's pinned view table, so new poses of the
// same resolutions are set between replays without recapturing.
#include <cuda_runtime.h>

#include <cstring>

#include "internal.h"

using namespace hg;

struct hg_graph {
  hg_state* state = nullptr;
  hg_scene* scene = nullptr;
  hg_render_opts opts{};
  int V = 0;
  hg_camera cams[MAX_VIEWS];
  float* out_rgb = nullptr;
  float* out_T = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaStream_t st = nullptr;
  long long launches = 0;
};

extern "C" hg_status hg_graph_create(hg_scene* scene, const hg_camera* cams, int n_views, const hg_render_opts* opts,
                                     float* out_rgb, float* out_T, hg_state* state, void* stream, hg_graph** out) {
  if (!scene || !cams || !opts || !out_rgb || !state || !out || n_views <= 0 || n_views > MAX_VIEWS) {
    hg_set_error("hg_graph_create: bad arguments");
    return HG_ERR_INVALID_ARG;
  }
  if (!stream) {
    hg_set_error("hg_graph_create: capture needs a non-default stream");
    return HG_ERR_INVALID_ARG;
  }
  cudaSetDevice(scene->ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  // sizing frame: grows the workspace to this scene and these views
  hg_render_opts sized = *opts;
  sized.flags &= ~HG_FLAG_ASYNC;
  FrameInputs in{scene, nullptr, scene->n};
  hg_status r = run_frame(state, in, &sized, cams, n_views, out_rgb, out_T, st);
  if (r != HG_OK) return r;
  // a little headroom for poses that bin more pairs than the sizing one
  state->cap_pairs += state->cap_pairs / 4;
  state->cap_batches += state->cap_batches / 4;
  state->cap_tiles += state->cap_tiles / 4;
  state->cap_big_segs += state->cap_big_segs / 4;
  r = run_frame(state, in, &sized, cams, n_views, out_rgb, out_T, st);
  if (r != HG_OK) return r;
  hg_graph* G = new hg_graph();
  G->state = state;
  G->scene = scene;
  G->opts = *opts;
  G->opts.flags |= HG_FLAG_ASYNC;
  G->V = n_views;
  memcpy(G->cams, cams, sizeof(hg_camera) * n_views);
  G->out_rgb = out_rgb;
  G->out_T = out_T;
  G->st = st;
  FrameGeom g;
  r = build_views(state, cams, n_views, &G->opts, g);
  if (r != HG_OK) {
    delete G;
    return r;
  }
  const long long l0 = launches_issued();
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    delete G;
    return hg_cuda_status(e, "begin capture");
  }
  r = enqueue_frame(state, in, &G->opts, g, out_rgb, out_T, st);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(st, &graph);
  if (r != HG_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    delete G;
    return r != HG_OK ? r : hg_cuda_status(e, "end capture");
  }
  G->launches = launches_issued() - l0;
  G->g = graph;
  e = cudaGraphInstantiate(&G->ge, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    delete G;
    return hg_cuda_status(e, "graph instantiate");
  }
  state->geom = g;
  state->opts = G->opts;
  state->last_stream = st;
  *out = G;
  return HG_OK;
}

extern "C" hg_status hg_graph_launch(hg_graph* G, void* stream) {
  if (!G) return HG_ERR_INVALID_ARG;
  cudaStream_t st = stream ? (cudaStream_t)stream : G->st;
  cudaError_t e = cudaGraphLaunch(G->ge, st);
  if (e == cudaSuccess) e = cudaEventRecord(G->state->frame_done, st);
  if (e != cudaSuccess) return hg_cuda_status(e, "graph launch");
  G->state->last_stream = st;
  G->state->has_frame = true;
  G->state->frame_in_graph = true;
  ++G->state->frame_id;  // a new frame (a saved one needs its own backward suffix)
  G->state->has_grad2d = false;
  return HG_OK;
}

// New poses (same count and resolutions) for the next replay.  The previous
// replay must have completed (hg_graph_sync) because the camera upload reads
// the pinned view table when the graph runs.
extern "C" hg_status hg_graph_set_cameras(hg_graph* G, const hg_camera* cams, int n_views) {
  if (!G || !cams || n_views != G->V) return HG_ERR_INVALID_ARG;
  for (int v = 0; v < n_views; ++v)
    if (cams[v].width != G->cams[v].width || cams[v].height != G->cams[v].height) {
      hg_set_error("hg_graph_set_cameras: resolution differs from the captured one");
      return HG_ERR_INVALID_ARG;
    }
  FrameGeom g;
  hg_status r = build_views(G->state, cams, n_views, &G->opts, g);
  if (r != HG_OK) return r;
  memcpy(G->cams, cams, sizeof(hg_camera) * n_views);
  return HG_OK;
}

extern "C" hg_status hg_graph_sync(hg_graph* G) {
  if (!G) return HG_ERR_INVALID_ARG;
  cudaError_t e = state_wait(G->state);
  if (e != cudaSuccess) return hg_cuda_status(e, "graph sync");
  const int status = G->state->fc_host->status;
  if (status != HG_OK) hg_set_error(std::string("device status: ") + hg_status_str((hg_status)status));
  return (hg_status)status;
}

extern "C" int64_t hg_graph_kernels(const hg_graph* G) { return G ? G->launches : 0; }

extern "C" void hg_graph_destroy(hg_graph* G) {
  if (!G) return;
  cudaStreamSynchronize(G->state->last_stream);
  if (G->ge) cudaGraphExecDestroy(G->ge);
  if (G->g) cudaGraphDestroy(G->g);
  delete G;
}
