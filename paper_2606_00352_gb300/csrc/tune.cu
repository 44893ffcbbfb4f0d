// Autotuner for the two free parameters of the hierarchy: the macro-tile
// shape (partitioning scale, Sec. 3.1) and the batch cap B_r (work-unit
// size).  For every candidate it renders the given views a few times on the
// given stream, takes the median of the CUDA-event frame times and keeps the
// fastest.  Results can be cached in a small text file keyed by the scene
// size, SH degree and the views' resolutions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"

using namespace hg;

static std::string tune_key(const hg_scene* s, const hg_camera* cams, int V) {
  std::ostringstream k;
  k << "n" << s->n << "_d" << s->deg << "_v" << V;
  for (int v = 0; v < V; ++v) k << "_" << cams[v].width << "x" << cams[v].height;
  return k.str();
}

static bool cache_lookup(const char* path, const std::string& key, hg_render_opts* o) {
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream in(line);
    std::string k;
    int mw, mh, cap;
    if (in >> k >> mw >> mh >> cap && k == key) {
      o->macro_w = mw;
      o->macro_h = mh;
      o->batch_cap = cap;
      return true;
    }
  }
  return false;
}

static void cache_store(const char* path, const std::string& key, const hg_render_opts* o, float ms) {
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << " " << o->macro_w << " " << o->macro_h << " " << o->batch_cap << " " << ms << "\n";
}

extern "C" hg_status hg_autotune(hg_scene* scene, const hg_camera* cams, int n_views, const hg_render_opts* base,
                                 int iters, const char* cache_path, hg_render_opts* best, hg_tune_result* results,
                                 int max_results, int* n_results, void* stream) {
  if (!scene || !cams || !base || !best || n_views <= 0 || n_views > MAX_VIEWS || iters <= 0) {
    hg_set_error("hg_autotune: bad arguments");
    return HG_ERR_INVALID_ARG;
  }
  *best = *base;
  best->path = HG_PATH_HIGS;
  best->flags &= ~(HG_FLAG_ASYNC | HG_FLAG_KEEP_SPLATS | HG_FLAG_PROFILE);
  if (n_results) *n_results = 0;
  const std::string key = tune_key(scene, cams, n_views);
  if (cache_lookup(cache_path, key, best)) return HG_OK;
  cudaSetDevice(scene->ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  long long pix = 0;
  for (int v = 0; v < n_views; ++v) pix += (long long)cams[v].width * cams[v].height;
  float* out = (float*)ctx_alloc(scene->ctx, sizeof(float) * 3 * (size_t)pix, st);
  if (!out) {
    hg_set_error("hg_autotune: output allocation failed");
    return HG_ERR_OOM;
  }
  hg_state* state = nullptr;
  hg_status r = state_create(scene->ctx, &state);
  if (r != HG_OK) {
    ctx_free(scene->ctx, out, sizeof(float) * 3 * (size_t)pix, st);
    return r;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int shapes[3][2] = {{4, 4}, {8, 4}, {8, 8}};
  const int caps[4] = {256, 512, 1024, 2048};
  float best_ms = 1e30f;
  int nr = 0;
  for (const auto& sh : shapes) {
    for (int cap : caps) {
      hg_render_opts o = *best;
      o.macro_w = sh[0];
      o.macro_h = sh[1];
      o.batch_cap = cap;
      o.save_for_backward = 0;
      FrameInputs in{scene, nullptr, scene->n};
      r = run_frame(state, in, &o, cams, n_views, out, nullptr, st);  // sizing + warm-up
      if (r != HG_OK) break;
      std::vector<float> ms;
      for (int it = 0; it < iters && r == HG_OK; ++it) {
        cudaEventRecord(e0, st);
        r = run_frame(state, in, &o, cams, n_views, out, nullptr, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms.push_back(t);
      }
      if (r != HG_OK) break;
      std::sort(ms.begin(), ms.end());
      const float med = ms[ms.size() / 2];
      if (results && nr < max_results) results[nr] = hg_tune_result{o.macro_w, o.macro_h, o.batch_cap, med};
      ++nr;
      if (med < best_ms) {
        best_ms = med;
        best->macro_w = o.macro_w;
        best->macro_h = o.macro_h;
        best->batch_cap = o.batch_cap;
      }
    }
    if (r != HG_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  hg_state_free(state);
  ctx_free(scene->ctx, out, sizeof(float) * 3 * (size_t)pix, st);
  if (n_results) *n_results = std::min(nr, max_results);
  if (r != HG_OK) return r;
  cache_store(cache_path, key, best, best_ms);
  return HG_OK;
}
