// Serving loop: continuous batching of render requests over device-resident
// scenes (not in the paper; the spec serving piece).
//
// A dispatcher thread owns `max_inflight` launch slots, each with its own
// stream, frame workspace (hg_state), output buffer and completion event.
// Whenever a slot is free and requests are pending, it takes the scene of
// the oldest pending request, packs up to `max_views_per_launch` pending
// requests of that scene (any mix of resolutions) into one multi-view
// launch, admits it if the memory the slots would then hold stays within
// `mem_budget_bytes`, enqueues the render and the copies of every view to
// its request's destination, and records the slot's event.  Launches in
// different slots overlap on the device; requests that arrive meanwhile are
// admitted as slots free up.  A launch that outgrew its workspace (device
// capacity status) is grown and re-run; a request whose launch fails gets
// the error and the loop keeps running.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

using namespace hg;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t id;
  int scene;
  hg_camera cam;
  float* out;
  bool out_on_host;
  Clock::time_point t_submit;
  hg_status status = HG_OK;
  bool done = false;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  hg_state* state = nullptr;
  float* out = nullptr;
  size_t out_bytes = 0;
  bool busy = false;
  int scene = -1;
  std::vector<uint64_t> reqs;
  std::vector<hg_camera> cams;
  long long pixels = 0;
};

size_t state_bytes(const hg_state* s) {
  size_t b = 0;
  for (int i = 0; i < BUF_COUNT; ++i) b += s->bufs[i].bytes;
  return b;
}

}  // namespace

struct hg_server {
  hg_ctx* ctx = nullptr;
  hg_serve_config cfg{};
  std::vector<hg_scene*> scenes;
  std::vector<Slot> slots;
  std::map<uint64_t, Request> reqs;
  std::deque<uint64_t> pending;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  uint64_t next_id = 1;
  // statistics
  std::vector<double> lat_ms;
  int64_t submitted = 0, completed = 0, rejected = 0, cancelled = 0, failed = 0, launches = 0, views = 0,
          max_inflight_seen = 0;
  Clock::time_point t0 = Clock::now();
};

static size_t launch_estimate(const hg_scene* s, long long pixels, int V) {
  // records + bin records + pairs/batches/partials ~ proportional to the
  // scene and the views, plus the outputs and per-pixel state
  return (size_t)s->n * V * (64 + 48) + (size_t)pixels * (12 + 16 + 24) + (64u << 20);
}

static size_t slot_bytes(const Slot& sl) { return (sl.state ? state_bytes(sl.state) : 0) + sl.out_bytes; }

static size_t held_bytes(const hg_server* S) {
  size_t b = 0;
  for (const Slot& sl : S->slots) b += slot_bytes(sl);
  return b;
}

// Memory the busy slots hold (the admission budget counts launches in flight).
static size_t busy_bytes(const hg_server* S) {
  size_t b = 0;
  for (const Slot& sl : S->slots)
    if (sl.busy) b += slot_bytes(sl);
  return b;
}

static void finish_request(hg_server* S, uint64_t id, hg_status st) {
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return;
  Request& r = it->second;
  r.status = st;
  r.done = true;
  if (st == HG_OK) {
    S->completed++;
    const double ms = std::chrono::duration<double, std::milli>(Clock::now() - r.t_submit).count();
    if (S->lat_ms.size() < (1u << 20)) S->lat_ms.push_back(ms);
  } else {
    S->failed++;
  }
}

// Enqueue the slot's launch (called with the lock held).
static hg_status start_launch(hg_server* S, Slot& sl) {
  hg_scene* sc = S->scenes[sl.scene];
  hg_render_opts o = S->cfg.opts;
  o.flags |= HG_FLAG_ASYNC;
  o.save_for_backward = 0;
  const size_t need = sizeof(float) * 3 * (size_t)sl.pixels;
  if (sl.out_bytes < need) {
    if (sl.out) ctx_free(S->ctx, sl.out, sl.out_bytes, sl.stream);
    sl.out = (float*)ctx_alloc(S->ctx, need, sl.stream);
    sl.out_bytes = sl.out ? need : 0;
    if (!sl.out) return HG_ERR_OOM;
  }
  FrameInputs in{sc, nullptr, sc->n};
  hg_status r = run_frame(sl.state, in, &o, sl.cams.data(), (int)sl.cams.size(), sl.out, nullptr, sl.stream);
  if (r != HG_OK) return r;
  size_t off = 0;
  for (size_t v = 0; v < sl.reqs.size(); ++v) {
    Request& q = S->reqs[sl.reqs[v]];
    const size_t bytes = sizeof(float) * 3 * (size_t)q.cam.width * q.cam.height;
    cudaError_t e = cudaMemcpyAsync(q.out, (const char*)sl.out + off, bytes, cudaMemcpyDefault, sl.stream);
    if (e != cudaSuccess) return hg_cuda_status(e, "serve copy");
    off += bytes;
  }
  cudaError_t e = cudaEventRecord(sl.done, sl.stream);
  if (e != cudaSuccess) return hg_cuda_status(e, "serve event");
  S->launches++;
  S->views += (int64_t)sl.reqs.size();
  return HG_OK;
}

static void dispatcher(hg_server* S) {
  cudaSetDevice(S->ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    bool progressed = false;
    // reap finished launches
    for (Slot& sl : S->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      const int status = q == cudaSuccess ? sl.state->fc_host->status : (int)HG_ERR_CUDA;
      if (q != cudaSuccess) cudaGetLastError();
      if (status == HG_ERR_CAPACITY) {
        // grow from the device counters and render the same requests again
        sl.state->cap_pairs = std::max(sl.state->cap_pairs, (size_t)sl.state->fc_host->n_pairs * 5 / 4 + 1024);
        sl.state->cap_batches = std::max(sl.state->cap_batches, (size_t)sl.state->fc_host->n_batches * 5 / 4 + 64);
        sl.state->cap_tiles = std::max(sl.state->cap_tiles, (size_t)sl.state->fc_host->n_big_tiles * 5 / 4 + 16);
        sl.state->cap_big_segs = std::max(sl.state->cap_big_segs, (size_t)sl.state->fc_host->n_big_segs + 16);
        if (start_launch(S, sl) == HG_OK) {
          progressed = true;
          continue;
        }
      }
      for (uint64_t id : sl.reqs) finish_request(S, id, status == HG_OK ? HG_OK : (hg_status)status);
      sl.busy = false;
      sl.reqs.clear();
      sl.cams.clear();
      progressed = true;
      S->cv_done.notify_all();
    }
    // admit pending requests into free slots
    bool holding = false;
    for (Slot& sl : S->slots) {
      if (sl.busy || S->pending.empty()) continue;
      const Request& oldest = S->reqs[S->pending.front()];
      const int scene = oldest.scene;
      if (S->cfg.batch_window_us > 0) {
        int same = 0;
        for (uint64_t id : S->pending) same += S->reqs[id].scene == scene;
        const double age_us = std::chrono::duration<double, std::micro>(Clock::now() - oldest.t_submit).count();
        if (same < S->cfg.max_views_per_launch && age_us < S->cfg.batch_window_us) {
          holding = true;  // wait for more views of this scene
          break;
        }
      }
      sl.reqs.clear();
      sl.cams.clear();
      sl.pixels = 0;
      for (auto it = S->pending.begin(); it != S->pending.end() && (int)sl.reqs.size() < S->cfg.max_views_per_launch;) {
        Request& q = S->reqs[*it];
        if (q.scene == scene) {
          sl.reqs.push_back(*it);
          sl.cams.push_back(q.cam);
          sl.pixels += (long long)q.cam.width * q.cam.height;
          it = S->pending.erase(it);
        } else {
          ++it;
        }
      }
      const size_t est = std::max(launch_estimate(S->scenes[scene], sl.pixels, (int)sl.reqs.size()), slot_bytes(sl));
      const size_t busy = busy_bytes(S);
      if (S->cfg.mem_budget_bytes > 0 && busy > 0 && busy + est > (size_t)S->cfg.mem_budget_bytes) {
        // not admitted now: back to the front of the queue, in order
        for (auto it = sl.reqs.rbegin(); it != sl.reqs.rend(); ++it) S->pending.push_front(*it);
        sl.reqs.clear();
        sl.cams.clear();
        break;
      }
      sl.scene = scene;
      sl.busy = true;
      const hg_status r = start_launch(S, sl);
      if (r != HG_OK) {
        for (uint64_t id : sl.reqs) finish_request(S, id, r);
        sl.busy = false;
        sl.reqs.clear();
        sl.cams.clear();
        S->cv_done.notify_all();
      }
      progressed = true;
    }
    int64_t inflight = 0;
    for (const Slot& sl : S->slots) inflight += sl.busy;
    S->max_inflight_seen = std::max(S->max_inflight_seen, inflight);
    if (!progressed) {
      if (inflight == 0 && S->pending.empty() && !holding)
        S->cv_work.wait(lk, [S] { return S->stop || !S->pending.empty(); });
      else
        S->cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

extern "C" hg_status hg_serve_create(hg_ctx* ctx, const hg_serve_config* cfg, hg_server** out) {
  if (!ctx || !cfg || !out || cfg->max_inflight < 1 || cfg->max_inflight > 64 || cfg->max_views_per_launch < 1 ||
      cfg->max_views_per_launch > MAX_VIEWS || cfg->presize_width < 0 || cfg->presize_height < 0 ||
      cfg->presize_width > 16384 || cfg->presize_height > 16384) {
    hg_set_error("hg_serve_create: bad configuration");
    return HG_ERR_INVALID_ARG;
  }
  cudaSetDevice(ctx->device);
  hg_server* S = new hg_server();
  S->ctx = ctx;
  S->cfg = *cfg;
  S->slots.resize(cfg->max_inflight);
  for (Slot& sl : S->slots) {
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    hg_status r = e == cudaSuccess ? state_create(ctx, &sl.state) : hg_cuda_status(e, "serve slot");
    if (r != HG_OK) {
      hg_serve_destroy(S);
      return r;
    }
  }
  S->worker = std::thread(dispatcher, S);
  *out = S;
  return HG_OK;
}

// Sizes a slot for a launch of max_views_per_launch views at the presize
// resolution over n gaussians (pair capacity 3 n V and what follows from it),
// so that no launch up to that size grows the slot on the request path.
static hg_status presize_slot(hg_server* S, Slot& sl, long long n) {
  const hg_serve_config& c = S->cfg;
  hg_render_opts o = c.opts;
  o.save_for_backward = 0;
  o.flags = 0;
  const int V = c.max_views_per_launch, W = c.presize_width, H = c.presize_height;
  FrameGeom g;
  g.V = V;
  const int tx = (W + TILE - 1) / TILE, ty = (H + TILE - 1) / TILE;
  const int mgx = (tx + o.macro_w - 1) / o.macro_w, mgy = (ty + o.macro_h - 1) / o.macro_h;
  g.S = V * mgx * mgy;
  g.total_tiles = V * tx * ty;
  g.pixels = (long long)V * W * H;
  g.max_nm = mgx * mgy;
  hg_state* st = sl.state;
  st->cap_pairs = std::max(st->cap_pairs, (size_t)(3 * n * V));
  st->cap_batches = std::max(st->cap_batches, st->cap_pairs / (size_t)o.batch_cap + (size_t)g.S + 64);
  st->cap_tiles = std::max(st->cap_tiles, st->cap_pairs / OS_TILE + 16);
  st->cap_big_segs = std::max(st->cap_big_segs, std::min<size_t>((size_t)g.S, st->cap_pairs / TIER3_MAX + 16));
  hg_status r = ensure_workspace(st, n, g, &o, sl.stream);
  if (r != HG_OK) return r;
  const size_t need = sizeof(float) * 3 * (size_t)g.pixels;
  if (sl.out_bytes < need) {
    if (sl.out) {
      cudaStreamSynchronize(sl.stream);
      ctx_free(S->ctx, sl.out, sl.out_bytes, sl.stream);
    }
    sl.out = (float*)ctx_alloc(S->ctx, need, sl.stream);
    sl.out_bytes = sl.out ? need : 0;
    if (!sl.out) return HG_ERR_OOM;
  }
  return HG_OK;
}

extern "C" hg_status hg_serve_add_scene(hg_server* S, hg_scene* scene, int* scene_id) {
  if (!S || !scene || !scene_id || scene->ctx != S->ctx) return HG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  S->scenes.push_back(scene);
  *scene_id = (int)S->scenes.size() - 1;
  if (S->cfg.presize_width > 0 && S->cfg.presize_height > 0) {
    long long n = 0;
    for (const hg_scene* sc : S->scenes) n = std::max<long long>(n, sc->n);
    for (Slot& sl : S->slots) {
      const hg_status r = presize_slot(S, sl, n);
      if (r != HG_OK) return r;
    }
  }
  return HG_OK;
}

extern "C" hg_status hg_serve_submit(hg_server* S, int scene_id, const hg_camera* cam, float* out_rgb,
                                     int out_on_host, uint64_t* req_id) {
  if (!S || !cam || !out_rgb || !req_id) return HG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (scene_id < 0 || scene_id >= (int)S->scenes.size()) {
    S->rejected++;
    hg_set_error("hg_serve_submit: unknown scene id");
    return HG_ERR_NOT_FOUND;
  }
  if (cam->width <= 0 || cam->height <= 0 || cam->width > 16384 || cam->height > 16384) {
    S->rejected++;
    hg_set_error("hg_serve_submit: bad resolution");
    return HG_ERR_INVALID_ARG;
  }
  const long long px = (long long)cam->width * cam->height;
  if (S->cfg.mem_budget_bytes > 0 && launch_estimate(S->scenes[scene_id], px, 1) > (size_t)S->cfg.mem_budget_bytes) {
    S->rejected++;
    hg_set_error("hg_serve_submit: the request alone exceeds the memory budget");
    return HG_ERR_OOM;
  }
  Request r;
  r.id = S->next_id++;
  r.scene = scene_id;
  r.cam = *cam;
  r.out = out_rgb;
  r.out_on_host = out_on_host != 0;
  r.t_submit = Clock::now();
  S->reqs[r.id] = r;
  S->pending.push_back(r.id);
  S->submitted++;
  *req_id = r.id;
  S->cv_work.notify_one();
  return HG_OK;
}

extern "C" hg_status hg_serve_poll(hg_server* S, uint64_t id, int* done) {
  if (!S || !done) return HG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return HG_ERR_NOT_FOUND;
  *done = it->second.done ? 1 : 0;
  return it->second.done ? it->second.status : HG_OK;
}

extern "C" hg_status hg_serve_wait(hg_server* S, uint64_t id, int timeout_ms) {
  if (!S) return HG_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return HG_ERR_NOT_FOUND;
  const auto pred = [&] { return it->second.done; };
  if (timeout_ms < 0)
    S->cv_done.wait(lk, pred);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
    return HG_ERR_BUSY;
  const hg_status st = it->second.status;
  S->reqs.erase(it);  // a completed request is released once waited for
  return st;
}

extern "C" hg_status hg_serve_cancel(hg_server* S, uint64_t id) {
  if (!S) return HG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto pit = std::find(S->pending.begin(), S->pending.end(), id);
  if (pit == S->pending.end()) return S->reqs.count(id) ? HG_ERR_BUSY : HG_ERR_NOT_FOUND;
  S->pending.erase(pit);
  Request& r = S->reqs[id];
  r.done = true;
  r.status = HG_ERR_CANCELLED;
  S->cancelled++;
  S->cv_done.notify_all();
  return HG_OK;
}

static double pct(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const size_t k = std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5));
  return v[k];
}

extern "C" hg_status hg_serve_stats(hg_server* S, hg_serve_counters* o) {
  if (!S || !o) return HG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  memset(o, 0, sizeof(*o));
  o->submitted = S->submitted;
  o->completed = S->completed;
  o->rejected = S->rejected;
  o->cancelled = S->cancelled;
  o->failed = S->failed;
  o->launches = S->launches;
  o->queued = (int64_t)S->pending.size();
  for (const Slot& sl : S->slots) o->inflight_launches += sl.busy;
  o->max_inflight_seen = S->max_inflight_seen;
  o->p50_ms = pct(S->lat_ms, 0.50);
  o->p99_ms = pct(S->lat_ms, 0.99);
  o->max_ms = S->lat_ms.empty() ? 0.0 : *std::max_element(S->lat_ms.begin(), S->lat_ms.end());
  double sum = 0.0;
  for (double x : S->lat_ms) sum += x;
  o->mean_ms = S->lat_ms.empty() ? 0.0 : sum / (double)S->lat_ms.size();
  const double secs = std::chrono::duration<double>(Clock::now() - S->t0).count();
  o->req_per_s = secs > 0 ? (double)S->completed / secs : 0.0;
  o->mean_views_per_launch = S->launches ? (double)S->views / (double)S->launches : 0.0;
  o->held_bytes = (int64_t)held_bytes(S);
  return HG_OK;
}

extern "C" hg_status hg_serve_reset_stats(hg_server* S) {
  if (!S) return HG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  S->lat_ms.clear();
  S->submitted = S->completed = S->rejected = S->cancelled = S->failed = S->launches = S->views = 0;
  S->max_inflight_seen = 0;
  S->t0 = Clock::now();
  return HG_OK;
}

extern "C" void hg_serve_destroy(hg_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (Slot& sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.state) hg_state_free(sl.state);
    if (sl.out) ctx_free(S->ctx, sl.out, sl.out_bytes, sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete S;
}
