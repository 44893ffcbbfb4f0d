#!/usr/bin/env python
"""Benchmark of the hierarchically tiled 3DGS render path on one node.

One step = one pass of the whole forward path (projection + SH, macro-tile
binning, segmented sort, batch split, raster, ordered merge) over one batch of
4 views of the 5.8M-gaussian SH-3 cluster scene at 1920x1080, replayed from a
captured CUDA graph with the next 4 poses of a 64-pose orbit.  The value is
frames (views) per second over all ranks; the plain one-CTA-per-8x8-tile path
with a global 64-bit sort is timed the same way on the same GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank renders its own poses of its own replica of
the scene (weak scaling, no data-path collective).  `--impl reference` times
the FP64 CPU oracle on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import copy
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p frames/s at 5.8M gaussians, HiGS vs per-tile path; serving p99 ms"
UNIT = "frames/s"
VIEWS = 4
N_POSES = 64
WIDTH, HEIGHT = 1920, 1080
# Sample of one oracle step: 1/ORACLE_FRACTION of the projection plus
# ORACLE_TILES tiles of one view; a frame is ORACLE_FRACTION such steps.
ORACLE_FRACTION = 1024
ORACLE_TILES = 32
# FP32-pipe instructions per (pixel, gaussian) evaluation of the blend step
# (dy, u, w, w^2, e, support test, o*2^-e, min, alpha test, 1-alpha, T',
# stop test, alpha*T, three colour FMAs)
RASTER_OPS_PER_EVAL = 16
FP32_LANES_PER_SM = 128


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "sm_max_mhz": d.get("sm_max_mhz", 2070.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def workload_config():
    from paper_2606_00352_gb300 import scenes
    return {"workload": "5.8M-gaussian SH-3 cluster scene (256 clusters, Zipf 1.4), 1920x1080, "
                        "4 views per captured CUDA graph, 64-pose orbit",
            "n_gaussians": 5_800_000, "resolution": f"{WIDTH}x{HEIGHT}", "views_per_step": VIEWS,
            "sh_degree": 3, "macro_tile": "4x4", "batch_cap": 1024, "bin_test": "ellipse", "scene_order": "spatial",
            "scene_extent": scenes.EXTENT,
            "orbit_radius": scenes.ORBIT_RADIUS,
            "l2": "inputs larger than L2 (scene arrays 1.37 GB, records 1.5 GB per step)"}


# ------------------------------------------------------------------ oracle
# The oracle's sampled work runs in a subprocess that never touches CUDA, so
# its worker pool is forked there (each worker inherits the scene and the
# full projection); one worker per host core.
_ORACLE = {}


def _oracle_state():
    import numpy as np
    from paper_2606_00352_gb300 import scenes
    from oracle import project as P, composite as Cmp
    if not _ORACLE:
        scene = scenes.scene_5m8()
        cam = scenes.scene_orbit(N_POSES, WIDTH, HEIGHT)[0]
        full = P.project(scene, cam)  # full projection for the sampled tiles (not timed)
        _ORACLE.update(scene=scene, cam=cam, full=full, cand=Cmp.tile_candidates(full), np=np)
    return _ORACLE


# Decision-ambiguity bands of the parity tests (support q, alpha, transmittance)
AMB_BANDS = (5e-5, 5e-5, 1e-5)


def _ambiguous_count(ref):
    """(decision-ambiguous pixels, evaluated pixels) of an oracle render."""
    a = ((ref["m_q"] < AMB_BANDS[0]) | (ref["m_alpha"] < AMB_BANDS[1]) | (ref["m_T"] < AMB_BANDS[2])) & ref["done"]
    return int(a.sum()), int(ref["done"].sum())


def _oracle_chunk(job):
    """One worker's share of a sampled step: the projection + binning of the
    slice [lo, lo + sl) and the compositing of `tiles`.  Returns (seconds,
    decision-ambiguous pixels, pixels) of the composited tiles."""
    from oracle import project as P, composite as Cmp
    st = _oracle_state()
    lo, sl, tiles = job
    t0 = time.perf_counter()
    Cmp.tile_candidates(P.project(st["scene"].subset(slice(lo, lo + sl)), st["cam"]))
    ref = Cmp.render(st["full"], tiles=tiles, cand=st["cand"])
    dt = time.perf_counter() - t0
    return (dt, *_ambiguous_count(ref))


def oracle_sample_steps(steps: int, warmup: int, seed: int = 0, cores: int = 1):
    """Times the FP64 oracle on bounded samples of the workload: per step
    each of `cores` workers projects and bins 1/ORACLE_FRACTION of the
    gaussians and composites ORACLE_TILES sampled tiles of one view (numpy,
    one thread per worker), so a frame is ORACLE_FRACTION / cores steps.
    Returns per-step wall seconds."""
    import multiprocessing as mp
    st = _oracle_state()
    np = st["np"]
    n = st["scene"].n
    sl = n // ORACLE_FRACTION
    gw, gh = -(-WIDTH // 8), -(-HEIGHT // 8)
    g = np.random.default_rng(seed)
    pool = mp.get_context("fork").Pool(cores) if cores > 1 else None
    times, amb = [], [0, 0]
    try:
        for k in range(warmup + steps):
            jobs = []
            for c in range(cores):
                lo = ((k * cores + c) * sl) % (n - sl)
                jobs.append((lo, sl, g.choice(gw * gh, ORACLE_TILES, replace=False)))
            t0 = time.perf_counter()
            res = [_oracle_chunk(jobs[0])] if pool is None else pool.map(_oracle_chunk, jobs, chunksize=1)
            dt = time.perf_counter() - t0
            if k >= warmup:
                times.append(dt)
                amb[0] += sum(r[1] for r in res)
                amb[1] += sum(r[2] for r in res)
    finally:
        if pool is not None:
            pool.close()
            pool.join()
    oracle_sample_steps.ambiguous = amb
    return times


def _config_tile_chunk(job):
    from oracle import composite as Cmp
    st = _ORACLE["cfg"]
    t0 = time.perf_counter()
    Cmp.render(st["proj"], tiles=job, cand=st["cand"])
    return time.perf_counter() - t0


def oracle_configs(cores: int):
    """The oracle on the tiny and the 1M configurations, one pose each, on one
    core and on `cores` workers: the tiny frame in full (projection and all
    1,024 tiles); the 1M frame at 1080p as its full projection plus a sample
    of 256 tiles per worker, scaled to the 32,400 tiles of the frame."""
    import multiprocessing as mp
    import numpy as np
    from paper_2606_00352_gb300 import scenes
    from oracle import project as P, composite as Cmp
    out = {}
    tiny_scene, tiny_cams = scenes.tiny_workload()
    cases = (("tiny_10k_256x256", tiny_scene, tiny_cams[0], None),
             ("1m_1920x1080", scenes.scene_1m(), scenes.scene_orbit(32, 1920, 1080)[0], 256))
    for name, scene, cam, sample in cases:
        t0 = time.perf_counter()
        proj = P.project(scene, cam)
        cand = Cmp.tile_candidates(proj)
        t_proj = time.perf_counter() - t0
        n_tiles = cand[0] * cand[1]
        _ORACLE["cfg"] = {"proj": proj, "cand": cand}
        g = np.random.default_rng(1)
        row = {"tiles": n_tiles, "projection_s_1core": round(t_proj, 3)}
        for workers in (1, cores):
            per = n_tiles if sample is None else sample
            if sample is None:
                chunks = np.array_split(np.arange(n_tiles), workers)
            else:
                chunks = [g.choice(n_tiles, per, replace=False) for _ in range(workers)]
            t0 = time.perf_counter()
            if workers == 1:
                _config_tile_chunk(chunks[0])
            else:
                with mp.get_context("fork").Pool(workers) as pool:
                    pool.map(_config_tile_chunk, chunks, chunksize=1)
            t_tiles = time.perf_counter() - t0
            tiles_done = n_tiles if sample is None else per * workers
            # the projection splits over the workers like the tiles do
            frame_s = t_proj / workers + t_tiles * n_tiles / tiles_done
            row[f"frames_per_s_{'1core' if workers == 1 else 'all_cores'}"] = round(1.0 / frame_s, 5)
        row["sample"] = ("whole frame" if sample is None else
                         f"full projection (timed on one core, divided by the workers) + {sample} sampled tiles per "
                         f"worker, scaled to {n_tiles} tiles")
        out[name] = row
    return out


def run_oracle_subprocess(steps: int, warmup: int, cores: int = 1, configs: bool = False):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-steps", str(steps), "--warmup", str(warmup),
           "--oracle-cores", str(cores)] + (["--oracle-configs"] if configs else [])
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample_desc(steps, cores=1):
    return (f"per step and worker ({cores} worker{'s' if cores > 1 else ''}, one per host core): FP64 projection + "
            f"tile binning of 1/{ORACLE_FRACTION} of the 5.8M gaussians + {ORACLE_TILES} sampled 8x8 tiles of one "
            f"1080p view; {steps} steps; frame time = mean step x {ORACLE_FRACTION} / {cores} "
            f"({ORACLE_FRACTION * ORACLE_TILES} tiles ~ the 32,400 of a frame)")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait(timeout=5)
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 9:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.strip() == "Active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------------ GPU arm
def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce_device():
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(local_ms: float, local_frames: float, world: int):
    """Whole-job frames/s: the frames all ranks rendered over the slowest
    rank's time.  Returns (value, max ms)."""
    ms = max_over_ranks(local_ms, world)
    frames = sum_over_ranks(local_frames, world)
    return frames / (ms * 1e-3), ms


def pose_batch(cams, step, rank):
    base = (step * VIEWS + rank * 7 * VIEWS) % N_POSES
    return [cams[(base + i) % N_POSES] for i in range(VIEWS)]


def sc_mod_decay(scene):
    from paper_2606_00352_gb300 import scenes
    return scenes.decaying_sh(scene)


def time_graph(lib, gs, cams, opts, steps, warmup, rank, world, stream, collect_stats=True, overlap=False):
    """Replays the captured frame: two graphs (two states, two output
    buffers) alternate on one stream, so the next step is always queued
    behind the running one and the device never waits for the host between
    steps; steps never overlap on the device (one stream), so each step's
    stage events time that step alone.  Per step: wait for the graph's
    previous replay (its own completion event), read its statistics, new
    poses, launch.  With overlap the two graphs replay on two streams, so
    two frames are in flight and one frame's stage tails overlap the next
    frame's start (the stage events then no longer time one step alone).
    Returns (ms for the timed steps, per-step stage stats, kernels per
    step)."""
    import torch
    pix = sum(c.width * c.height for c in cams[:VIEWS])
    streams = [stream, torch.cuda.Stream() if overlap else stream]
    graphs, states = [], []
    for gi in range(2):
        rgb = torch.empty(pix * 3, device="cuda", dtype=torch.float32)
        T = torch.empty(pix, device="cuda", dtype=torch.float32)
        state = lib.State(gs.ctx)
        # size the workspace for every pose batch the replays will use: a
        # captured graph cannot grow its buffers, and pair counts differ
        # between poses (the synchronous render grows the buffers as needed)
        sizing = lib.Options(**{**opts.__dict__, "flags": 0})
        for k in range(warmup + steps + 1):
            lib.render(gs, pose_batch(cams, k, rank), sizing, state=state, stream=stream, out_rgb=rgb, out_T=T)
        graphs.append(lib.Graph(gs, pose_batch(cams, 0, rank), opts, rgb, T, state, streams[gi]))
        states.append(state)
    for w in range(warmup):
        g = graphs[w % 2]
        g.set_cameras(pose_batch(cams, w + 1, rank))
        g.launch()
        g.sync()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stats = []
    pending = [False, False]
    ev0.record(stream)
    if overlap:
        streams[1].wait_event(ev0)
    for k in range(steps):
        i = k % 2
        if pending[i]:
            graphs[i].sync()
            if collect_stats:
                stats.append(states[i].stats())
        graphs[i].set_cameras(pose_batch(cams, warmup + 1 + k, rank))
        graphs[i].launch()
        pending[i] = True
    for i in (steps % 2, (steps + 1) % 2):
        if pending[i]:
            graphs[i].sync()
            if collect_stats:
                stats.append(states[i].stats())
    if overlap:
        joined = torch.cuda.Event()
        joined.record(streams[1])
        stream.wait_event(joined)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    kernels = graphs[0].kernels
    for g in graphs:
        g.close()
    for st in states:
        st.close()
    return ms, stats, kernels


def time_e2e(lib, gs, cams, opts, steps, warmup, rank, stream):
    """Public-API frames: hg_render with host cameras (uploaded by the call)
    and the rendered images read back into pinned host memory every step.
    Two image buffers alternate: the read-back of step k runs on a copy
    stream while hg_render draws step k + 1; every step's copies are inside
    the timed region, which ends when the last read-back has landed."""
    import torch
    pix = sum(c.width * c.height for c in cams[:VIEWS])
    rgb = [torch.empty(pix * 3, device="cuda", dtype=torch.float32) for _ in range(2)]
    host = [torch.empty(pix * 3, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    state = lib.State(gs.ctx)

    # the warm-up frames size the workspace (synchronous calls); the timed
    # ones are asynchronous, so the host enqueues the next frame while the
    # device renders, as a throughput client of hg_render would
    async_opts = copy.copy(opts)
    async_opts.flags = opts.flags | lib.FLAG_ASYNC

    def step(k, o=opts):
        b = k % 2
        stream.wait_event(copied[b])  # the buffer's previous read-back is done
        lib.render(gs, pose_batch(cams, k, rank), o, state=state, stream=stream, out_rgb=rgb[b], with_T=False)
        rendered[b].record(stream)
        copy_stream.wait_event(rendered[b])
        with torch.cuda.stream(copy_stream):
            host[b].copy_(rgb[b], non_blocking=True)
        copied[b].record(copy_stream)

    with torch.cuda.stream(stream):
        for b in range(2):
            copied[b].record(copy_stream)
        for w in range(warmup):
            step(w)
        copy_stream.synchronize()
        stream.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            step(warmup + k, async_opts)
        copy_stream.synchronize()
        stream.synchronize()
        dt = time.perf_counter() - t0
    status = state.sync()
    state.close()
    if status != 0:
        raise RuntimeError(f"asynchronous frames ended with device status {status}")
    view_desc_bytes = 144  # camera table entry uploaded per view by hg_render
    return {"seconds": dt, "h2d": VIEWS * view_desc_bytes, "d2h": pix * 3 * 4}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# each stage's kernels on this workload (spatially ordered scene), from ncu
# captures of the first frame of `bench.py --case 5m8 --macro 4x4 --steps 1
# --warmup 1`, one stage's kernels per capture (summary under profiles/),
# valid while the CUDA sources hash to `digest`.
MEASURED_TRAFFIC = {"digest": "1c9a648071c5868e",
                    "bytes": {"project": 2929.9e6, "partition": 916.5e6, "sort": 231.2e6, "raster": 2195.0e6,
                              "merge": 0.05e6}}


# CUDA sources that do not build or launch a kernel of the forward HiGS frame
# (backward, training, serving, CUDA graphs, autotuner, plain path, SH
# encoder): a change there leaves the forward kernels' DRAM bytes as captured
FORWARD_INDEPENDENT = ("backward.cu", "train.cu", "serve.cu", "graph.cu", "tune.cu", "plain.cu", "sh_codec.cu")


def sources_digest() -> str:
    """Digest of the CUDA sources the forward frame's kernels are built from
    (every header, every translation unit but FORWARD_INDEPENDENT)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2606_00352_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")) and f not in FORWARD_INDEPENDENT:
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def measured_traffic(stage: str):
    if MEASURED_TRAFFIC["digest"] != sources_digest():
        return None
    return MEASURED_TRAFFIC["bytes"].get(stage)


def roofline(stage_ms, stats0, n, pk, clock_mhz, sms):
    """Roofline of the stage that takes the most time per step; `sms` is the
    device's multiprocessor count."""
    hbm_peak = pk["hbm_gbs"]
    K = 16
    vis = statistics.mean(s["n_visible"] for s in stats0)
    vis_bits = VIEWS * ((n + 31) // 32) * 4
    proj_bytes = n * (44 + 12 * K) + vis * (16 + 4 + 48) + vis_bits
    pairs = statistics.mean(s["n_pairs"] for s in stats0)
    evals = statistics.mean(s["raster_evals"] for s in stats0)
    alu_peak = sms * FP32_LANES_PER_SM * pk["sm_max_mhz"] * 1e6 / 1e12  # T FP32-pipe ops/s
    table = {
        "project": {"bound": "hbm", "units": proj_bytes, "peak": hbm_peak, "unit": "GB/s",
                    "per_unit": "bytes: 236 read per gaussian + 68 written per visible (view, gaussian): "
                                "16 binning record, 4 depth key, 48 raster record; + visibility bits"},
        "partition": {"bound": "hbm", "units": vis * 16 * 2 + vis_bits * 2 + pairs * 8, "peak": hbm_peak,
                      "unit": "GB/s",
                      "per_unit": "bytes: 16 per visible (view, gaussian) and the visibility bits, read by count "
                                  "and by fill, + 8 written per pair"},
        "sort": {"bound": "hbm", "units": pairs * 16, "peak": hbm_peak, "unit": "GB/s",
                 "per_unit": "bytes: 8 read + 8 written per pair"},
        "raster": {"bound": "alu", "units": evals * RASTER_OPS_PER_EVAL, "peak": alu_peak, "unit": "Tops/s",
                   "per_unit": f"{RASTER_OPS_PER_EVAL} FP32-pipe ops per (pixel, gaussian) evaluation"},
    }
    out = {}
    for name, d in table.items():
        ms = max(stage_ms[name], 1e-6)
        if d["unit"] == "GB/s":
            ach = d["units"] / (ms * 1e-3) / 1e9
        else:
            ach = d["units"] / (ms * 1e-3) / 1e12
        out[name] = {"bound": d["bound"], "achieved": round(ach, 2), "peak": round(d["peak"], 1),
                     "unit": d["unit"], "frac": round(ach / d["peak"], 4), "ms": round(ms, 4),
                     "per_unit": d["per_unit"], "traffic": measured_traffic(name)}
    top = max(("project", "partition", "sort", "raster"), key=lambda k: stage_ms[k])
    return top, out


SERVE_RATES = (200, 500, 1000, 2000)
SERVE_RES = ((1280, 720), (1920, 1080), (3840, 2160))
SERVE_RES_W = (0.3, 0.5, 0.2)


def serving_run(higs, ctx, gscenes, seconds, seed=0, opts=None):
    """Poisson arrivals at each rate over the resident scenes; every request
    is a random orbit pose at a random resolution (weights 0.3/0.5/0.2).
    Returns one row per rate."""
    import numpy as np
    import torch
    from paper_2606_00352_gb300 import scenes
    rng = np.random.default_rng(seed)
    # every slot is sized when the scenes are added for the largest launch
    # (8 views at 3840 x 2160 of the largest scene), so no slot grows its
    # workspace while serving; the warm-up is one launch per slot
    big = max(SERVE_RES, key=lambda r: r[0] * r[1])
    srv = higs.Server(ctx, max_inflight=4, max_views_per_launch=8, mem_budget_bytes=64 << 30, opts=opts,
                      presize=big)
    sids = [srv.add_scene(g) for g in gscenes]
    pool = [torch.empty(3840 * 2160 * 3, device="cuda") for _ in range(48)]
    poses = {r: scenes.scene_orbit(N_POSES, r[0], r[1]) for r in SERVE_RES}
    warm = [srv.submit(sids[k % len(sids)], poses[SERVE_RES[k % 3]][k], pool[k]) for k in range(4)]
    for rid in warm:
        srv.wait(rid)
    rows = []
    for rate in SERVE_RATES:
        srv.reset_stats()
        inflight = [None] * len(pool)
        n = int(rate * seconds)
        gaps = rng.exponential(1.0 / rate, n)
        t = time.perf_counter()
        t_next = t
        for k in range(n):
            t_next += gaps[k]
            while time.perf_counter() < t_next:
                pass
            slot = k % len(pool)
            if inflight[slot] is not None:
                srv.wait(inflight[slot])  # back-pressure: the output buffer is still in use
            res = SERVE_RES[rng.choice(3, p=SERVE_RES_W)]
            cam = poses[res][int(rng.integers(0, N_POSES))]
            inflight[slot] = srv.submit(sids[int(rng.integers(0, len(sids)))], cam, pool[slot])
        for rid in inflight:
            if rid is not None:
                srv.wait(rid)
        wall = time.perf_counter() - t
        st = srv.stats()
        rows.append({"offered_req_per_s": rate, "completed": st["completed"],
                     "throughput_req_per_s": round(st["completed"] / wall, 1),
                     "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
                     "max_ms": round(st["max_ms"], 3), "views_per_launch": round(st["mean_views_per_launch"], 2),
                     "max_inflight": st["max_inflight_seen"]})
    srv.close()
    return rows


def train_setup(higs, ctx, spatial=True, opts=None):
    """The training workload: the 1M-gaussian scene, 4 views at 1080p, a
    Trainer (default launch configuration unless `opts`) whose target is the
    render of a perturbed copy (means + N(0, 1e-3), opacity logits + N(0,
    0.1)).  With `spatial` the parameter tensors are permuted once into
    hg_spatial_order before training (the optimiser state follows the same
    order)."""
    import torch
    from paper_2606_00352_gb300 import scenes
    scene = scenes.scene_1m()
    cams = scenes.scene_orbit(32, WIDTH, HEIGHT)[:VIEWS]
    target_gs = higs.GpuScene.from_scene(ctx, scenes.perturbed(scene))
    target, _ = higs.render(target_gs, cams, higs.Options(), with_T=False)
    target_gs.close()
    dev = torch.device("cuda", ctx.device)
    params = [torch.as_tensor(x, device=dev).contiguous()
              for x in (scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh)]
    if spatial:
        perm = higs.spatial_order(ctx, params[0]).long()
        params = [p[perm].contiguous() for p in params]
    return higs.Trainer(ctx, params, scene.sh_degree, cams, target, opts=opts), cams


def train_step_ms(higs, ctx, steps=10, spatial=True, opts=None):
    """Densification-free optimisation steps of the training workload
    (train_setup): forward (saving what the backward needs), L2 loss,
    backward, Adam, each timed with CUDA events."""
    import torch
    tr, cams = train_setup(higs, ctx, spatial, opts)
    stream = torch.cuda.current_stream()
    times, losses = [], []
    for k in range(steps + 2):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        rgb, _ = higs.render(tr.scene, cams, tr.opts, state=tr.state, with_T=False)
        ev[1].record(stream)
        higs.l2_loss(ctx, rgb, tr.target, tr.dl, tr.loss)
        ev[2].record(stream)
        higs.render_backward(tr.state, tr.scene, tr.dl, out=tr.grads)
        ev[3].record(stream)
        tr.t += 1
        higs.adam_step(tr.scene, tr.grads, tr.m, tr.v, tr.t, tr.lr)
        ev[4].record(stream)
        ev[4].synchronize()
        losses.append(float(tr.loss.item()))
        if k >= 2:
            times.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
    tr.close()
    med = [round(statistics.median(t[i] for t in times), 3) for i in range(4)]
    return {"forward_ms": med[0], "loss_ms": med[1], "backward_ms": med[2], "adam_ms": med[3],
            "step_ms": round(sum(med), 3), "loss_first": round(losses[0], 3), "loss_last": round(losses[-1], 3),
            "workload": "1M-gaussian SH-3 scene (64 clusters, Zipf 1.2), 4 views at 1920x1080, target = render "
                        "of a perturbed copy; forward with saved prefixes + hg_l2_loss + hg_render_backward + "
                        "hg_adam_step (3DGS learning rates)" + ("; parameters in hg_spatial_order" if spatial else "")
                        + (f"; macro {opts.macro_w}x{opts.macro_h}, B_r {opts.batch_cap}, "
                           f"{'ellipse' if opts.bin_test else 'rect'} binning" if opts else "")}


def gpu_arm(args):
    import numpy as np
    import torch
    from paper_2606_00352_gb300 import higs, scenes
    rank, world, local = dist_setup(args.gpus)
    higs.load()
    scene = scenes.scene_5m8()
    cams = scenes.scene_orbit(N_POSES, WIDTH, HEIGHT)
    ctx = higs.Context(torch.cuda.current_device())
    order = higs.ORDER_SPATIAL if args.order == "spatial" else higs.ORDER_INPUT
    gs = higs.GpuScene.from_scene(ctx, scene, order=order)
    scene16 = scene if not args.skip_plain else None
    del scene
    stream = torch.cuda.Stream()
    pk = peaks()
    tuned = None
    mw, mh = (int(x) for x in args.macro.split("x"))
    bin_test = higs.BIN_ELLIPSE if args.bin == "ellipse" else higs.BIN_RECT
    opts = higs.Options(path=higs.PATH_HIGS, macro_w=mw, macro_h=mh, batch_cap=args.cap, bin_test=bin_test,
                        flags=higs.FLAG_TIMING)
    if not args.skip_tune:
        best, table = higs.autotune(gs, pose_batch(cams, 0, rank), higs.Options(bin_test=bin_test), iters=3,
                                    stream=stream)
        opts = higs.Options(path=higs.PATH_HIGS, macro_w=best.macro_w, macro_h=best.macro_h,
                            batch_cap=best.batch_cap, bin_test=bin_test, flags=higs.FLAG_TIMING)
        tuned = {"chosen": f"{best.macro_w}x{best.macro_h}/{best.batch_cap}",
                 "candidates_ms": {f"{r[0]}x{r[1]}/{r[2]}": round(r[3], 3) for r in table}}

    sampler = ClockSampler(local)
    sampler.start()
    ms, stats, kernels = time_graph(higs, gs, cams, opts, args.steps, args.warmup, rank, world, stream)
    clocks = sampler.stop()
    value, ms = job_throughput(ms, args.steps * VIEWS, world)

    stage_ms = {k: statistics.mean(s["ms_" + k] for s in stats) for k in
                ("project", "partition", "sort", "raster", "merge")}
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    top, rl = roofline(stage_ms, stats, gs.n, pk, clocks.get("sm_mhz") or pk["sm_max_mhz"], sms)
    # the same replays with two frames in flight (two graphs on two streams)
    oms, _, _ = time_graph(higs, gs, cams, opts, args.steps, min(args.warmup, 3), rank, world, stream,
                           collect_stats=False, overlap=True)
    ovalue, oms = job_throughput(oms, args.steps * VIEWS, world)
    overlapped = {"value": round(ovalue, 2), "unit": UNIT, "ms_per_step": round(oms / args.steps, 4),
                  "note": "two captured frames in flight on two streams; the headline keeps one"}

    # the same workload with the SH coefficients stored in half precision
    # (236 -> 140 bytes read per gaussian) or in the 32-byte packed form
    # (236 -> 76), float32 arithmetic either way; PSNR of the first pose batch
    # against the float32-SH render
    sh_variants = {}
    if scene16 is not None:
        ref_img, _ = higs.render(gs, pose_batch(cams, 0, rank), opts, with_T=False, stream=stream)
        ref_img = ref_img.clone()
        for name, code in (("sh_f16", higs.SH_F16), ("sh_codec32", higs.SH_CODEC32)):
            gsv = higs.GpuScene.from_scene(ctx, scene16, sh_storage=code, order=order)
            hsteps = max(3, min(args.steps, 10))
            hms, hstats, _ = time_graph(higs, gsv, cams, opts, hsteps, min(args.warmup, 3), rank, world, stream)
            hvalue, hms = job_throughput(hms, hsteps * VIEWS, world)
            img, _ = higs.render(gsv, pose_batch(cams, 0, rank), opts, with_T=False, stream=stream)
            mse = float(((img - ref_img) ** 2).mean().item())
            sh_variants[name] = {"value": round(hvalue, 2), "unit": UNIT, "ms_per_step": round(hms / hsteps, 3),
                                 "project_ms": round(statistics.mean(s_["ms_project"] for s_ in hstats), 4),
                                 "psnr_db_vs_f32_sh": round(10 * math.log10(1.0 / max(mse, 1e-30)), 1)}
            gsv.close()
        # the packed codec on higher-order SH whose energy falls with the
        # degree (the stand-in for trained scenes): PSNR against the same
        # scene with float32 SH
        dscene = sc_mod_decay(scene16)
        gsd32 = higs.GpuScene.from_scene(ctx, dscene, order=order)
        gsdc = higs.GpuScene.from_scene(ctx, dscene, sh_storage=higs.SH_CODEC32, order=order)
        del dscene
        ref_d, _ = higs.render(gsd32, pose_batch(cams, 0, rank), opts, with_T=False, stream=stream)
        img_d, _ = higs.render(gsdc, pose_batch(cams, 0, rank), opts, with_T=False, stream=stream)
        mse = float(((img_d - ref_d) ** 2).mean().item())
        sh_variants["sh_codec32_decaying_sh"] = {
            "psnr_db_vs_f32_sh": round(10 * math.log10(1.0 / max(mse, 1e-30)), 1),
            "input": "the same scene with SH bands l >= 1 drawn from N(0, 0.2 * 0.25^l)"}
        gsd32.close()
        gsdc.close()
        del ref_d, img_d
        # half-precision rasterisation on the float32-SH scene
        fopts = higs.Options(path=higs.PATH_HIGS, macro_w=opts.macro_w, macro_h=opts.macro_h,
                             batch_cap=opts.batch_cap, bin_test=opts.bin_test,
                             flags=higs.FLAG_TIMING | higs.FLAG_FP16)
        hsteps = max(3, min(args.steps, 10))
        hms, hstats, _ = time_graph(higs, gs, cams, fopts, hsteps, min(args.warmup, 3), rank, world, stream)
        hvalue, hms = job_throughput(hms, hsteps * VIEWS, world)
        img, _ = higs.render(gs, pose_batch(cams, 0, rank), fopts, with_T=False, stream=stream)
        mse = float(((img - ref_img) ** 2).mean().item())
        sh_variants["fp16_raster"] = {"value": round(hvalue, 2), "unit": UNIT, "ms_per_step": round(hms / hsteps, 3),
                                      "raster_ms": round(statistics.mean(s_["ms_raster"] for s_ in hstats), 4),
                                      "psnr_db_vs_f32": round(10 * math.log10(1.0 / max(mse, 1e-30)), 1)}
    del scene16

    plain = None
    if not args.skip_plain:
        popts = higs.Options(path=higs.PATH_PLAIN, flags=higs.FLAG_TIMING)
        psteps = max(3, min(args.steps, 10))
        pms, pstats, _ = time_graph(higs, gs, cams, popts, psteps, min(args.warmup, 3), rank, world, stream)
        pvalue, pms = job_throughput(pms, psteps * VIEWS, world)
        plain = {"value": round(pvalue, 2), "unit": UNIT,
                 "ms_per_step": round(pms / psteps, 3),
                 "tile_pairs_per_step": int(statistics.mean(s["n_pairs"] for s in pstats)),
                 "peak_tile_gaussians": int(max(s["max_segment"] for s in pstats))}

    # the same scene at 3840x2160 (the paper's second resolution), HiGS with
    # the chosen shape and the plain per-tile path, 4 views per step
    uhd = None
    if not args.skip_plain:
        cams4k = scenes.scene_orbit(N_POSES, 3840, 2160)
        usteps = max(3, min(args.steps, 10))
        hopts = higs.Options(path=higs.PATH_HIGS, macro_w=opts.macro_w, macro_h=opts.macro_h,
                             batch_cap=opts.batch_cap, bin_test=opts.bin_test, flags=higs.FLAG_TIMING)
        ums, ustats, _ = time_graph(higs, gs, cams4k, hopts, usteps, min(args.warmup, 3), rank, world, stream)
        uvalue, ums = job_throughput(ums, usteps * VIEWS, world)
        popts4 = higs.Options(path=higs.PATH_PLAIN, flags=higs.FLAG_TIMING)
        pums, _, _ = time_graph(higs, gs, cams4k, popts4, usteps, min(args.warmup, 3), rank, world, stream,
                                collect_stats=False)
        puvalue, pums = job_throughput(pums, usteps * VIEWS, world)
        u_stage = {k: round(statistics.mean(s_["ms_" + k] for s_ in ustats), 4)
                   for k in ("project", "partition", "sort", "raster", "merge")}
        u_pairs = statistics.mean(s_["n_pairs"] for s_ in ustats)
        uhd = {"resolution": "3840x2160", "value": round(uvalue, 2), "unit": UNIT,
               "ms_per_step": round(ums / usteps, 3), "plain_path_value": round(puvalue, 2),
               "speedup_vs_plain": round(uvalue / puvalue, 3), "stage_ms": u_stage,
               "pairs_per_step": int(u_pairs),
               "sort": {"achieved_gbs": round(u_pairs * 16 / (u_stage["sort"] * 1e-3) / 1e9, 1),
                        "frac_of_hbm": round(u_pairs * 16 / (u_stage["sort"] * 1e-3) / 1e9 / pk["hbm_gbs"], 4),
                        "per_unit": "8 B read + 8 B written per pair"}}

    serving = None
    if not args.skip_serve and world == 1:
        from paper_2606_00352_gb300 import scenes as sc_mod
        small = [higs.GpuScene.from_scene(ctx, sc_mod.cluster_scene(n, 256, 1.4, seed=11 + k,
                                                                    sigma_range=sc_mod.CLUSTER_SIGMA,
                                                                    extent=sc_mod.EXTENT), order=order)
                 for k, n in enumerate((500_000, 2_000_000))]
        sopts = higs.Options(path=higs.PATH_HIGS, macro_w=opts.macro_w, macro_h=opts.macro_h,
                             batch_cap=opts.batch_cap, bin_test=opts.bin_test)
        serving = {"rows": serving_run(higs, ctx, small + [gs], seconds=1.5, opts=sopts),
                   "workload": "3 resident scenes (0.5M, 2M, 5.8M gaussians, 256 clusters, Zipf 1.4); Poisson "
                               "arrivals; random orbit pose at 1280x720 / 1920x1080 / 3840x2160 (0.3/0.5/0.2); "
                               "up to 4 launches in flight, up to 8 views per launch; latency submit -> completion"}
        del small
    training = None
    if not args.skip_train and world == 1:
        # the training default of higs.Trainer (macro 4x4, B_r 512, ellipse)
        training = train_step_ms(higs, ctx, spatial=args.order == "spatial",
                                 opts=higs.Options(macro_w=4, macro_h=4, batch_cap=512, bin_test=higs.BIN_ELLIPSE))

    e2e_opts = higs.Options(path=higs.PATH_HIGS, macro_w=opts.macro_w, macro_h=opts.macro_h,
                            batch_cap=opts.batch_cap, bin_test=opts.bin_test)
    e2e_steps = max(3, min(args.steps, 10))
    e = time_e2e(higs, gs, cams, e2e_opts, e2e_steps, min(args.warmup, 3), rank, stream)
    e2e_t = max_over_ranks(e["seconds"], world)
    e2e = {"value": round(sum_over_ranks(e2e_steps * VIEWS, world) / e2e_t, 2), "unit": UNIT,
           "h2d_bytes_per_step": e["h2d"], "d2h_bytes_per_step": e["d2h"]}

    # one profiled frame: raster phase cycles and the intrinsic per-pixel work
    pst = higs.State(ctx)
    popts_prof = higs.Options(path=higs.PATH_HIGS, macro_w=opts.macro_w, macro_h=opts.macro_h,
                              batch_cap=opts.batch_cap, bin_test=opts.bin_test, flags=higs.FLAG_PROFILE)
    higs.render(gs, pose_batch(cams, 0, rank), popts_prof, state=pst, stream=stream, with_T=False)
    prof = pst.stats()
    pst.close()

    if rank != 0:
        return
    cpu, amb_stats = None, None
    if world == 1 and not args.skip_cpu:
        # the oracle on every host core (the headline baseline), one core, and
        # the tiny and 1M configurations on one and on all cores
        cores = host_cores()
        r = run_oracle_subprocess(steps=4, warmup=1, cores=cores, configs=True)
        r1 = run_oracle_subprocess(steps=4, warmup=1, cores=1)
        cpu = {"value": r["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": oracle_sample_desc(4, cores),
               "one_core": {"value": r1["value"], "unit": UNIT, "cores": 1, "sample": oracle_sample_desc(4, 1)},
               "host_cores": os.cpu_count(), "configs": r.get("configs")}
        amb_stats = {"decision_ambiguous_pixels": r["ambiguous_pixels"], "oracle_sampled_pixels": r["sampled_pixels"],
                     "decision_ambiguous_fraction": round(r["ambiguous_pixels"] / max(1, r["sampled_pixels"]), 6),
                     "bands_q_alpha_T": list(AMB_BANDS)}
    s0 = stats
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config() | {"macro_tile": f"{opts.macro_w}x{opts.macro_h}", "batch_cap": opts.batch_cap,
                                       "bin_test": args.bin, "scene_order": args.order},
        "roofline": {k: v for k, v in rl[top].items() if k in ("bound", "achieved", "peak", "unit", "frac")}
        | {"kernel": top, "traffic": rl[top]["traffic"], "peak_source": pk["source"], "sms": sms,
           "peak_derivation": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {pk['sm_max_mhz']:.0f} MHz"
           if rl[top]["bound"] == "alu" else "measured copy bandwidth"},
        "stages": rl | {"merge": {"ms": round(stage_ms["merge"], 4)}},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(kernels * args.steps),
        "clocks": clocks,
        "plain_path": plain,
        "uhd_4k": uhd,
        "two_frames_in_flight": overlapped,
        "precision_variants": sh_variants or None,
        "speedup_vs_plain": round(value / plain["value"], 3) if plain else None,
        "frame_stats": {
            "pairs_per_step": int(statistics.mean(s["n_pairs"] for s in s0)),
            "batches_per_step": int(statistics.mean(s["n_batches"] for s in s0)),
            "max_segment": int(max(s["max_segment"] for s in s0)),
            "peak_unit_gaussians": int(min(opts.batch_cap, max(s["max_segment"] for s in s0))),
            "segments_by_tier_last_pose": s0[-1]["seg_by_tier"],
            "replays_per_step": int(statistics.mean(s["n_replays"] for s in s0)),
            "raster_evals_per_step": int(statistics.mean(s["raster_evals"] for s in s0)),
            "visible_per_step": int(statistics.mean(s["n_visible"] for s in s0)),
            "pixel_support_evals_first_step": prof["pixel_support_evals"],
            "pixel_contrib_evals_first_step": prof["pixel_contrib_evals"],
            "raster_evals_first_step": prof["raster_evals"],
            "pixel_live_evals_first_step": prof["pixel_live_evals"],
            "intrinsic_share_of_raster_evals": round(prof["pixel_support_evals"] / max(1, prof["raster_evals"]), 4),
            # the other evaluations: live pixels outside the support, and
            # pixels that stopped before their tile's last live pixel
            "live_outside_support_share": round((prof["pixel_live_evals"] - prof["pixel_support_evals"])
                                                / max(1, prof["raster_evals"]), 4),
            "stopped_pixel_share": round((prof["raster_evals"] - prof["pixel_live_evals"])
                                         / max(1, prof["raster_evals"]), 4),
            "raster_phase_cycles_first_step": dict(zip(("gather", "masks", "chain_wait", "blend_warps",
                                                        "end_barrier_warps", "units"), prof["raster_cycles"])),
        } | (amb_stats or {}),
        "serving_p99_ms": next((r["p99_ms"] for r in serving["rows"] if r["offered_req_per_s"] == 1000), None)
        if serving else None,
        "serving": serving,
        "autotune": tuned,
        "train_step": training,
    }
    print(json.dumps(line), flush=True)


def profile_case(args):
    """Small case for kernel captures: the 1M-gaussian SH-3 scene, 4 views
    at 1080p, rendered `--steps` times through hg_render (no graph)."""
    import torch
    from paper_2606_00352_gb300 import higs, scenes
    higs.load()
    torch.cuda.set_device(0)
    scene = scenes.scene_5m8() if args.case == "5m8" else scenes.scene_1m()
    cams = scenes.scene_orbit(N_POSES, WIDTH, HEIGHT)
    ctx = higs.Context(0)
    gs = higs.GpuScene.from_scene(ctx, scene, order=higs.ORDER_SPATIAL if args.order == "spatial" else higs.ORDER_INPUT)
    st = higs.State(ctx)
    path = higs.PATH_PLAIN if args.case == "1m-plain" else higs.PATH_HIGS
    mw, mh = (int(x) for x in args.macro.split("x"))
    opts = higs.Options(path=path, macro_w=mw, macro_h=mh, batch_cap=args.cap,
                        bin_test=higs.BIN_ELLIPSE if args.bin == "ellipse" else higs.BIN_RECT,
                        flags=higs.FLAG_TIMING | (higs.FLAG_PROFILE if args.profile else 0))
    for k in range(args.warmup + args.steps):
        higs.render(gs, pose_batch(cams, k, 0), opts, state=st)
    torch.cuda.synchronize()
    s = st.stats()
    print(json.dumps({"case": args.case, "stats": s}), flush=True)


def profile_train_case(args):
    """Small case for kernel captures of the training step: the training
    workload (train_setup) in the Trainer's default launch configuration
    (macro 4x4, B_r = 512, ellipse), `--warmup + --steps` optimisation
    steps through Trainer.step."""
    import torch
    from paper_2606_00352_gb300 import higs
    higs.load()
    torch.cuda.set_device(0)
    ctx = higs.Context(0)
    tr, _ = train_setup(higs, ctx, spatial=args.order == "spatial")
    loss = None
    for _ in range(args.warmup + args.steps):
        loss = tr.step()
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "loss": float(loss.item())}), flush=True)
    tr.close()


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = host_cores()
    r = run_oracle_subprocess(steps=args.steps, warmup=args.warmup, cores=cores)
    fps = r["value"]
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": int(args.gpus),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": fps, "unit": UNIT, "kind": "oracle", "cores": cores,
                             "sample": oracle_sample_desc(args.steps, cores)},
            "e2e": {"value": fps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--skip-train", action="store_true")
    ap.add_argument("--skip-tune", action="store_true")
    ap.add_argument("--oracle-steps", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-cores", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-configs", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--case", default="", choices=["", "1m", "1m-plain", "5m8", "train1m"],
                    help="small profiling case instead of the benchmark")
    ap.add_argument("--profile", action="store_true", help="count rasteriser phase cycles (profiling case)")
    ap.add_argument("--macro", default="8x4", choices=["4x4", "8x4", "8x8"], help="macro shape without autotuning")
    ap.add_argument("--cap", type=int, default=1024, help="batch cap B_r without autotuning")
    ap.add_argument("--bin", default="ellipse", choices=["rect", "ellipse"], help="macro-tile binning test")
    ap.add_argument("--order", default="spatial", choices=["input", "spatial"],
                    help="scene storage order (hg_create_scene HG_ORDER_*)")
    args = ap.parse_args()
    if args.warmup < 3 and not args.oracle_steps and not args.case:
        args.warmup = 3
    if args.oracle_steps:
        c = max(1, args.oracle_cores)
        times = oracle_sample_steps(args.oracle_steps, args.warmup, cores=c)
        ms = statistics.mean(times) * 1e3
        amb, px = oracle_sample_steps.ambiguous
        out = {"value": c / (statistics.mean(times) * ORACLE_FRACTION), "ms_per_step": ms, "cores": c,
               "times": times, "ambiguous_pixels": amb, "sampled_pixels": px}
        if args.oracle_configs:
            out["configs"] = oracle_configs(c)
        print(json.dumps(out))
        return
    if args.case == "train1m":
        profile_train_case(args)
    elif args.case:
        profile_case(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
