"""Serving loop (continuous batching) and autotuner, through the C ABI."""
import numpy as np
import pytest

from paper_2606_00352_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    return lib.Context(0)


@pytest.fixture(scope="module")
def scene_set(lib, ctx):
    a = lib.GpuScene.from_scene(ctx, scenes.cluster_scene(60_000, 16, 1.4, seed=1, sigma_range=scenes.CLUSTER_SIGMA,
                                                          extent=scenes.EXTENT))
    b = lib.GpuScene.from_scene(ctx, scenes.cluster_scene(150_000, 32, 1.2, seed=2, sigma_range=scenes.CLUSTER_SIGMA,
                                                          extent=scenes.EXTENT))
    return [a, b]


def _alone(lib, gs, cam):
    import torch
    rgb, _ = lib.render(gs, [cam], lib.Options(), with_T=False)
    torch.cuda.synchronize()
    return rgb.cpu().numpy()


def test_results_equal_alone_and_in_the_mix(lib, ctx, scene_set):
    """A burst of mixed-resolution requests over two scenes: every result is
    the same as rendering that view alone (views are independent, so bit
    for bit), and requests were batched and overlapped on the device."""
    import torch
    srv = lib.Server(ctx, max_inflight=3, max_views_per_launch=6, batch_window_us=3000)
    ids = [srv.add_scene(g) for g in scene_set]
    g = np.random.default_rng(0)
    res = [(320, 180), (640, 360), (200, 120), (97, 61)]
    reqs = []
    for k in range(40):
        sid = int(g.integers(0, 2))
        w, h = res[int(g.integers(0, len(res)))]
        cam = scenes.orbit(24, scenes.ORBIT_RADIUS, w, h)[k % 24]
        out = torch.empty(w * h * 3, device="cuda")
        reqs.append((srv.submit(sid, cam, out), sid, cam, out))
    for rid, _, _, _ in reqs:
        assert srv.wait(rid, 60_000) == 0
    st = srv.stats()
    assert st["completed"] == 40 and st["failed"] == 0
    assert st["launches"] < 40 and st["mean_views_per_launch"] > 1.0
    assert st["max_inflight_seen"] >= 2
    for rid, sid, cam, out in reqs:
        alone = _alone(lib, scene_set[sid], cam)
        assert np.array_equal(out.cpu().numpy(), alone)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_mixed_resolution_launch_matches_oracle(lib, ctx):
    """Requests of one scene at four resolutions submitted in one burst are
    served by multi-view launches that mix resolutions (a launch shape only
    the server makes); every served image matches the float64 oracle."""
    import torch
    from oracle import composite as C
    from oracle import project as P
    from tests.helpers import compare_image
    scene = scenes.cluster_scene(20_000, 8, 1.2, seed=23, sigma_range=scenes.CLUSTER_SIGMA, extent=scenes.EXTENT)
    gs = lib.GpuScene.from_scene(ctx, scene)
    srv = lib.Server(ctx, max_inflight=1, max_views_per_launch=8, batch_window_us=20_000)
    sid = srv.add_scene(gs)
    res = [(96, 64), (64, 48), (120, 72), (33, 17)]
    reqs = []
    for k in range(8):
        w, h = res[k % len(res)]
        cam = scenes.orbit(8, scenes.ORBIT_RADIUS, w, h)[k]
        out = torch.empty(w * h * 3, device="cuda")
        reqs.append((srv.submit(sid, cam, out), cam, out))
    for rid, _, _ in reqs:
        assert srv.wait(rid, 60_000) == 0
    st = srv.stats()
    assert st["launches"] < len(reqs) and st["mean_views_per_launch"] > 1.0, st
    for _, cam, out in reqs:
        img = out.view(cam.height, cam.width, 3).cpu().numpy()
        compare_image(img, None, C.render(P.project(scene, cam)), max_amb=0.011)  # measured 0.53%
    srv.close()


def test_presized_slots_never_grow(lib, ctx, scene_set):
    """presize=(W, H): adding a scene sizes every slot for a full launch at
    that resolution, so bursts of full launches hold no more memory than
    after the sizing (no workspace growth on the request path), and the
    results equal renders alone."""
    import torch
    srv = lib.Server(ctx, max_inflight=2, max_views_per_launch=4, batch_window_us=2000, presize=(640, 360))
    sid = srv.add_scene(scene_set[1])
    held0 = srv.stats()["held_bytes"]
    assert held0 > 0
    cams = scenes.scene_orbit(16, 640, 360)
    outs = [torch.empty(640 * 360 * 3, device="cuda") for _ in cams]
    for k0 in range(0, len(cams), 8):
        ids = [srv.submit(sid, cams[k], outs[k]) for k in range(k0, k0 + 8)]
        for r in ids:
            assert srv.wait(r, 60_000) == 0
    st = srv.stats()
    assert st["held_bytes"] == held0, (st["held_bytes"], held0)
    assert st["mean_views_per_launch"] > 1.0
    for c, o in zip(cams, outs):
        assert np.array_equal(o.cpu().numpy(), _alone(lib, scene_set[1], c))
    srv.close()


def test_host_outputs_cancel_and_errors(lib, ctx, scene_set):
    import torch
    srv = lib.Server(ctx, max_inflight=1, max_views_per_launch=2)
    sid = srv.add_scene(scene_set[0])
    cam = scenes.scene_orbit(4, 160, 90)[0]
    host = torch.empty(160 * 90 * 3, dtype=torch.float32, pin_memory=True)
    rid = srv.submit(sid, cam, host, on_host=True)
    assert srv.wait(rid, 60_000) == 0
    assert np.array_equal(host.numpy(), _alone(lib, scene_set[0], cam))
    # unknown scene and bad resolution are refused at submission
    dev = torch.empty(16, device="cuda")
    st, _ = srv.submit_status(7, cam, dev)
    assert st == -7
    bad = scenes.scene_orbit(4, 160, 90)[1]
    bad.width = 0
    st, _ = srv.submit_status(sid, bad, dev)
    assert st == -1
    # cancel: flood one slot, cancel the last request before it launches
    outs = [torch.empty(640 * 360 * 3, device="cuda") for _ in range(12)]
    big = scenes.scene_orbit(12, 640, 360)
    ids = [srv.submit(sid, c, o) for c, o in zip(big, outs)]
    c = srv.cancel(ids[-1])
    assert c in (0, -6)
    for r in ids[:-1]:
        assert srv.wait(r, 60_000) == 0
    assert srv.wait(ids[-1], 60_000) in (0, -8)
    srv.close()


def test_memory_budget_admission(lib, ctx, scene_set):
    import torch
    srv = lib.Server(ctx, max_inflight=4, max_views_per_launch=4, mem_budget_bytes=1 << 20)
    sid = srv.add_scene(scene_set[1])
    st, _ = srv.submit_status(sid, scenes.scene_orbit(2, 320, 180)[0], torch.empty(320 * 180 * 3, device="cuda"))
    assert st == -2  # a single request larger than the budget is rejected
    srv.close()
    # a budget that fits one launch at a time still completes everything
    srv = lib.Server(ctx, max_inflight=4, max_views_per_launch=2, mem_budget_bytes=600 << 20)
    sid = srv.add_scene(scene_set[1])
    cams = scenes.scene_orbit(8, 320, 180)
    outs = [torch.empty(320 * 180 * 3, device="cuda") for _ in cams]
    ids = [srv.submit(sid, c, o) for c, o in zip(cams, outs)]
    for r in ids:
        assert srv.wait(r, 60_000) == 0
    for c, o in zip(cams, outs):
        assert np.array_equal(o.cpu().numpy(), _alone(lib, scene_set[1], c))
    srv.close()


def test_autotune_picks_a_valid_candidate(lib, ctx, scene_set, tmp_path):
    cams = scenes.scene_orbit(4, 480, 270)
    cache = str(tmp_path / "tune.txt")
    best, res = lib.autotune(scene_set[1], cams, iters=2, cache_path=cache)
    assert len(res) == 12
    shapes = {(r[0], r[1]) for r in res}
    assert shapes == {(4, 4), (8, 4), (8, 8)} and {r[2] for r in res} == {256, 512, 1024, 2048}
    fastest = min(res, key=lambda r: r[3])
    assert (best.macro_w, best.macro_h, best.batch_cap) == fastest[:3]
    again, res2 = lib.autotune(scene_set[1], cams, iters=2, cache_path=cache)
    assert res2 == [] and (again.macro_w, again.macro_h, again.batch_cap) == fastest[:3]


def test_graph_replay_equals_render(lib, ctx, scene_set):
    """Views captured in one CUDA graph and replayed with new poses give the
    same images as direct renders of those poses."""
    import torch
    gs = scene_set[1]
    cams = scenes.scene_orbit(8, 256, 144)
    pix = 4 * 256 * 144
    rgb = torch.empty(pix * 3, device="cuda")
    T = torch.empty(pix, device="cuda")
    st = lib.State(ctx)
    stream = torch.cuda.Stream()
    graph = lib.Graph(gs, cams[:4], lib.Options(), rgb, T, st, stream)
    graph.set_cameras(cams[4:])
    graph.launch()
    graph.sync()
    ref, _ = lib.render(gs, cams[4:], lib.Options(), with_T=False)
    torch.cuda.synchronize()
    assert np.array_equal(rgb.cpu().numpy(), ref.cpu().numpy())
    graph.close()
