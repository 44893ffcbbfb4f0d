"""Failure detection without a GPU fault: every bounded device wait can be
made to give up at once from the host (hg_ctx_set_wait_limits), and device
memory can run out on the host side (an allocator callback that returns
NULL).  The frame reports the failure as a status, the context stays usable,
and where a fallback exists its image is still the oracle's."""
import numpy as np
import pytest

from paper_2606_00352_gb300 import scenes
from oracle import composite as C
from oracle import project as P
from tests.helpers import compare_image

pytestmark = pytest.mark.gpu


def _scene():
    # dense enough that macro-tiles hold several batches of 64 and pixels
    # stop inside later batches
    return scenes.cluster_scene(12000, 8, 1.2, seed=41, sigma_range=(0.2, 0.8), extent=1.0)


def _img(lib, rgb, T, cam):
    return (rgb.view(cam.height, cam.width, 3).cpu().numpy(), T.view(cam.height, cam.width).cpu().numpy())


def test_chain_wait_gives_up_and_the_merge_replays(lib):
    """chain_polls = 0: every batch after a macro-tile's first gives up
    waiting for its predecessor, renders from T = 1, and the merge
    composites it by Eq. 1 with exact-termination replay: replays happen and
    the image is still the oracle's.  The default limit then chains again
    (no replay), with the same image."""
    ctx = lib.Context(0)
    scene = _scene()
    cam = scenes.look_at((2.6, 0.4, 0.3), width=120, height=88)
    ref = C.render(P.project(scene, cam))
    gs = lib.GpuScene.from_scene(ctx, scene)
    opts = lib.Options(macro_w=8, macro_h=4, batch_cap=64)
    ctx.set_wait_limits(chain_polls=0)
    st = lib.State(ctx)
    rgb, T = lib.render(gs, [cam], opts, state=st)
    stats = st.stats()
    assert stats["n_batches"] > stats["n_segments"], stats
    assert stats["n_replays"] > 0, stats
    img, t = _img(lib, rgb, T, cam)
    compare_image(img, t, ref, max_amb=0.004)  # measured 0.18%
    ctx.set_wait_limits()
    rgb2, T2 = lib.render(gs, [cam], opts, state=st)
    assert st.stats()["n_replays"] == 0
    img2, t2 = _img(lib, rgb2, T2, cam)
    compare_image(img2, t2, ref, max_amb=0.004)


def test_mbarrier_wait_gives_up_with_a_status(lib):
    """wait_polls = 0: the first staged TMA copy of the frame is not waited
    for, the frame ends with HG_ERR_DEVICE_TIMEOUT (each CTA still lets its
    copies land before it exits), and the next frame with the default limit
    renders the oracle's image on the same context."""
    ctx = lib.Context(0)
    scene = _scene()
    cam = scenes.look_at((2.6, 0.4, 0.3), width=120, height=88)
    gs = lib.GpuScene.from_scene(ctx, scene)
    ctx.set_wait_limits(wait_polls=0)
    with pytest.raises(lib.HgError) as e:
        lib.render(gs, [cam], lib.Options())
    assert e.value.status == -5
    ctx.set_wait_limits()
    rgb, T = lib.render(gs, [cam], lib.Options())
    img, t = _img(lib, rgb, T, cam)
    compare_image(img, t, C.render(P.project(scene, cam)), max_amb=0.004)


def test_allocator_out_of_memory_is_a_status(lib):
    """An allocator that returns NULL: scene creation and frame workspaces
    fail with HG_ERR_OOM, no crash; with memory back, the same context
    renders the same image as a context on cudaMalloc."""
    import torch
    budget = {"bytes": 0}
    live = {}

    def alloc(nbytes, stream, user):
        if nbytes > budget["bytes"]:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))
        live[p] = nbytes
        budget["bytes"] -= nbytes
        return p

    def free(ptr, nbytes, stream, user):
        budget["bytes"] += live.pop(int(ptr), 0)
        torch.cuda.caching_allocator_delete(int(ptr))

    ctx = lib.Context(0, allocator=(alloc, free))
    scene = scenes.tiny_workload()[0]
    cam = scenes.tiny_workload()[1][0]
    with pytest.raises(lib.HgError) as e:
        lib.GpuScene.from_scene(ctx, scene)
    assert e.value.status == -2
    budget["bytes"] = 4 << 20  # the scene (0.6 MB) fits, a frame workspace does not
    gs = lib.GpuScene.from_scene(ctx, scene)
    with pytest.raises(lib.HgError) as e:
        lib.render(gs, [cam], lib.Options())
    assert e.value.status == -2
    budget["bytes"] += 1 << 30
    rgb, T = lib.render(gs, [cam], lib.Options())
    ref_ctx = lib.Context(0, allocator="cuda")
    rgb_ref, T_ref = lib.render(lib.GpuScene.from_scene(ref_ctx, scene), [cam], lib.Options())
    assert torch.equal(rgb, rgb_ref) and torch.equal(T, T_ref)


def test_torch_caching_allocator_backs_the_default_context(lib):
    """The default context takes its device memory from the torch caching
    allocator: creating a scene adds at least the scene's bytes to torch's
    cumulative allocation counter, and closing it frees them back."""
    import torch
    torch.cuda.synchronize()
    key_a, key_f = "allocated_bytes.all.allocated", "allocated_bytes.all.freed"
    a0 = torch.cuda.memory_stats(0)[key_a]
    ctx = lib.Context(0)
    scene = scenes.tiny_workload()[0]
    gs = lib.GpuScene.from_scene(ctx, scene)
    a1 = torch.cuda.memory_stats(0)[key_a]
    assert a1 - a0 >= 56 * scene.n, (a0, a1)  # the scene's 56 bytes per gaussian came from torch's pool
    f1 = torch.cuda.memory_stats(0)[key_f]
    gs.close()
    ctx.close()
    assert torch.cuda.memory_stats(0)[key_f] - f1 >= 56 * scene.n
