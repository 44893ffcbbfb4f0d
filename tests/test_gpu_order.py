"""Spatial storage order (hg_spatial_order, HG_ORDER_SPATIAL scenes) through
the C ABI against the oracle's definition (oracle.order): the permutation
bit for bit, and the render of a spatially ordered scene against the FP64
oracle's render of the same permuted scene."""
import numpy as np
import pytest

from paper_2606_00352_gb300 import scenes
from oracle import composite as C
from oracle import order as O
from oracle import project as P
from tests.helpers import compare_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    return lib.Context(0)


def _means(n, seed):
    g = np.random.default_rng(seed)
    m = g.normal(0, 3, (n, 3)).astype(np.float32)
    if n > 10:
        m[g.integers(0, n, 5), g.integers(0, 3, 5)] = np.nan      # non-finite coordinates
        m[g.integers(0, n, 3), 1] = np.inf
        m[n // 3] = m[n // 2]                                        # an exact duplicate (tie)
    return m


@pytest.mark.parametrize("n", [1, 1000, 8192, 123457, 2_000_003])
def test_spatial_order_matches_oracle(lib, ctx, n):
    import torch
    m = _means(n, n)
    perm = lib.spatial_order(ctx, torch.from_numpy(m).cuda()).cpu().numpy()
    np.testing.assert_array_equal(perm, O.spatial_order(m))


def test_spatial_order_empty_and_bad_arguments(lib, ctx):
    import torch
    assert lib.spatial_order(ctx, torch.zeros((0, 3), device="cuda")).numel() == 0
    with pytest.raises(lib.HgError):
        lib.check(ctx.lib.hg_spatial_order(ctx.h, None, -1, None, None))
    with pytest.raises(lib.HgError):
        lib.check(ctx.lib.hg_spatial_order(ctx.h, None, 10, None, None))


def _permuted(scene, perm):
    sc = scene.copy()
    sc.means, sc.log_scales = scene.means[perm], scene.log_scales[perm]
    sc.quats, sc.opacity_logits, sc.sh = scene.quats[perm], scene.opacity_logits[perm], scene.sh[perm]
    return sc


@pytest.mark.parametrize("macro", [(4, 4), (8, 4)])
def test_spatial_scene_renders_the_permuted_scene(lib, ctx, macro):
    """HG_ORDER_SPATIAL: the stored order is the oracle's order of the
    means, and the image is the oracle's image of the scene in that order
    (the (depth key, index) order then uses the stored indices)."""
    import torch
    scene = scenes.cluster_scene(30_000, 8, 1.2, seed=31, sigma_range=scenes.CLUSTER_SIGMA, extent=scenes.EXTENT)
    gs = lib.GpuScene.from_scene(ctx, scene, order=lib.ORDER_SPATIAL)
    perm = gs.order()
    np.testing.assert_array_equal(perm, O.spatial_order(scene.means))
    ref_scene = _permuted(scene, perm)
    cams = scenes.scene_orbit(8, 320, 200)[2:4]
    rgb, T = lib.render(gs, cams, lib.Options(macro_w=macro[0], macro_h=macro[1]))
    torch.cuda.synchronize()
    imgs = [x.detach().cpu().numpy() for x in lib.split_views(rgb, cams, 3)]
    ts = [x.detach().cpu().numpy() for x in lib.split_views(T, cams, 1)]
    for v, cam in enumerate(cams):
        compare_image(imgs[v], ts[v], C.render(P.project(ref_scene, cam)), max_amb=0.001)  # measured 0.04%
    gs.close()


def test_spatial_scene_with_packed_sh(lib, ctx):
    """Packed SH codes follow the stored order: the codes of the spatial
    scene are the input-order scene's codes permuted (same scales)."""
    scene = scenes.cluster_scene(5000, 4, 1.2, seed=32, sigma_range=scenes.CLUSTER_SIGMA, extent=scenes.EXTENT)
    a = lib.GpuScene.from_scene(ctx, scene, sh_storage=lib.SH_CODEC32)
    b = lib.GpuScene.from_scene(ctx, scene, sh_storage=lib.SH_CODEC32, order=lib.ORDER_SPATIAL)
    sa, ca = a.sh_codec()
    sb, cb = b.sh_codec()
    np.testing.assert_array_equal(sa, sb)
    np.testing.assert_array_equal(cb, ca[b.order()])
    np.testing.assert_array_equal(a.order(), np.arange(scene.n))
    a.close()
    b.close()


def test_spatial_order_needs_an_owned_copy(lib, ctx):
    scene = scenes.uniform_scene(100, seed=3)
    with pytest.raises(lib.HgError):
        lib.GpuScene.from_scene(ctx, scene, borrow=True, order=lib.ORDER_SPATIAL)
    with pytest.raises(lib.HgError):
        lib.GpuScene.from_scene(ctx, scene, order=7)
