"""Loss, Adam and the optimisation loop of the differentiable path, through
the C ABI, against the float64 oracle (oracle.train)."""
import numpy as np
import pytest

from paper_2606_00352_gb300 import scenes
from oracle import train as TR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    return lib.Context(0)


@pytest.mark.parametrize("n", [0, 1, 1000, 2_500_003])
def test_l2_loss_matches_oracle_and_is_deterministic(lib, ctx, n):
    import torch
    g = np.random.default_rng(n)
    rgb = g.uniform(0, 1.2, n).astype(np.float32)
    tgt = g.uniform(0, 1.0, n).astype(np.float32)
    r, t = torch.from_numpy(rgb).cuda(), torch.from_numpy(tgt).cuda()
    loss, dl = lib.l2_loss(ctx, r, t)
    loss2, _ = lib.l2_loss(ctx, r, t)
    torch.cuda.synchronize()
    ref_loss, ref_dl = TR.l2_loss(rgb, tgt)
    assert loss.item() == loss2.item()
    assert abs(loss.item() - ref_loss) <= 1e-6 * max(ref_loss, 1e-30)
    # float32 subtraction: within half an ulp of the exact difference
    np.testing.assert_allclose(dl.cpu().numpy(), ref_dl, rtol=1.2e-7, atol=1e-12)


def test_adam_matches_oracle(lib, ctx):
    import torch
    sc = scenes.cluster_scene(1000, 4, 1.2, seed=3, sigma_range=scenes.CLUSTER_SIGMA, sh_degree=3,
                              extent=scenes.EXTENT)
    params = [torch.from_numpy(np.ascontiguousarray(x)).cuda()
              for x in (sc.means, sc.log_scales, sc.quats, sc.opacity_logits, sc.sh)]
    gs = lib.GpuScene(ctx, *params, sh_degree=3, borrow=True)
    ref_p = [x.cpu().numpy().astype(np.float64) for x in params]
    m = [torch.zeros_like(x) for x in params]
    v = [torch.zeros_like(x) for x in params]
    ref_m = [np.zeros_like(x) for x in ref_p]
    ref_v = [np.zeros_like(x) for x in ref_p]
    lrs = (1e-3, 2e-3, 3e-3, 5e-2, 1e-2)
    g = np.random.default_rng(7)
    for t in range(1, 6):
        grads32 = [g.normal(0, 10.0 ** -k, x.shape).astype(np.float32) for k, x in enumerate(ref_p)]
        grads = [torch.from_numpy(x).cuda() for x in grads32]
        lib.adam_step(gs, grads, m, v, t, lrs, beta1=0.9, beta2=0.999, eps=1e-8)
        for k in range(5):
            ref_p[k], ref_m[k], ref_v[k] = TR.adam_step(ref_p[k], grads32[k], ref_m[k], ref_v[k], t, lrs[k],
                                                       0.9, 0.999, 1e-8)
    torch.cuda.synchronize()
    for k in range(5):
        # float32 moments: a few ulps of the gradient scale sigma per step
        # (entries that cancel towards 0 keep that absolute error)
        sigma = 10.0 ** -k
        np.testing.assert_allclose(m[k].cpu().numpy(), ref_m[k], rtol=2e-6, atol=2e-6 * sigma)
        np.testing.assert_allclose(v[k].cpu().numpy(), ref_v[k], rtol=2e-6, atol=2e-6 * sigma * sigma)
        # the parameter moved by ~lr per step; the update agrees to float32 rounding
        np.testing.assert_allclose(params[k].cpu().numpy(), ref_p[k], rtol=1e-6, atol=lrs[k] * 1e-4)
    gs.close()


def test_adam_rejects_bad_arguments(lib, ctx):
    import torch
    sc = scenes.uniform_scene(10, seed=1)
    params = [torch.from_numpy(np.ascontiguousarray(x)).cuda()
              for x in (sc.means, sc.log_scales, sc.quats, sc.opacity_logits, sc.sh)]
    gs = lib.GpuScene(ctx, *params, sh_degree=0, borrow=True)
    z = [torch.zeros_like(x) for x in params]
    with pytest.raises(lib.HgError):
        lib.adam_step(gs, z, z, z, 0, 1e-3)       # step must be >= 1
    with pytest.raises(lib.HgError):
        lib.adam_step(gs, z, z, z, 1, 1e-3, beta1=1.0)
    gs.close()


def test_optimisation_reduces_the_loss(lib, ctx):
    """Densification-free optimisation towards the render of a perturbed copy
    of the scene (means + N(0, 0.02), opacity logits + N(0, 0.3); scene
    extent 10): render, L2 loss, backward and Adam lower the loss."""
    import torch
    sc = scenes.cluster_scene(20_000, 8, 1.2, seed=4, sigma_range=scenes.CLUSTER_SIGMA, extent=scenes.EXTENT)
    cams = scenes.scene_orbit(8, 256, 144)[:2]
    tgt_scene = scenes.perturbed(sc, mean_sigma=0.02, logit_sigma=0.3)
    tg = lib.GpuScene.from_scene(ctx, tgt_scene)
    target, _ = lib.render(tg, cams, lib.Options(), with_T=False)
    params = [torch.from_numpy(np.ascontiguousarray(x)).cuda()
              for x in (sc.means, sc.log_scales, sc.quats, sc.opacity_logits, sc.sh)]
    tr = lib.Trainer(ctx, params, sc.sh_degree, cams, target, lr=(1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3))
    losses = [float(tr.step().item()) for _ in range(40)]
    assert losses[0] > 0
    assert min(losses[-5:]) < 0.5 * losses[0]
    # the parameters the caller owns are the ones that moved
    assert not np.allclose(params[3].cpu().numpy(), sc.opacity_logits)
    tr.close()
    tg.close()
