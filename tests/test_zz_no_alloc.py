"""hg_segmented_sort_noalloc: the segmented (depth key, id) sort of the
render path in a variant that allocates nothing, for callers that cannot
allocate device memory where they call it.  Its output must equal the sorted
pair list that hg_render_splats produces for the same pairs, on two calls in
a row (the scratch array keeps the previous call's contents)."""
import numpy as np
import pytest

from paper_2606_00352_gb300 import scenes

pytestmark = pytest.mark.gpu


def _records(n, w, h, n_keys, seed, splat_dtype):
    g = np.random.default_rng(seed)
    keys = np.sort(g.uniform(2.0, 3.0, n_keys)).astype(np.float32).view(np.uint32)
    rec = np.zeros(n, splat_dtype)
    rec["mean2d"] = np.stack([g.uniform(0, w, n), g.uniform(0, h, n)], 1)
    rec["conic"] = (0.5, 0.0, 0.5)
    rec["opacity"] = 0.5
    rec["rgb"] = 0.5
    rec["depth_key"] = keys[g.integers(0, n_keys, n)]
    rec["radius"] = g.integers(1, 4, n)
    rec["depth"] = 2.5
    return rec


def test_noalloc_sort_matches_render_sort(lib):
    import torch
    ctx = lib.Context(0)
    cam = scenes.look_at((3, 0, 0), width=130, height=70)
    rec = _records(90_000, 130, 70, 2500, seed=11, splat_dtype=lib.SPLAT_DTYPE)
    st = lib.State(ctx)
    lib.render_splats(ctx, lib.splats_to_device(rec), len(rec), [cam], lib.Options(), state=st)
    seg_off = st.read(lib.BUF_SEG_OFF)
    keys = st.read(lib.BUF_PAIR_KEYS)
    ids = st.read(lib.BUF_PAIR_IDS)
    assert len(keys) > 100_000 and np.diff(seg_off).max() > 16384  # multi-tile segments
    dev = torch.device("cuda", 0)
    d_off = torch.from_numpy(seg_off.view(np.int32)).to(dev)
    g = np.random.default_rng(5)
    for call in range(2):
        perm = np.arange(len(keys))
        for s in range(len(seg_off) - 1):
            a, b = seg_off[s], seg_off[s + 1]
            perm[a:b] = a + g.permutation(b - a)
        k_in = torch.from_numpy(keys[perm].view(np.int32)).to(dev)
        v_in = torch.from_numpy(ids[perm].view(np.int32)).to(dev)
        k_out = torch.empty_like(k_in)
        v_out = torch.empty_like(v_in)
        assert lib.segmented_sort_noalloc(d_off, k_in, v_in, k_out, v_out) == 0, lib.load().hg_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(k_out.cpu().numpy().view(np.uint32), keys), f"keys differ on call {call}"
        assert np.array_equal(v_out.cpu().numpy().view(np.uint32), ids), f"ids differ on call {call}"


def test_noalloc_sort_rejects_oversized_input(lib):
    import torch
    dev = torch.device("cuda", 0)
    n = (1 << 19) + 1
    off = torch.tensor([0, n], dtype=torch.int32, device=dev)
    k = torch.zeros(n, dtype=torch.int32, device=dev)
    assert lib.segmented_sort_noalloc(off, k, k, k, k) == -1
    assert b"at most 524288 pairs" in lib.load().hg_last_error()
