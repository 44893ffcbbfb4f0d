"""hg_segmented_sort_noalloc: the segmented (depth key, id) sort of the
render path in a variant that allocates nothing, for callers that cannot
allocate device memory where they call it (code inside another allocator's
callback, or a process that must not touch the device heap while other work
is in flight).  Its output must equal the sorted pair list that
hg_render_splats produces for the same pairs, on two calls in a row (the
scratch array keeps the previous call's contents), and the (key, value)
order of any input within its limits: every key equal with the values
reversed at the 524,288-pair cap, 512 segments mixing empty, one-pair and
multi-tile segments, and in-place calls."""
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


def _expected(seg_off, keys, vals):
    """(key, value) order inside each segment, by definition."""
    ko, vo = keys.copy(), vals.copy()
    for s in range(len(seg_off) - 1):
        a, b = int(seg_off[s]), int(seg_off[s + 1])
        o = np.lexsort((vals[a:b], keys[a:b]))
        ko[a:b], vo[a:b] = keys[a:b][o], vals[a:b][o]
    return ko, vo


def _run(lib, seg_off, keys, vals, in_place=False):
    import torch
    dev = torch.device("cuda", 0)
    d_off = torch.from_numpy(seg_off.astype(np.uint32).view(np.int32)).to(dev)
    k = torch.from_numpy(keys.view(np.int32).copy()).to(dev)
    v = torch.from_numpy(vals.view(np.int32).copy()).to(dev)
    ko, vo = (k, v) if in_place else (torch.empty_like(k), torch.empty_like(v))
    st = lib.segmented_sort_noalloc(d_off, k, v, ko, vo)
    assert st == 0, lib.load().hg_last_error()
    torch.cuda.synchronize()
    return ko.cpu().numpy().view(np.uint32), vo.cpu().numpy().view(np.uint32)


def test_noalloc_sort_all_equal_keys_at_the_size_cap(lib):
    """One segment of 524,288 pairs, every key equal, values in descending
    order: the id tie-break alone orders it (linear-time passes, no
    quadratic run fix-up); twice in a row."""
    n = 1 << 19
    seg_off = np.array([0, n], np.uint32)
    keys = np.full(n, 0x40200000, np.uint32)
    vals = np.arange(n, 0, -1, dtype=np.uint32)
    for _ in range(2):
        ko, vo = _run(lib, seg_off, keys, vals)
        assert np.array_equal(ko, keys)
        assert np.array_equal(vo, np.sort(vals))


def test_noalloc_sort_segment_cap_mixed_sizes(lib):
    """512 segments: empty, one-pair, small, and multi-tile (> 8,192 pairs)
    segments side by side, heavy key ties, values in arbitrary order; then
    the same call in place."""
    g = np.random.default_rng(17)
    sizes = g.integers(0, 400, 512)
    sizes[::7] = 0
    sizes[3::11] = 1
    sizes[[5, 100, 300]] = [30000, 20000, 8193]
    sizes = sizes[:512]
    seg_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint32)
    n = int(seg_off[-1])
    assert n <= 1 << 19
    keys = g.integers(0, 64, n).astype(np.uint32) * np.uint32(0x01010101)
    vals = g.permutation(1 << 22)[:n].astype(np.uint32)
    want_k, want_v = _expected(seg_off, keys, vals)
    for in_place in (False, True):
        ko, vo = _run(lib, seg_off, keys, vals, in_place=in_place)
        assert np.array_equal(ko, want_k), in_place
        assert np.array_equal(vo, want_v), in_place


def test_noalloc_sort_rejects_overlap_and_capture(lib):
    import torch
    dev = torch.device("cuda", 0)
    n = 4096
    off = torch.tensor([0, n], dtype=torch.int32, device=dev)
    buf = torch.zeros(2 * n, dtype=torch.int32, device=dev)
    k, v = buf[:n], buf[n:]
    other = torch.zeros(2 * n, dtype=torch.int32, device=dev)
    # keys_out overlapping vals_in (shifted by half a buffer)
    assert lib.segmented_sort_noalloc(off, k, v, buf[n // 2:n // 2 + n], other[:n]) == -1
    assert b"overlapping" in lib.load().hg_last_error()
    # a capturing stream: rejected before anything is enqueued
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    x = torch.zeros(1, device=dev)
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
            x.add_(1.0)
            status = lib.segmented_sort_noalloc(off, k, v, other[:n], other[n:])
    assert status == -1
    assert b"capturing" in lib.load().hg_last_error()
