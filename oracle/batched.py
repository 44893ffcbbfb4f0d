"""The macro-tile / batch decomposition of Sec. 3.1-3.4 in float64, used to
pin the claim that the decomposition does not change the image.

Per macro-tile segment (sorted by (key, id)), the list is cut into batches of
at most B_r gaussians (Sec. 3.1).  Every batch is composited independently
with initial transmittance 1, giving a partial (C_k, T_k) per pixel plus a
flag telling whether the pixel stopped inside the batch.  The partials are
merged front to back by Eq. 1, C = C_0 + T_0 C_1 + T_0 T_1 C_2 + ...

Exact termination across batches (reading).  The paper stops the merge once
prod T_i < eps and checks saturation only per drain batch (Sec. 3.4, 5.3),
which is not the per-pixel 3DGS rule.  Here: with T_acc the transmittance
entering batch k, if batch k stopped locally or T_acc T_k < 1e-4 the global
stop lies inside batch k; then batch k is replayed for that pixel with initial
transmittance T_acc using the per-pixel rule, which reproduces the sequential
result.  When T_acc = 1 (no earlier batch contributed) the local result is
already exact.
"""
from __future__ import annotations

import numpy as np

from .binning import segments, batches
from .composite import alpha_at, composite_block, composite_sequence, T_EPS


def render_batched(proj: dict, macro_w: int, macro_h: int, cap: int, tile: int = 8):
    """Image [H, W, 3], T [H, W] and the number of replays."""
    w, h = proj["width"], proj["height"]
    bw, bh = macro_w * tile, macro_h * tile
    mx = proj["mean2d"][:, 0]
    my = proj["mean2d"][:, 1]
    # binning on the float64 oracle positions (floor is taken in float64)
    x0 = np.floor(mx)
    y0 = np.floor(my)
    seg = segments([(x0.astype(np.float32), y0.astype(np.float32),
                     proj["radius"], proj["depth_key"])], [(w, h)], bw, bh)
    table, first = batches(seg["seg_off"], cap)
    gw = -(-w // bw)
    rgb = np.zeros((h, w, 3))
    tt = np.ones((h, w))
    replays = 0
    for s in range(seg["n_seg"]):
        mxi, myi = s % gw, s // gw
        xs = np.arange(mxi * bw, min((mxi + 1) * bw, w))
        ys = np.arange(myi * bh, min((myi + 1) * bh, h))
        if len(xs) == 0 or len(ys) == 0:
            continue
        px, py = (a.ravel().astype(np.float64) for a in np.meshgrid(xs, ys))
        npx = len(px)
        parts = []
        for b in range(first[s], first[s + 1]):
            _, start, count = table[b]
            ids = seg["ids"][start:start + count]
            q, a = alpha_at(proj, ids, px, py)
            col, tk, st, _ = composite_block(a, q, proj["rgb"][ids])
            parts.append((ids, q, a, col, tk, st))
        c_acc = np.zeros((npx, 3))
        t_acc = np.ones(npx)
        done = np.zeros(npx, bool)
        for ids, q, a, col, tk, st in parts:
            for p in np.nonzero(~done)[0]:
                if st[p] or t_acc[p] * tk[p] < T_EPS:
                    if t_acc[p] == 1.0 and st[p]:
                        # nothing in front of this batch: the local stop is the global one
                        c_acc[p] += col[p]
                        t_acc[p] = tk[p]
                        done[p] = True
                        continue
                    replays += 1
                    c, t, stopped, _ = composite_sequence(a[:, p], q[:, p], proj["rgb"][ids], t_acc[p])
                    c_acc[p] += c
                    t_acc[p] = t
                    done[p] = stopped
                else:
                    c_acc[p] += t_acc[p] * col[p]
                    t_acc[p] *= tk[p]
        iy, ix = py.astype(np.int64), px.astype(np.int64)
        rgb[iy, ix] = c_acc
        tt[iy, ix] = t_acc
    return rgb, tt, replays


def compose(parts):
    """Eq. 1 over a list of (C, T) partials (no termination)."""
    c = np.zeros_like(parts[0][0])
    t = np.ones_like(parts[0][1])
    for ck, tk in parts:
        c = c + t[..., None] * ck
        t = t * tk
    return c, t
