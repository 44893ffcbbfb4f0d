"""Per-pixel compositing in float64 (Sec. 3.4: exact front-to-back alpha
compositing; the 3DGS rules the paper keeps).

For one pixel p and the gaussians ordered by ascending (depth key, id):

  q_i     = d^T Sigma2_i^-1 d,  d = p - mean2d_i           (Sec. 3.5)
  support : q_i <= 9  (the 3-sigma ellipse; reading, see below)
  alpha_i = min(0.99, o_i exp(-q_i / 2)); skipped when alpha_i < 1/255
  T' = T (1 - alpha_i); if T' < 1e-4 the pixel stops and i is excluded,
  else C += c_i alpha_i T and T = T'.          Output C + T bg, and T.

Reading of the support rule: 3DGS evaluates every pixel of every tile its
3-sigma rectangle touches, which makes its image depend on the tile size.  The
paper's claim that partitioning scale does not change the image (Sec. 3.1,
exact compositing) holds only with a per-pixel support test, so the support
is the 3-sigma ellipse q <= 9, which every rect-based binning contains.

``render`` evaluates this definition for every pixel, using the 3-sigma
rectangle only to skip gaussians that provably miss the pixel (q <= 9 implies
|dx| <= 3 sqrt(Sigma_xx) <= radius); ``pixel_brute_force`` evaluates it with
no pruning at all and is what the tests pin ``render`` against.

Per pixel the oracle also reports the smallest relative distance of any
significant discontinuous decision (support, alpha threshold, termination)
from its threshold, so a float32 implementation can be compared outside the
band where float32 and float64 may legitimately decide differently.
"""
from __future__ import annotations

import numpy as np

SUPPORT_Q = 9.0
ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0
T_EPS = 1e-4
# A flipped decision whose estimated effect on the pixel is below this is
# not counted as significant for the margin report.
SIGNIFICANT = 5e-5


def alpha_at(proj: dict, idx: np.ndarray, px: np.ndarray, py: np.ndarray):
    """q and alpha [len(idx), len(px)] of gaussians idx at pixels (px, py)."""
    m = proj["mean2d"][idx]
    cA, cB, cC = (proj["conic"][idx, k][:, None] for k in range(3))
    dx = px[None, :] - m[:, 0:1]
    dy = py[None, :] - m[:, 1:2]
    q = cA * dx * dx + 2.0 * cB * dx * dy + cC * dy * dy
    alpha = np.minimum(ALPHA_MAX, proj["opacity"][idx][:, None] * np.exp(-0.5 * q))
    return q, alpha


def composite_sequence(alpha, q, rgb, t_in: float = 1.0):
    """Plain sequential loop for one pixel (used by the brute-force pin and
    by the replay step of the batched oracle).  alpha, q: [n]; rgb [n, 3].
    Returns (C[3], T, stopped, n_contrib)."""
    c = np.zeros(3)
    t = float(t_in)
    n_c = 0
    for i in range(len(alpha)):
        if q[i] > SUPPORT_Q or alpha[i] < ALPHA_MIN:
            continue
        t_next = t * (1.0 - alpha[i])
        if t_next < T_EPS:
            return c, t, True, n_c
        c = c + rgb[i] * alpha[i] * t
        t = t_next
        n_c += 1
    return c, t, False, n_c


def composite_block(alpha, q, rgb, opacity=None, t_in=None):
    """Vectorised form of ``composite_sequence`` over a block of pixels.

    alpha, q [n, P] for n gaussians in depth order; rgb [n, 3].
    Returns C [P, 3], T [P], stopped [P], margins dict of [P] arrays.
    """
    n, p = alpha.shape
    contrib = (q <= SUPPORT_Q) & (alpha >= ALPHA_MIN)
    a_eff = np.where(contrib, alpha, 0.0)
    t0 = np.ones(p) if t_in is None else np.asarray(t_in, np.float64)
    if n == 0:
        return (np.zeros((p, 3)), t0.copy(), np.zeros(p, bool),
                {k: np.full(p, np.inf) for k in ("q", "alpha", "T")})
    t_after = t0[None, :] * np.cumprod(1.0 - a_eff, axis=0)
    stop_here = contrib & (t_after < T_EPS)
    stopped = stop_here.any(axis=0)
    stop = np.where(stopped, np.argmax(stop_here, axis=0), n)
    t_before = np.vstack([t0[None, :], t_after[:-1]])
    keep = np.arange(n)[:, None] < stop[None, :]
    w = a_eff * t_before * keep
    col = w.T @ rgb
    t_fin = np.where(stopped, t_before[np.minimum(stop, n - 1), np.arange(p)], t_after[-1])

    # decision margins over the gaussians up to and including the stop
    upto = np.arange(n)[:, None] <= stop[None, :]
    cmag = (np.abs(rgb).max(axis=1) + 1.0)[:, None]
    inf = np.inf
    mq = np.full((n, p), inf)
    ma = np.full((n, p), inf)
    mt = np.full((n, p), inf)
    if opacity is not None:
        a9 = np.minimum(ALPHA_MAX, opacity * np.exp(-0.5 * SUPPORT_Q))[:, None]
        sig_q = upto & (a9 >= ALPHA_MIN) & (a9 * t_before * cmag >= SIGNIFICANT)
        mq = np.where(sig_q, np.abs(q - SUPPORT_Q) / SUPPORT_Q, inf)
    sig_a = upto & (q <= SUPPORT_Q) & (ALPHA_MIN * t_before * cmag >= SIGNIFICANT)
    ma = np.where(sig_a, np.abs(alpha - ALPHA_MIN) / ALPHA_MIN, inf)
    sig_t = upto & contrib & (alpha * t_before * cmag >= SIGNIFICANT)
    mt = np.where(sig_t, np.abs(t_after - T_EPS) / T_EPS, inf)
    margins = {"q": mq.min(axis=0), "alpha": ma.min(axis=0), "T": mt.min(axis=0)}
    return col, t_fin, stopped, margins


def _order(proj, idx):
    """Sort gaussian ids by ascending (depth key, id)."""
    idx = np.asarray(idx, np.int64)
    o = np.lexsort((idx, proj["depth_key"][idx]))
    return idx[o]


def tile_candidates(proj: dict, tile: int = 8):
    """Rect pruning: for each tile, ids of visible gaussians whose 3-sigma
    rectangle [floor(mx) - r, floor(mx) + r] x [...] touches it, in
    (depth key, id) order.  Returns (tile_ids, offsets, ids)."""
    w, h = proj["width"], proj["height"]
    gw, gh = -(-w // tile), -(-h // tile)
    vis = np.nonzero(proj["visible"])[0]
    x0 = np.floor(proj["mean2d"][vis, 0]).astype(np.int64)
    y0 = np.floor(proj["mean2d"][vis, 1]).astype(np.int64)
    r = proj["radius"][vis]
    tx0 = np.clip(np.floor_divide(x0 - r, tile), 0, None)
    tx1 = np.clip(np.floor_divide(x0 + r, tile), None, gw - 1)
    ty0 = np.clip(np.floor_divide(y0 - r, tile), 0, None)
    ty1 = np.clip(np.floor_divide(y0 + r, tile), None, gh - 1)
    nx = np.maximum(tx1 - tx0 + 1, 0)
    ny = np.maximum(ty1 - ty0 + 1, 0)
    cnt = nx * ny
    tot = int(cnt.sum())
    gid = np.repeat(vis, cnt)
    k = np.arange(tot) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    nxr = np.repeat(nx, cnt)
    tid = (np.repeat(ty0, cnt) + k // np.maximum(nxr, 1)) * gw + np.repeat(tx0, cnt) + k % np.maximum(nxr, 1)
    o = np.lexsort((gid, proj["depth_key"][gid], tid))
    tid, gid = tid[o], gid[o]
    off = np.searchsorted(tid, np.arange(gw * gh + 1))
    return gw, gh, off, gid


def _tile_pixels(tx, ty, tile, w, h):
    xs = np.arange(tx * tile, min((tx + 1) * tile, w))
    ys = np.arange(ty * tile, min((ty + 1) * tile, h))
    px, py = np.meshgrid(xs, ys)
    return px.ravel(), py.ravel()


def render(proj: dict, bg=(0.0, 0.0, 0.0), tiles=None, tile: int = 8, cand=None):
    """Full image (or only the listed tile indices) in float64.

    `cand` may hold the result of ``tile_candidates(proj, tile)`` computed
    earlier.  Returns dict: rgb [H, W, 3], T [H, W], stopped [H, W], margins
    (q, alpha, T) [H, W] and a boolean `done` mask of evaluated pixels.
    """
    w, h = proj["width"], proj["height"]
    bg = np.asarray(bg, np.float64)
    out = {"rgb": np.zeros((h, w, 3)), "T": np.ones((h, w)),
           "stopped": np.zeros((h, w), bool), "done": np.zeros((h, w), bool)}
    for k in ("q", "alpha", "T"):
        out["m_" + k] = np.full((h, w), np.inf)
    gw, gh, off, gid = tile_candidates(proj, tile) if cand is None else cand
    todo = range(gw * gh) if tiles is None else tiles
    rgb_all, op_all = proj["rgb"], proj["opacity"]
    for t in todo:
        tx, ty = t % gw, t // gw
        px, py = _tile_pixels(tx, ty, tile, w, h)
        ids = gid[off[t]:off[t + 1]]
        q, alpha = alpha_at(proj, ids, px.astype(np.float64), py.astype(np.float64))
        col, tf, st, mg = composite_block(alpha, q, rgb_all[ids], op_all[ids])
        out["rgb"][py, px] = col + tf[:, None] * bg[None, :]
        out["T"][py, px] = tf
        out["stopped"][py, px] = st
        out["done"][py, px] = True
        for k in ("q", "alpha", "T"):
            out["m_" + k][py, px] = mg[k]
    return out


def pixel_work(proj: dict, tiles=None, tile: int = 8, cand=None):
    """Per-pixel work counts of the compositing definition (Sec. 3.4), the
    intrinsic work a per-pixel renderer cannot skip: n_support [H, W], the
    gaussians with q <= 9 at the pixel up to and including the one that
    stops it (all of them when it never stops), and n_contrib [H, W], the
    gaussians blended into it (q <= 9 and alpha >= 1/255, before the stop).
    Pixels of tiles not listed are -1."""
    w, h = proj["width"], proj["height"]
    n_sup = np.full((h, w), -1, np.int64)
    n_con = np.full((h, w), -1, np.int64)
    gw, gh, off, gid = tile_candidates(proj, tile) if cand is None else cand
    todo = range(gw * gh) if tiles is None else tiles
    for t in todo:
        tx, ty = t % gw, t // gw
        px, py = _tile_pixels(tx, ty, tile, w, h)
        ids = gid[off[t]:off[t + 1]]
        n = len(ids)
        if n == 0:
            n_sup[py, px] = 0
            n_con[py, px] = 0
            continue
        q, alpha = alpha_at(proj, ids, px.astype(np.float64), py.astype(np.float64))
        contrib = (q <= SUPPORT_Q) & (alpha >= ALPHA_MIN)
        t_after = np.cumprod(1.0 - np.where(contrib, alpha, 0.0), axis=0)
        stop_here = contrib & (t_after < T_EPS)
        stop = np.where(stop_here.any(axis=0), np.argmax(stop_here, axis=0), n)
        i = np.arange(n)[:, None]
        n_sup[py, px] = ((q <= SUPPORT_Q) & (i <= stop[None, :])).sum(axis=0)
        n_con[py, px] = (contrib & (i < stop[None, :])).sum(axis=0)
    return n_sup, n_con


def pixel_brute_force(proj: dict, px: int, py: int, bg=(0.0, 0.0, 0.0)):
    """One pixel, every visible gaussian considered, explicit loop."""
    vis = np.nonzero(proj["visible"])[0]
    order = _order(proj, vis)
    q, alpha = alpha_at(proj, order, np.array([float(px)]), np.array([float(py)]))
    c, t, stopped, _ = composite_sequence(alpha[:, 0], q[:, 0], proj["rgb"][order])
    return c + t * np.asarray(bg, np.float64), t, stopped
