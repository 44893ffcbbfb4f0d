"""Analytic float64 gradient of the forward model (test infrastructure only).

The paper is forward-only and sketches the backward (Sec. 6): the merge of
batch partials becomes a prefix scan and the last contributor becomes
per-(pixel, batch).  What a backward must produce is fixed by the forward
model itself: the derivative of the rendered colour with respect to the
scene parameters.  This module differentiates the oracle's forward model
(``project`` + ``composite``) by the chain rule, in the forward's order:

  pixel:  C = sum_i c_i a_i T_i + T_n bg,   T_{i+1} = T_i (1 - a_i)
          dC/dc_i = a_i T_i,  dC/da_i = c_i T_i - S_i / (1 - a_i),
          S_i = sum_{j>i} c_j a_j T_j + T_n bg   (the colour behind i)
  alpha:  a = o exp(-q/2) (zero derivative where clamped at 0.99),
          q = d^T A d, d = p - mean2d, A = conic
  conic:  A = Sigma2^-1,  dL/dSigma2 = -A G A  (G = dL/dA, symmetric)
  EWA:    Sigma2 = T Sigma3 T^T + 0.3 I, T = J V3, Sigma3 = M M^T, M = R S
  mean2d = (fx tx/tz + cx - 0.5, fy ty/tz + cy - 0.5), t = V3 mu + tv
  colour: c = max(0, sum_k sh_k Y_k(dir) + 0.5), dir = (mu - campos)/|.|
  opacity: o = sigmoid(logit); scale = exp(log_scale); R = rot(q/|q|)

Decisions (support q <= 9, alpha >= 1/255, termination, the 0.99 clamp, the
Jacobian clamp, the colour clamp at 0) are held fixed: their branches carry
zero derivative, and the radius is treated as a constant.

The SH direction derivative uses the real SH written as polynomials in the
unit direction, derived symbolically (sympy) from the same Legendre
definition as ``oracle.sh`` and checked against it in the tests.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
import sympy as sp

from .composite import ALPHA_MAX, ALPHA_MIN, SUPPORT_Q, T_EPS, tile_candidates, _tile_pixels
from .project import JAC_CLAMP


@lru_cache(maxsize=None)
def _sh_poly(degree: int):
    """Real SH (Condon-Shortley phase, k = l*l + l + m) as polynomials in the
    unit direction (x, y, z), and their partial derivatives, as numpy
    functions.  Y_l^m = sqrt(2) K_l^m P_l^|m|(z) {Re, Im}((x + i y)^|m|) /
    sin^|m|(t) * sin^|m|(t): on the unit sphere sin^m(t) cos(m p) =
    Re((x + i y)^m) and P_l^m(z) = (-1)^m (1 - z^2)^{m/2} d^m P_l / dz^m."""
    x, y, z = sp.symbols("x y z", real=True)
    exprs = []
    for l in range(degree + 1):
        pl = sp.legendre(l, z)
        for m in range(-l, l + 1):
            am = abs(m)
            k = sp.sqrt(sp.Rational(2 * l + 1, 4) / sp.pi * sp.factorial(l - am) / sp.factorial(l + am))
            dpl = sp.diff(pl, z, am)
            cplx = sp.expand((x + sp.I * y) ** am)
            if m == 0:
                e = k * dpl
            elif m > 0:
                e = sp.sqrt(2) * k * (-1) ** am * dpl * sp.re(cplx)
            else:
                e = sp.sqrt(2) * k * (-1) ** am * dpl * sp.im(cplx)
            exprs.append(sp.expand(e))
    f = sp.lambdify((x, y, z), exprs, "numpy")
    dfs = [sp.lambdify((x, y, z), [sp.diff(e, v) for e in exprs], "numpy") for v in (x, y, z)]
    return f, dfs


def sh_poly_eval(dirs: np.ndarray, degree: int):
    """Y [N, K] and dY/d(x, y, z) [3, N, K] of the polynomial form."""
    f, dfs = _sh_poly(degree)
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    n = dirs.shape[0]

    def arr(vals):
        return np.stack([np.broadcast_to(np.asarray(v, np.float64), (n,)) for v in vals], axis=1)
    return arr(f(x, y, z)), np.stack([arr(d(x, y, z)) for d in dfs])


def pixel_grads(proj: dict, dl_drgb: np.ndarray, bg=(0.0, 0.0, 0.0), tile: int = 8, tiles=None):
    """Per-gaussian gradients of sum(dl_drgb * C) w.r.t. the projected
    quantities: mean2d [N, 2], conic [N, 3] (A, B, C of q = A dx^2 + 2B dx dy
    + C dy^2), opacity [N], rgb [N, 3].  dl_drgb [H, W, 3].  `tiles` lists
    the tile indices whose pixels carry a non-zero dl_drgb (None: all
    tiles); a tile with dl_drgb = 0 adds exactly zero, so it is skipped."""
    n = proj["n"]
    w, h = proj["width"], proj["height"]
    bg = np.asarray(bg, np.float64)
    g_mean = np.zeros((n, 2))
    g_conic = np.zeros((n, 3))
    g_op = np.zeros(n)
    g_rgb = np.zeros((n, 3))
    gw, gh, off, gid = tile_candidates(proj, tile)
    for t in (range(gw * gh) if tiles is None else tiles):
        ids = gid[off[t]:off[t + 1]]
        if len(ids) == 0:
            continue
        px, py = _tile_pixels(t % gw, t // gw, tile, w, h)
        fx, fy = px.astype(np.float64), py.astype(np.float64)
        m = proj["mean2d"][ids]
        cA, cB, cC = (proj["conic"][ids, k][:, None] for k in range(3))
        dx = fx[None, :] - m[:, 0:1]
        dy = fy[None, :] - m[:, 1:2]
        q = cA * dx * dx + 2.0 * cB * dx * dy + cC * dy * dy
        op = proj["opacity"][ids][:, None]
        raw = op * np.exp(-0.5 * q)
        alpha = np.minimum(ALPHA_MAX, raw)
        contrib = (q <= SUPPORT_Q) & (alpha >= ALPHA_MIN)
        a_eff = np.where(contrib, alpha, 0.0)
        t_after = np.cumprod(1.0 - a_eff, axis=0)
        stop_here = contrib & (t_after < T_EPS)
        stopped = stop_here.any(axis=0)
        nn = len(ids)
        stop = np.where(stopped, np.argmax(stop_here, axis=0), nn)
        t_before = np.vstack([np.ones((1, len(px))), t_after[:-1]])
        keep = contrib & (np.arange(nn)[:, None] < stop[None, :])
        rgb = proj["rgb"][ids]
        wgt = np.where(keep, alpha * t_before, 0.0)               # a_i T_i
        t_fin = np.where(stopped, t_before[np.minimum(stop, nn - 1), np.arange(len(px))], t_after[-1])
        # colour behind i: S_i = total - sum_{j<=i} c_j a_j T_j
        acc = np.cumsum(wgt[:, :, None] * rgb[:, None, :], axis=0)
        total = acc[-1] + t_fin[:, None] * bg[None, :]
        behind = total[None, :, :] - acc
        v = dl_drgb[py, px].astype(np.float64)                     # [P, 3]
        d_alpha = np.where(keep, np.einsum("gpc,pc->gp", rgb[:, None, :] * t_before[:, :, None]
                                           - behind / (1.0 - alpha)[:, :, None], v), 0.0)
        g_rgb[ids] += np.einsum("gp,pc->gc", wgt, v)
        unclamped = keep & (raw < ALPHA_MAX)
        d_raw = np.where(unclamped, d_alpha, 0.0)                   # dL/d(o e^{-q/2})
        e = np.exp(-0.5 * q)
        g_op[ids] += (d_raw * e).sum(axis=1)
        d_q = d_raw * op * e * (-0.5)
        g_conic[ids, 0] += (d_q * dx * dx).sum(axis=1)
        g_conic[ids, 1] += (d_q * 2.0 * dx * dy).sum(axis=1)
        g_conic[ids, 2] += (d_q * dy * dy).sum(axis=1)
        # dq/dmean = -2 A d
        g_mean[ids, 0] += (d_q * -2.0 * (cA * dx + cB * dy)).sum(axis=1)
        g_mean[ids, 1] += (d_q * -2.0 * (cB * dx + cC * dy)).sum(axis=1)
    return {"mean2d": g_mean, "conic": g_conic, "opacity": g_op, "rgb": g_rgb}


def _dquat_rot(q: np.ndarray, g_r: np.ndarray) -> np.ndarray:
    """dL/dq for R(q) of a unit quaternion (w, x, y, z), given dL/dR."""
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    G = g_r
    gw = 2 * (-z * G[:, 0, 1] + y * G[:, 0, 2] + z * G[:, 1, 0] - x * G[:, 1, 2] - y * G[:, 2, 0] + x * G[:, 2, 1])
    gx = 2 * (y * G[:, 0, 1] + z * G[:, 0, 2] + y * G[:, 1, 0] - 2 * x * G[:, 1, 1] - w * G[:, 1, 2]
              + z * G[:, 2, 0] + w * G[:, 2, 1] - 2 * x * G[:, 2, 2])
    gy = 2 * (-2 * y * G[:, 0, 0] + x * G[:, 0, 1] + w * G[:, 0, 2] + x * G[:, 1, 0] + z * G[:, 1, 2]
              - w * G[:, 2, 0] + z * G[:, 2, 1] - 2 * y * G[:, 2, 2])
    gz = 2 * (-2 * z * G[:, 0, 0] - w * G[:, 0, 1] + x * G[:, 0, 2] + w * G[:, 1, 0] - 2 * z * G[:, 1, 1]
              + y * G[:, 1, 2] + x * G[:, 2, 0] + y * G[:, 2, 1])
    return np.stack([gw, gx, gy, gz], axis=1)


def project_grads(scene, cam, proj: dict, g: dict):
    """Chain the projected-quantity gradients back to the scene parameters.
    Returns dict of means [N,3], log_scales [N,3], quats [N,4],
    opacity_logits [N], sh [N,K,3]."""
    n = proj["n"]
    vis = proj["visible"]
    vm = np.asarray(cam.viewmat, np.float64)
    v3 = vm[:3, :3]
    fx, fy = float(cam.fx), float(cam.fy)
    t = proj["t_cam"]
    tx, ty, tz = t[:, 0], t[:, 1], np.where(vis, t[:, 2], 1.0)
    # --- conic -> Sigma2 (symmetric G with the off-diagonal counted once)
    a, b, c = proj["cov2d"][:, 0], proj["cov2d"][:, 1], proj["cov2d"][:, 2]
    A = np.zeros((n, 2, 2))
    A[:, 0, 0], A[:, 0, 1], A[:, 1, 0], A[:, 1, 1] = proj["conic"][:, 0], proj["conic"][:, 1], proj["conic"][:, 1], proj["conic"][:, 2]
    G = np.zeros((n, 2, 2))
    G[:, 0, 0] = g["conic"][:, 0]
    G[:, 0, 1] = G[:, 1, 0] = 0.5 * g["conic"][:, 1]
    G[:, 1, 1] = g["conic"][:, 2]
    g_s2 = -A @ G @ A                                            # dL/dSigma2
    # --- Sigma2 = T Sigma3 T^T + 0.3 I,  T = J V3
    jac = proj["jac"]
    tm = jac @ v3
    sig3 = proj["sigma3"]
    g_s3 = np.transpose(tm, (0, 2, 1)) @ g_s2 @ tm
    g_tm = 2.0 * g_s2 @ tm @ sig3
    g_j = g_tm @ v3.T
    # --- J(t): clamped x/z, y/z carry no derivative through the clamp
    limx = JAC_CLAMP * 0.5 * cam.width / fx
    limy = JAC_CLAMP * 0.5 * cam.height / fy
    ux, uy = tx / tz, ty / tz
    cx_ok = (ux > -limx) & (ux < limx)
    cy_ok = (uy > -limy) & (uy < limy)
    uxc, uyc = np.clip(ux, -limx, limx), np.clip(uy, -limy, limy)
    g_t = np.zeros((n, 3))
    # J00 = fx/tz, J11 = fy/tz
    g_t[:, 2] += g_j[:, 0, 0] * (-fx / tz ** 2) + g_j[:, 1, 1] * (-fy / tz ** 2)
    # J02 = -fx ux_c / tz with ux_c = clamp(tx/tz)
    g_t[:, 0] += np.where(cx_ok, g_j[:, 0, 2] * (-fx / tz ** 2), 0.0)
    g_t[:, 2] += np.where(cx_ok, g_j[:, 0, 2] * (2 * fx * tx / tz ** 3), g_j[:, 0, 2] * (fx * uxc / tz ** 2))
    g_t[:, 1] += np.where(cy_ok, g_j[:, 1, 2] * (-fy / tz ** 2), 0.0)
    g_t[:, 2] += np.where(cy_ok, g_j[:, 1, 2] * (2 * fy * ty / tz ** 3), g_j[:, 1, 2] * (fy * uyc / tz ** 2))
    # --- mean2d
    g_t[:, 0] += g["mean2d"][:, 0] * fx / tz
    g_t[:, 1] += g["mean2d"][:, 1] * fy / tz
    g_t[:, 2] += -g["mean2d"][:, 0] * fx * tx / tz ** 2 - g["mean2d"][:, 1] * fy * ty / tz ** 2
    g_means = g_t @ v3
    # --- Sigma3 = M M^T, M = R diag(s)
    rot, s = proj["rot"], proj["scale"]
    m = rot * s[:, None, :]
    g_m = 2.0 * g_s3 @ m
    g_s = np.einsum("nij,nij->nj", g_m, rot)
    g_rot = g_m * s[:, None, :]
    g_logs = g_s * s
    qraw = scene.quats.astype(np.float64)
    qn = np.linalg.norm(qraw, axis=1, keepdims=True)
    qhat = qraw / qn
    g_qhat = _dquat_rot(qhat, g_rot)
    g_quat = (g_qhat - qhat * (qhat * g_qhat).sum(axis=1, keepdims=True)) / qn
    # --- opacity
    o = proj["opacity"]
    g_logit = g["opacity"] * o * (1.0 - o)
    # --- colour: SH coefficients and the view direction
    dirs = proj["dirs"]
    y_b, dy_b = sh_poly_eval(dirs, scene.sh_degree)
    g_c = np.where(proj["rgb_raw"] > 0.0, g["rgb"], 0.0)          # [N, 3]
    g_sh = y_b[:, :, None] * g_c[:, None, :]
    shc = scene.sh.astype(np.float64)
    g_dir = np.stack([np.einsum("nk,nkc,nc->n", dy_b[d], shc, g_c) for d in range(3)], axis=1)
    campos = -v3.T @ vm[:3, 3]
    dist = np.linalg.norm(scene.means.astype(np.float64) - campos, axis=1, keepdims=True)
    g_means += (g_dir - dirs * (dirs * g_dir).sum(axis=1, keepdims=True)) / dist
    z = ~vis
    for arr in (g_means, g_logs, g_quat):
        arr[z] = 0.0
    g_logit[z] = 0.0
    g_sh[z] = 0.0
    return {"means": g_means, "log_scales": g_logs, "quats": g_quat, "opacity_logits": g_logit, "sh": g_sh}


def render_grads(scene, cams, dl_drgb_views, bg=(0.0, 0.0, 0.0), tiles_views=None):
    """Gradient of sum_v sum(dl_drgb_v * C_v) over views w.r.t. the scene.
    `tiles_views[v]` (optional) lists the tiles of view v outside which
    dl_drgb_v is zero."""
    from .project import project
    out = None
    for v, (cam, dl) in enumerate(zip(cams, dl_drgb_views)):
        pr = project(scene, cam)
        tl = None if tiles_views is None else tiles_views[v]
        g = project_grads(scene, cam, pr, pixel_grads(pr, dl, bg, tiles=tl))
        if out is None:
            out = g
        else:
            for k in out:
                out[k] = out[k] + g[k]
    return out
