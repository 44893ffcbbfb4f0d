"""Per-gaussian projection + SH colour in float64 (Sec. 4.2, the fused
projection front end: view transform, EWA 2-D covariance through the
projection Jacobian, inverse covariance, view direction, SH colour).

The paper defers the formulas to the "standard" front end; the reading here
is the original 3DGS one, which the evaluated models were trained with:

  1. R = rot(q / |q|) for q = (w, x, y, z); S = diag(exp(log_scale));
     Sigma3 = R S S^T R^T.
  2. t = V[:3,:3] mu + V[:3,3]; the gaussian is culled when t_z <= 0.2.
  3. J = [[fx/t_z, 0, -fx tx'/t_z^2], [0, fy/t_z, -fy ty'/t_z^2]] with
     tx' = clamp(t_x/t_z, +-1.3 W/(2 fx)) t_z (same for y).
  4. Sigma2 = J V3 Sigma3 V3^T J^T + 0.3 I (the 3DGS low-pass dilation).
  5. det = ac - b^2 of Sigma2 = [[a, b], [b, c]]; culled when det <= 0;
     conic (A, B, C) = (c, -b, a) / det so q(d) = A dx^2 + 2B dx dy + C dy^2.
  6. lambda = (a+c)/2 + sqrt(max(0.1, ((a+c)/2)^2 - det)); r = ceil(3 sqrt(lambda));
     culled when r = 0.
  7. mean2d = (fx t_x/t_z + cx - 0.5, fy t_y/t_z + cy - 0.5): pixel (i, j)
     has its centre at (i, j).
  8. colour = max(0, SH(normalise(mu - campos)) + 0.5), campos = -V3^T V[:3,3].
  9. opacity = sigmoid(logit).

Depth key (Sec. 4.3: raw IEEE bits of the positive depth, which sort as
unsigned integers).  Reading: the key is the float32 depth evaluated as
(((V20*x + V21*y) + V22*z) + V23) with every operation rounded to float32 and
no fused multiply-add, so that any implementation that follows this order
produces the same 32-bit key and hence the same depth order.
"""
from __future__ import annotations

import numpy as np

from .sh import sh_colour

NEAR = 0.2
JAC_CLAMP = 1.3
DILATION = 0.3
LAMBDA_FLOOR = 0.1
SIGMAS = 3.0


def quat_to_rot(q: np.ndarray) -> np.ndarray:
    """Rotation matrix of unit quaternions (w, x, y, z), [N, 3, 3]."""
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    r = np.empty((q.shape[0], 3, 3), np.float64)
    r[:, 0, 0] = 1 - 2 * (y * y + z * z)
    r[:, 0, 1] = 2 * (x * y - w * z)
    r[:, 0, 2] = 2 * (x * z + w * y)
    r[:, 1, 0] = 2 * (x * y + w * z)
    r[:, 1, 1] = 1 - 2 * (x * x + z * z)
    r[:, 1, 2] = 2 * (y * z - w * x)
    r[:, 2, 0] = 2 * (x * z - w * y)
    r[:, 2, 1] = 2 * (y * z + w * x)
    r[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return r


def depth_key(means_f32: np.ndarray, viewmat_f32: np.ndarray) -> np.ndarray:
    """uint32 key: float32 bits of the camera-space depth in the pinned order."""
    m = np.asarray(means_f32, np.float32)
    v = np.asarray(viewmat_f32, np.float32)
    d = v[2, 0] * m[:, 0]
    d = d + v[2, 1] * m[:, 1]
    d = d + v[2, 2] * m[:, 2]
    d = d + v[2, 3]
    assert d.dtype == np.float32
    return d.view(np.uint32).copy()


def project(scene, cam) -> dict:
    """Project every gaussian of `scene` for camera `cam` (float64).

    Returns a dict of per-gaussian arrays; culled gaussians have
    visible=False and radius=0 (their other fields are meaningless).
    Also returns `ambiguous`: gaussians whose discrete outputs (cull, radius,
    floor of the mean) sit so close to a decision boundary that float32
    evaluation of the same formulas may decide them differently.
    """
    mu = scene.means.astype(np.float64)
    n = mu.shape[0]
    vm = np.asarray(cam.viewmat, np.float64)
    v3, tv = vm[:3, :3], vm[:3, 3]
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    width, height = int(cam.width), int(cam.height)

    t = mu @ v3.T + tv
    tx, ty, tz = t[:, 0], t[:, 1], t[:, 2]
    in_front = tz > NEAR
    tzs = np.where(in_front, tz, 1.0)

    q = scene.quats.astype(np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    rot = quat_to_rot(q)
    s = np.exp(scene.log_scales.astype(np.float64))
    m = rot * s[:, None, :]
    sig3 = m @ np.transpose(m, (0, 2, 1))

    limx = JAC_CLAMP * 0.5 * width / fx
    limy = JAC_CLAMP * 0.5 * height / fy
    txc = np.clip(tx / tzs, -limx, limx) * tzs
    tyc = np.clip(ty / tzs, -limy, limy) * tzs
    jac = np.zeros((n, 2, 3), np.float64)
    jac[:, 0, 0] = fx / tzs
    jac[:, 0, 2] = -fx * txc / (tzs * tzs)
    jac[:, 1, 1] = fy / tzs
    jac[:, 1, 2] = -fy * tyc / (tzs * tzs)
    tm = jac @ v3
    sig2 = tm @ sig3 @ np.transpose(tm, (0, 2, 1))
    a = sig2[:, 0, 0] + DILATION
    b = sig2[:, 0, 1]
    c = sig2[:, 1, 1] + DILATION
    det = a * c - b * b
    det_ok = det > 0.0
    dets = np.where(det_ok, det, 1.0)
    conic = np.stack([c / dets, -b / dets, a / dets], axis=1)
    mid = 0.5 * (a + c)
    lam = mid + np.sqrt(np.maximum(LAMBDA_FLOOR, mid * mid - det))
    r_real = SIGMAS * np.sqrt(np.maximum(lam, 0.0))
    radius = np.ceil(r_real).astype(np.int64)
    visible = in_front & det_ok & (radius > 0)
    radius = np.where(visible, radius, 0)

    mean2d = np.stack([fx * tx / tzs + cx - 0.5, fy * ty / tzs + cy - 0.5], axis=1)

    campos = -v3.T @ tv
    dirs = mu - campos
    dirs = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    rgb, rgb_raw = sh_colour(scene.sh, dirs, scene.sh_degree)
    opacity = 1.0 / (1.0 + np.exp(-scene.opacity_logits.astype(np.float64)))

    frac = np.abs(mean2d - np.round(mean2d))
    amb = (np.abs(tz - NEAR) < 1e-5) | (np.abs(det) < 1e-6 * np.abs(a * c))
    amb |= visible & (np.abs(r_real - np.round(r_real)) < 1e-5 * np.maximum(r_real, 1.0))
    amb |= visible & ((frac[:, 0] < 1e-3) | (frac[:, 1] < 1e-3))

    return {
        "n": n, "width": width, "height": height,
        "visible": visible, "mean2d": mean2d, "cov2d": np.stack([a, b, c], 1),
        "conic": conic, "radius": radius, "r_real": r_real, "depth": tz,
        "depth_key": depth_key(scene.means, cam.viewmat),
        "rgb": rgb, "rgb_raw": rgb_raw, "opacity": opacity,
        "t_cam": t, "jac": jac, "sigma3": sig3, "rot": rot, "scale": s,
        "dirs": dirs, "ambiguous": amb,
    }
