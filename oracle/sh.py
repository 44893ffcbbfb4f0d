"""Real spherical harmonics up to degree 3 from their textbook definition.

The paper evaluates "degree-3 spherical harmonics" per gaussian in the
projection front end (Sec. 4.2) without giving the basis.  Reading: the basis
of the original 3DGS models the paper renders, i.e. the real SH with the
Condon-Shortley phase, coefficient index k = l*l + l + m (m = -l..l):

    Y_l^0  = K_l^0 P_l^0(cos t)
    Y_l^m  = sqrt(2) K_l^m P_l^m(cos t) cos(m p)      m > 0
    Y_l^-m = sqrt(2) K_l^m P_l^m(cos t) sin(m p)      m > 0
    K_l^m  = sqrt((2l+1)/(4 pi) * (l-m)!/(l+m)!)

with P_l^m the associated Legendre function including (-1)^m
(scipy.special.lpmv) and (t, p) the polar/azimuth angles of the unit
direction.  Colour = max(0, sum_k sh[k] * Y_k(dir) + 0.5) per channel.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import lpmv


def sh_basis(dirs: np.ndarray, degree: int) -> np.ndarray:
    """Y_k(dir) for k < (degree+1)^2; dirs [..., 3] unit vectors (float64)."""
    d = np.asarray(dirs, np.float64)
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    ct = np.clip(z, -1.0, 1.0)
    phi = np.arctan2(y, x)
    out = np.empty(d.shape[:-1] + ((degree + 1) ** 2,), np.float64)
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            k_lm = math.sqrt((2 * l + 1) / (4 * math.pi)
                             * math.factorial(l - am) / math.factorial(l + am))
            p = lpmv(am, l, ct)
            if m == 0:
                v = k_lm * p
            elif m > 0:
                v = math.sqrt(2.0) * k_lm * p * np.cos(am * phi)
            else:
                v = math.sqrt(2.0) * k_lm * p * np.sin(am * phi)
            out[..., l * l + l + m] = v
    return out


def sh_colour(sh: np.ndarray, dirs: np.ndarray, degree: int):
    """Returns (clamped colour, raw colour) [N, 3]; sh [N, K, 3]."""
    basis = sh_basis(dirs, degree)
    raw = np.einsum("nk,nkc->nc", basis, sh.astype(np.float64)) + 0.5
    return np.maximum(raw, 0.0), raw
