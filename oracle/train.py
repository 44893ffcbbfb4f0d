"""Loss and optimiser of the differentiable render path, in float64.

Test infrastructure only (see the package docstring).

* ``l2_loss``   - L = 1/2 sum (C - C*)^2 over views, pixels and channels
                  (reading of the paper's "L2" photometric loss for the
                  differentiable path, Sec. 6), and dL/dC = C - C*.
* ``adam_step`` - one Adam update (Kingma and Ba, 2015; the first-order
                  optimiser 3DGS training uses):
                    m <- b1 m + (1 - b1) g
                    v <- b2 v + (1 - b2) g^2
                    p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
                  with t the 1-based step count.
"""
from __future__ import annotations

import numpy as np


def l2_loss(rgb, target):
    c = np.asarray(rgb, np.float64)
    t = np.asarray(target, np.float64)
    d = c - t
    return 0.5 * float(np.sum(d * d)), d


def adam_step(p, g, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15):
    """Returns the updated (p, m, v) as new float64 arrays."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
