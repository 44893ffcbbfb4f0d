"""Spatial storage order of a scene: the gaussians sorted by the 30-bit
Morton code of their means.  Not part of the paper's method (a memory layout
for the front end's bandwidth, Sec. 4.2-4.3); written out here as its plain
definition.

Test infrastructure only (see the package docstring).

Definition, per axis a (x, y, z) over the bounding box [lo_a, hi_a] of the
finite coordinates (a non-finite coordinate counts as lo_a):
  s_a = 1024 / (hi_a - lo_a), or 1 when hi_a = lo_a
  q_a = min(1023, max(0, floor((x_a - lo_a) * s_a)))
with every operation in float32, rounded to nearest; the code has bit
3 b + a equal to bit b of q_a, and the order is ascending code, ties by
index.
"""
from __future__ import annotations

import numpy as np

F32 = np.float32


def quantise(means):
    """[n][3] float32 means -> [n][3] int64 cell coordinates q."""
    m = np.asarray(means, F32)
    q = np.zeros(m.shape, np.int64)
    for a in range(3):
        x = m[:, a]
        fin = np.isfinite(x)
        lo = F32(x[fin].min()) if fin.any() else F32(0)
        hi = F32(x[fin].max()) if fin.any() else F32(0)
        ext = F32(hi - lo)
        s = F32(F32(1024) / ext) if ext > 0 else F32(1)
        with np.errstate(invalid="ignore"):
            t = np.where(fin, F32(x - lo) * s, F32(0)).astype(F32)
        q[:, a] = np.clip(np.floor(t.astype(np.float64)), 0, 1023).astype(np.int64)
    return q


def morton(q):
    """[n][3] cell coordinates (0..1023) -> [n] codes: bit 3 b + a = bit b of q_a."""
    q = np.asarray(q, np.int64)
    code = np.zeros(q.shape[0], np.int64)
    for b in range(10):
        for a in range(3):
            code |= ((q[:, a] >> b) & 1) << (3 * b + a)
    return code


def spatial_order(means):
    """Indices of the gaussians in ascending Morton code, ties by index."""
    return np.argsort(morton(quantise(means)), kind="stable").astype(np.int64)
