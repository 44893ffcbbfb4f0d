"""Comparison helpers shared by the GPU parity tests (CPU side only)."""
import numpy as np

from oracle import binning as BN
from oracle import composite as C
from oracle import project as P

# Decision-ambiguity thresholds (relative distance of an oracle decision from
# its threshold below which float32 may legitimately decide the other way):
# support q vs 9, alpha vs 1/255, transmittance vs 1e-4.
AMB_Q, AMB_ALPHA, AMB_T = 1e-4, 5e-4, 1e-3
IMG_TOL = 2e-4          # max abs per channel outside ambiguous pixels
AMB_JUMP = 0.05         # bound for a single flipped decision
AMB_FRACTION = 0.02     # share of pixels allowed to be decision-ambiguous


def ambiguous(ref):
    return (ref["m_q"] < AMB_Q) | (ref["m_alpha"] < AMB_ALPHA) | (ref["m_T"] < AMB_T)


def compare_image(img, T, ref, mask=None):
    """img [H, W, 3], T [H, W] (GPU) vs oracle render dict.  Returns stats and
    asserts the parity bar."""
    done = ref["done"] if mask is None else (ref["done"] & mask)
    amb = ambiguous(ref) & done
    ok = done & ~amb
    err = np.abs(img.astype(np.float64) - ref["rgb"]).max(axis=2)
    terr = np.abs(T.astype(np.float64) - ref["T"])
    worst = float(err[ok].max()) if ok.any() else 0.0
    worst_t = float(terr[ok].max()) if ok.any() else 0.0
    frac = float(amb.sum()) / max(1, int(done.sum()))
    worst_amb = float(err[amb].max()) if amb.any() else 0.0
    stats = {"max_abs": worst, "max_abs_T": worst_t, "ambiguous": int(amb.sum()), "ambiguous_frac": frac,
             "max_abs_ambiguous": worst_amb, "pixels": int(done.sum())}
    print("image parity", stats)  # shown with pytest -s
    assert worst <= IMG_TOL, stats
    assert worst_t <= IMG_TOL, stats
    assert frac <= AMB_FRACTION, stats
    assert worst_amb <= AMB_JUMP, stats
    return stats


def splat_records(projs, splat_dtype):
    """Oracle projections (one per view) -> float32 hg_splat records [V*n]."""
    n = projs[0]["n"]
    rec = np.zeros(len(projs) * n, splat_dtype)
    for v, pr in enumerate(projs):
        s = rec[v * n:(v + 1) * n]
        s["mean2d"] = pr["mean2d"].astype(np.float32)
        s["conic"] = pr["conic"].astype(np.float32)
        s["opacity"] = pr["opacity"].astype(np.float32)
        s["rgb"] = pr["rgb"].astype(np.float32)
        s["depth_key"] = pr["depth_key"]
        s["radius"] = pr["radius"].astype(np.int32)
        s["depth"] = pr["depth"].astype(np.float32)
    return rec


def sample_tiles(width, height, k, seed, tile=8):
    g = np.random.default_rng(seed)
    gw, gh = -(-width // tile), -(-height // tile)
    t = g.choice(gw * gh, size=min(k, gw * gh), replace=False)
    # always include the ragged corner tile
    return sorted(set(int(x) for x in t) | {gw * gh - 1})


def tiles_mask(width, height, tiles, tile=8):
    gw = -(-width // tile)
    m = np.zeros((height, width), bool)
    for t in tiles:
        tx, ty = t % gw, t // gw
        m[ty * tile:(ty + 1) * tile, tx * tile:(tx + 1) * tile] = True
    return m
