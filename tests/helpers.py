"""Comparison helpers shared by the GPU parity tests (CPU side only)."""
import numpy as np

from oracle import binning as BN
from oracle import composite as C
from oracle import project as P

# Decision-ambiguity bands (relative distance of an oracle decision from its
# threshold below which float32 may legitimately decide the other way):
# support q vs 9, alpha vs 1/255, transmittance vs 1e-4.  Set just above the
# largest margins of the decisions the GPU actually took differently over
# every image comparison of the parity tests (q 3.05e-5, alpha 2.54e-5; no
# flip needed the transmittance band, which keeps the 1e-5 of the
# comparison protocol).
AMB_Q, AMB_ALPHA, AMB_T = 5e-5, 5e-5, 1e-5
IMG_TOL = 2e-4          # max abs per channel outside ambiguous pixels
AMB_JUMP = 0.02         # bound for a single flipped decision (worst measured 6.0e-3)
AMB_FRACTION = 0.01     # default share of decision-ambiguous pixels; each parity test passes its own
                        # cap, about twice the share it measures


def ambiguous(ref):
    return (ref["m_q"] < AMB_Q) | (ref["m_alpha"] < AMB_ALPHA) | (ref["m_T"] < AMB_T)


def flip_diagnostics(err, terr, ref, done):
    """Margins of the pixels whose GPU value is off by more than IMG_TOL (the
    decisions float32 took differently), and the share of pixels a band of
    each width would mark ambiguous: the data the bars above are set from
    (printed with pytest -s)."""
    bad = done & ((err > IMG_TOL) | (terr > IMG_TOL))
    rows = [(float(ref["m_q"][y, x]), float(ref["m_alpha"][y, x]), float(ref["m_T"][y, x]), float(err[y, x]))
            for y, x in zip(*np.nonzero(bad))]
    shares = {}
    for f in (1e-5, 3e-5, 1e-4, 3e-4, 1e-3):
        a = ((ref["m_q"] < f) | (ref["m_alpha"] < f) | (ref["m_T"] < f)) & done
        shares[f] = float(a.sum()) / max(1, int(done.sum()))
    return {"flipped": len(rows), "flipped_margins_q_alpha_T_err": sorted(rows, key=lambda r: -r[3])[:12],
            "ambiguous_share_by_band": shares}


def compare_image(img, T, ref, mask=None, max_amb=AMB_FRACTION):
    """img [H, W, 3], T [H, W] (GPU) vs oracle render dict.  Returns stats and
    asserts the parity bar: every channel (and T) within IMG_TOL outside the
    decision-ambiguous pixels, at most `max_amb` of the compared pixels
    ambiguous, each within AMB_JUMP."""
    done = ref["done"] if mask is None else (ref["done"] & mask)
    amb = ambiguous(ref) & done
    ok = done & ~amb
    err = np.abs(img.astype(np.float64) - ref["rgb"]).max(axis=2)
    # T may be None (an output without transmittance, e.g. a served image)
    terr = np.zeros_like(err) if T is None else np.abs(T.astype(np.float64) - ref["T"])
    print("parity-diag", flip_diagnostics(err, terr, ref, done))  # shown with pytest -s
    worst = float(err[ok].max()) if ok.any() else 0.0
    worst_t = float(terr[ok].max()) if ok.any() else 0.0
    frac = float(amb.sum()) / max(1, int(done.sum()))
    worst_amb = float(err[amb].max()) if amb.any() else 0.0
    stats = {"max_abs": worst, "max_abs_T": worst_t, "ambiguous": int(amb.sum()), "ambiguous_frac": frac,
             "max_abs_ambiguous": worst_amb, "pixels": int(done.sum())}
    print("image parity", stats)  # shown with pytest -s
    assert worst <= IMG_TOL, stats
    assert worst_t <= IMG_TOL, stats
    assert frac <= max_amb, stats
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
