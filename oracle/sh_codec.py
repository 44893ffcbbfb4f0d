"""32-byte packed SH representation (Sec. 4.2, optional bandwidth
optimisation of the projection front end), as a definition in numpy.

Test infrastructure only (see the package docstring).

The paper states the ingredients (YCoCg-R colour transform, square-root
gamma quantisation with 6 bits luma / 4 bits chroma, per-basis percentile
scaling, 32 bytes per gaussian for degree-3 SH) but not the layout.
Reading, for the 16 bases k of degree-3 SH with RGB coefficients (R, G, B):

  transform  YCoCg-R lifting on reals: Co = R - B, t = B + Co/2,
             Cg = G - t, Y = t + Cg/2 (inverse: t = Y - Cg/2, G = Cg + t,
             B = t - Co/2, R = B + Co)
  scales     s[k][c] = the 99.5th percentile of |value| over the scene's
             gaussians, for basis k and channel c in (Y, Co, Cg); 0 -> 1
  quantise   bases 1..15: x = clamp(v / s, -1, 1); g = sign(x) sqrt(|x|);
             q = round-half-even(g * Qc), Qc = 2^(bits-1) - 1, with
             Y 6 bits, Co 4, Cg 4
             basis 0 (DC, large and off-centre, where square-root steps are
             coarsest): Y as a float16 (16 bits, round to nearest even);
             Co, Cg linear: q = round-half-even(clamp(v / s, -1, 1) * 4095),
             13 bits each
  bits       42 + 15 * 14 = 252 of 256
  layout     the fields in order k = 0..15, c = Y, Co, Cg, each as a
             two's-complement field, packed from bit 0 of word 0 upwards
             into 8 little-endian uint32 words; unused high bits are 0
  decode     bases 1..15: g = q / Qc, v = sign(g) g^2 s; DC: the float16,
             and v = q / 4095 s; then the inverse transform

Encoding arithmetic is float32 with each operation rounded (v / s, sqrt,
g * Qc, round), so an implementation doing the same float32 operations
produces the same codes.
"""
from __future__ import annotations

import numpy as np

F32 = np.float32
N_BASES = 16
BITS = [(16, 13, 13)] + [(6, 4, 4)] * 15
DC_LINEAR_Q = 4095
PERCENTILE = 99.5


def ycocg_r(rgb):
    """[..., 3] RGB -> [..., 3] (Y, Co, Cg), float32 operations."""
    r, g, b = (np.asarray(rgb[..., i], F32) for i in range(3))
    co = r - b
    t = b + co * F32(0.5)
    cg = g - t
    y = t + cg * F32(0.5)
    return np.stack([y, co, cg], -1)


def ycocg_r_inverse(ycc):
    """[..., 3] (Y, Co, Cg) -> RGB, float64."""
    y, co, cg = (np.asarray(ycc[..., i], np.float64) for i in range(3))
    t = y - cg / 2
    g = cg + t
    b = t - co / 2
    r = b + co
    return np.stack([r, g, b], -1)


def scales(sh):
    """Per-basis, per-channel scales [16][3] (float32) of sh [n][16][3]."""
    ycc = ycocg_r(np.asarray(sh, F32))
    s = np.percentile(np.abs(ycc.astype(np.float64)), PERCENTILE, axis=0)
    s = np.where(s > 0, s, 1.0)
    return s.astype(F32)


def quantise(v32, s32, bits):
    q_max = F32(2 ** (bits - 1) - 1)
    x = np.clip(np.asarray(v32, F32) / F32(s32), F32(-1), F32(1))
    g = np.sign(x) * np.sqrt(np.abs(x))
    return np.rint(g * q_max).astype(np.int64)


def quantise_linear(v32, s32):
    x = np.clip(np.asarray(v32, F32) / F32(s32), F32(-1), F32(1))
    return np.rint(x * F32(DC_LINEAR_Q)).astype(np.int64)


def dequantise(q, s, bits):
    q_max = 2 ** (bits - 1) - 1
    g = np.asarray(q, np.float64) / q_max
    return np.sign(g) * g * g * float(s)


def encode(sh, s):
    """sh [n][16][3] float32, s [16][3] -> codes uint32 [n][8]."""
    ycc = ycocg_r(np.asarray(sh, F32))
    n = ycc.shape[0]
    words = np.zeros((n, 8), np.uint64)
    pos = 0
    for k in range(N_BASES):
        for c in range(3):
            b = BITS[k][c]
            if k == 0 and c == 0:
                field = ycc[:, 0, 0].astype(np.float16).view(np.uint16).astype(np.uint64)
            else:
                q = quantise_linear(ycc[:, k, c], s[k][c]) if k == 0 else quantise(ycc[:, k, c], s[k][c], b)
                field = (q & ((1 << b) - 1)).astype(np.uint64)
            w, o = divmod(pos, 32)
            words[:, w] |= (field << np.uint64(o)) & np.uint64(0xFFFFFFFF)
            if o + b > 32:
                words[:, w + 1] |= field >> np.uint64(32 - o)
            pos += b
    return words.astype(np.uint32)


def decode(codes, s):
    """codes uint32 [n][8], s [16][3] -> sh [n][16][3] float64."""
    codes = np.asarray(codes, np.uint64)
    n = codes.shape[0]
    ycc = np.zeros((n, N_BASES, 3))
    pos = 0
    for k in range(N_BASES):
        for c in range(3):
            b = BITS[k][c]
            w, o = divmod(pos, 32)
            field = codes[:, w] >> np.uint64(o)
            if o + b > 32:
                field |= codes[:, w + 1] << np.uint64(32 - o)
            field &= np.uint64((1 << b) - 1)
            if k == 0 and c == 0:
                ycc[:, 0, 0] = field.astype(np.uint16).view(np.float16).astype(np.float64)
                pos += b
                continue
            q = field.astype(np.int64)
            q = np.where(q >= (1 << (b - 1)), q - (1 << b), q)
            ycc[:, k, c] = q / DC_LINEAR_Q * float(s[k][c]) if k == 0 else dequantise(q, s[k][c], b)
            pos += b
    return ycocg_r_inverse(ycc)
