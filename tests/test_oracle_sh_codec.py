"""Pins of the oracle's 32-byte SH codec (oracle.sh_codec) against what its
definition fixes: the YCoCg-R lifting inverts exactly, the fields fit 32
bytes, the square-root gamma quantiser is within half a step, values on the
quantisation grid survive the round trip, and every field lands in its own
bits."""
import numpy as np

from oracle import sh_codec as SC

F32 = np.float32


def test_fields_fit_32_bytes():
    assert sum(sum(b) for b in SC.BITS) == 252 <= 256
    assert len(SC.BITS) == SC.N_BASES == 16


def test_ycocg_r_inverts():
    g = np.random.default_rng(0)
    rgb = g.normal(0, 0.5, (5000, 3)).astype(F32)
    back = SC.ycocg_r_inverse(SC.ycocg_r(rgb))
    np.testing.assert_allclose(back, rgb, rtol=1e-6, atol=1e-7)
    # grey has no chroma
    grey = np.full((4, 3), 0.3, F32)
    ycc = SC.ycocg_r(grey)
    np.testing.assert_allclose(ycc[:, 1:], 0, atol=1e-7)
    np.testing.assert_allclose(ycc[:, 0], 0.3, rtol=1e-6)


def test_quantiser_is_within_half_a_step_in_the_gamma_domain():
    g = np.random.default_rng(1)
    s = F32(0.7)
    for bits in (4, 6, 8, 10):
        q_max = 2 ** (bits - 1) - 1
        v = g.uniform(-0.7, 0.7, 20000).astype(F32)
        q = SC.quantise(v, s, bits)
        assert np.all(np.abs(q) <= q_max)
        gam = np.sign(v) * np.sqrt(np.abs(v.astype(np.float64)) / 0.7)
        assert np.all(np.abs(gam - q / q_max) <= 0.5 / q_max + 1e-6)
        # beyond the scale the value clamps to +-s
        assert np.all(SC.quantise(np.array([5.0, -5.0], F32), s, bits) == [q_max, -q_max])


def test_grid_values_round_trip():
    """Values on the quantisation grid decode to themselves: v = s (q / Q)^2
    sign(q) for the square-root fields, q / 4095 s for the linear DC chroma,
    float16 values for the DC luma."""
    s = np.full((16, 3), 0.5, F32)
    n = 31
    ycc = np.zeros((2 * n + 1, 16, 3), np.float64)
    for i, q in enumerate(range(-n, n + 1)):
        for k in range(16):
            for c in range(3):
                b = SC.BITS[k][c]
                if k == 0 and c == 0:
                    ycc[i, k, c] = float(np.float16(q / 8.0))
                elif k == 0:
                    ycc[i, k, c] = q * 100 / SC.DC_LINEAR_Q * 0.5
                else:
                    qm = 2 ** (b - 1) - 1
                    qq = int(np.clip(q, -qm, qm))
                    ycc[i, k, c] = np.sign(qq) * (qq / qm) ** 2 * 0.5
    rgb = SC.ycocg_r_inverse(ycc).astype(F32)
    dec = SC.decode(SC.encode(rgb, s), s)
    np.testing.assert_allclose(dec, rgb, atol=2e-6)


def test_dc_fields():
    """DC luma is the float16 of Y; DC chroma is within half a linear step."""
    g = np.random.default_rng(3)
    sh = np.zeros((3000, 16, 3), F32)
    sh[:, 0] = g.normal(1.8, 0.7, (3000, 3))
    s = SC.scales(sh)
    dec_ycc = SC.ycocg_r(SC.decode(SC.encode(sh, s), s).astype(F32))
    ycc = SC.ycocg_r(sh)
    np.testing.assert_allclose(dec_ycc[:, 0, 0], ycc[:, 0, 0].astype(np.float16).astype(np.float32), rtol=2e-6)
    inside = np.abs(ycc[:, 0, 1:]) <= s[0, 1:]
    err = np.abs(dec_ycc[:, 0, 1:] - ycc[:, 0, 1:])
    assert np.all(err[inside] <= (s[0, 1:] / SC.DC_LINEAR_Q * 0.5 + 1e-6)[None].repeat(3000, 0)[inside])


def test_every_field_has_its_own_bits():
    """Setting one field to its largest positive code leaves every other
    field at zero after decoding."""
    s = np.ones((16, 3), F32)
    for k in range(16):
        for c in range(3):
            ycc = np.zeros((1, 16, 3), np.float64)
            ycc[0, k, c] = 1.0
            rgb = SC.ycocg_r_inverse(ycc).astype(F32)
            dec_ycc = SC.ycocg_r(SC.decode(SC.encode(rgb, s), s).astype(F32))
            want = np.zeros((16, 3))
            want[k, c] = 1.0
            np.testing.assert_allclose(dec_ycc[0], want, atol=2e-6)


def test_percentile_scale():
    g = np.random.default_rng(2)
    sh = g.normal(0, 0.2, (20000, 16, 3)).astype(F32)
    s = SC.scales(sh)
    ycc = np.abs(SC.ycocg_r(sh))
    frac = (ycc <= s[None]).mean(axis=0)
    assert np.all(np.abs(frac - 0.995) < 0.002)
