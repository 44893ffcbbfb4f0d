"""Pins of the oracle's spatial storage order (oracle.order): the Morton bit
layout, the quantisation over the bounding box, the Z-curve order of a
lattice, stable ties, non-finite coordinates, and the locality it buys."""
import numpy as np

from oracle import order as O

F32 = np.float32


def test_morton_bit_layout():
    q = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [2, 0, 0], [0, 0, 2], [1023, 1023, 1023], [5, 3, 6]])
    # (5, 3, 6): x = 101, y = 011, z = 110; groups (z_b y_b x_b) for b = 2, 1, 0:
    # 101 110 011
    want_536 = 0
    for b in range(3):
        for a, v in enumerate((5, 3, 6)):
            want_536 |= ((v >> b) & 1) << (3 * b + a)
    assert want_536 == 0b101_110_011
    np.testing.assert_array_equal(O.morton(q), [1, 2, 4, 8, 32, (1 << 30) - 1, want_536])


def test_quantisation_over_the_bounding_box():
    m = np.array([[0, 10, -4], [2, 10, 4], [1, 10, 0]], F32)  # y has no extent
    q = O.quantise(m)
    np.testing.assert_array_equal(q[:, 0], [0, 1023, 512])      # lo -> 0, hi -> 1023 (clamped), middle -> 512
    np.testing.assert_array_equal(q[:, 1], [0, 0, 0])
    np.testing.assert_array_equal(q[:, 2], [0, 1023, 512])


def test_lattice_follows_the_z_curve():
    """Points at the corners of a box: the order is x fastest, then y, then z."""
    pts = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], F32)
    g = np.random.default_rng(0)
    sh = g.permutation(8)
    order = O.spatial_order(pts[sh])
    np.testing.assert_array_equal(pts[sh][order], pts)


def test_ties_keep_index_order_and_non_finite_counts_as_lo():
    m = np.array([[1, 1, 1], [0, 0, 0], [1, 1, 1], [np.nan, 0, 0], [0, np.inf, 0], [1, 1, 1]], F32)
    q = O.quantise(m)
    np.testing.assert_array_equal(q[3], [0, 0, 0])
    np.testing.assert_array_equal(q[4], [0, 0, 0])
    order = O.spatial_order(m)
    np.testing.assert_array_equal(np.sort(order), np.arange(6))
    # the three cell-(0,0,0) entries, then the three duplicates of (1,1,1), each group by index
    np.testing.assert_array_equal(order, [1, 3, 4, 0, 2, 5])


def test_order_brings_neighbours_together():
    g = np.random.default_rng(1)
    m = g.uniform(-10, 10, (20000, 3)).astype(F32)
    o = O.spatial_order(m)
    step_sorted = np.linalg.norm(np.diff(m[o], axis=0), axis=1).mean()
    step_random = np.linalg.norm(np.diff(m, axis=0), axis=1).mean()
    assert step_sorted < 0.1 * step_random
