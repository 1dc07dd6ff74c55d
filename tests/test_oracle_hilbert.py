"""Pins of the oracle's Hilbert curves (Section 3, Listing 1; Section 4.3)."""
import os

import numpy as np
import pytest

from oracle import hilbert

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hilbert_order2.txt")


def test_listing1_order2_hand_trace():
    ref = np.loadtxt(GOLD, dtype=np.int64, comments="#")
    np.testing.assert_array_equal(hilbert.listing1_cells(2), ref)


def test_listing1_order1():
    # step(0) onto (0,0); hilbert(0,+1,1): turn to up, step, turn back, step right, turn down, step
    assert hilbert.listing1_cells(1).tolist() == [[0, 0], [0, 1], [1, 1], [1, 0]]


@pytest.mark.parametrize("a", range(1, 7))
def test_listing1_equals_textbook_index_map(a):
    np.testing.assert_array_equal(hilbert.listing1_cells(a), hilbert.textbook_cells(a))


@pytest.mark.parametrize("a", range(0, 7))
def test_generalized_equals_standard_on_powers_of_two(a):
    n = 1 << a
    g = hilbert.generalized_cells(n, n)
    if a == 0:
        assert g.tolist() == [[0, 0]]
    else:
        np.testing.assert_array_equal(g, hilbert.listing1_cells(a))


def _check_path(c, W, H):
    assert c.shape == (W * H, 2)
    assert c[0].tolist() == [0, 0]
    assert c[:, 0].min() == 0 and c[:, 0].max() == W - 1
    assert c[:, 1].min() == 0 and c[:, 1].max() == H - 1
    assert len({tuple(v) for v in c.tolist()}) == W * H          # bijection onto the grid
    steps = np.abs(np.diff(c, axis=0)).sum(axis=1)
    assert np.all(steps == 1)                                    # consecutive cells share an edge


def test_generalized_bijection_and_adjacency_all_small():
    for W in range(1, 34):
        for H in range(1, 34):
            _check_path(hilbert.generalized_cells(W, H), W, H)


def test_generalized_large_rectangles():
    for W, H in [(2048, 8), (100, 37), (512, 128), (63, 64), (1, 97), (97, 1)]:
        _check_path(hilbert.generalized_cells(W, H), W, H)


def test_generalized_locality():
    """Cells close on the curve are close in the plane: every window of 16
    consecutive cells fits in a small box (a row-major walk of a 64-wide grid
    would not)."""
    c = hilbert.generalized_cells(64, 48)
    for s in range(0, c.shape[0] - 16, 16):
        w = c[s:s + 16]
        assert np.ptp(w[:, 0]) <= 7 and np.ptp(w[:, 1]) <= 7


def test_rank_grid_inverts_cells():
    W, H = 13, 7
    c = hilbert.generalized_cells(W, H)
    r = hilbert.rank_grid(W, H)
    np.testing.assert_array_equal(r[c[:, 0], c[:, 1]], np.arange(W * H))
