"""Pins of the oracle's narrow-band construction (Section 3.4): the center surface
against exact rational arithmetic and closed forms, the band gather against structural
identities, and a solve on a band that holds whole columns against the full-volume
Dinic solve."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import band
from paper_2601_17026_gb300 import synth


def _exact_center(X, Y, Zi, landmarks):
    out = np.empty((X, Y), dtype=np.int64)
    for x in range(X):
        for y in range(Y):
            hits = [z for (lx, ly, z) in landmarks if lx == x and ly == y]
            if hits:
                out[x, y] = hits[0]
                continue
            num = den = Fraction(0)
            for lx, ly, lz in landmarks:
                w = Fraction(1, (x - lx) ** 2 + (y - ly) ** 2)
                num += w * lz
                den += w
            q = num / den + Fraction(1, 2)
            out[x, y] = q.numerator // q.denominator  # floor
    return np.clip(out, 0, Zi - 1)


@pytest.mark.parametrize("seed", range(6))
def test_center_matches_exact_rational_interpolation(seed):
    rng = np.random.default_rng(seed)
    X, Y, Zi = 9, 7, 40
    L = int(rng.integers(1, 7))
    lm = [(int(rng.integers(0, X)), int(rng.integers(0, Y)), int(rng.integers(0, Zi))) for _ in range(L)]
    np.testing.assert_array_equal(band.band_center(X, Y, Zi, lm), _exact_center(X, Y, Zi, lm))


def test_center_closed_forms():
    # one landmark: its height everywhere; equal heights: that height everywhere
    np.testing.assert_array_equal(band.band_center(6, 5, 30, [(2, 3, 17)]), np.full((6, 5), 17))
    np.testing.assert_array_equal(band.band_center(6, 5, 30, [(0, 0, 9), (5, 4, 9), (3, 1, 9)]), np.full((6, 5), 9))
    # two landmarks on a line: halfway rounds half up, and weights 1 : 1/9 at distances 1 and 3
    c = band.band_center(1, 5, 40, [(0, 0, 10), (0, 4, 21)])
    assert c[0, 2] == 16 and c[0, 1] == 11 and c[0, 0] == 10 and c[0, 4] == 21
    # a column holding two landmarks takes the first one's height
    assert band.band_center(3, 3, 40, [(1, 1, 5), (1, 1, 30), (0, 0, 20)])[1, 1] == 5


def test_band_rows_are_shifted_columns():
    rng = np.random.default_rng(3)
    cost = rng.integers(0, 1000, size=(5, 4, 30)).astype(np.int32)
    lm = [(0, 0, 3), (4, 3, 26), (2, 1, 14)]
    b, c = band.narrow_band(cost, lm, stick=3, band_factor=2, outside_cost=-77)
    half = 6
    assert b.shape == (5, 4, 13)
    np.testing.assert_array_equal(b[:, :, half], np.take_along_axis(cost, c[:, :, None].astype(np.int64), 2)[:, :, 0])
    for x in range(5):
        for y in range(4):
            lo = c[x, y] - half
            inside = [k for k in range(13) if 0 <= lo + k < 30]
            np.testing.assert_array_equal(b[x, y, inside], cost[x, y, [lo + k for k in inside]])
            assert np.all(b[x, y, [k for k in range(13) if k not in inside]] == -77)


def test_wide_band_with_flat_center_reproduces_the_full_solve():
    """With one landmark the center is flat; a band at least as tall as twice the image
    holds every column whole, with outside rows priced out, so its solution mapped back
    is the full-volume solution."""
    spec = synth.scaled_spec(6, 5, 16, 5, stream=9)
    cost = synth.horizon_cost(spec)
    lm = [(0, 0, 7)]
    b, c = band.narrow_band(cost, lm, stick=8, band_factor=2, outside_cost=100000)
    assert np.all(c == 7)
    ref = oracle.solve(cost, 2, 3)
    got = oracle.solve(b, 2, 3)
    np.testing.assert_array_equal(band.band_heights(got.heights, c, 16), ref.heights)
