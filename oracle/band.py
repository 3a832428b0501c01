"""Narrow-band construction, plain numpy — TEST INFRASTRUCTURE (see the package docstring).

Section 3.4: the structured graph is built around landmark points; in each column it
spans the stick length, times the narrow-band factor, below and above a surface through
the landmarks. The paper gives no formula for that surface; the reading used here is the
inverse-squared-distance average of the landmark heights, rounded half up, in float64
with each operation rounded (no fused multiply-add), summed in landmark order, the
height of the first landmark on a column being that column's center. Band row k of
column (x, y) holds the image cost at height center - half + k, or `outside_cost` when
that height is outside the image.
"""
from __future__ import annotations

import numpy as np


def band_center(X: int, Y: int, Zi: int, landmarks) -> np.ndarray:
    """int32 [X, Y]: the center surface through the landmarks ((x, y, z) rows)."""
    lm = np.asarray(landmarks, dtype=np.int64).reshape(-1, 3)
    xs = np.arange(X, dtype=np.int64)[:, None]
    ys = np.arange(Y, dtype=np.int64)[None, :]
    num = np.zeros((X, Y), dtype=np.float64)
    den = np.zeros((X, Y), dtype=np.float64)
    on = np.full((X, Y), -1, dtype=np.int64)
    for lx, ly, lz in lm:  # in landmark order
        d2 = (xs - lx) ** 2 + (ys - ly) ** 2
        hit = d2 == 0
        on = np.where(hit & (on < 0), lz, on)
        w = 1.0 / np.where(hit, 1, d2).astype(np.float64)
        num = np.where(hit, num, num + w * np.float64(lz))
        den = np.where(hit, den, den + w)
    with np.errstate(invalid="ignore", divide="ignore"):
        avg = np.floor(num / den + 0.5)
    c = np.where(on >= 0, on, np.nan_to_num(avg, nan=0.0).astype(np.int64))
    return np.clip(c, 0, Zi - 1).astype(np.int32)


def narrow_band(cost, landmarks, stick: int, band_factor: int, outside_cost: int):
    """(band int32 [X, Y, 2*half+1], center int32 [X, Y]) of an image cost volume
    [X, Y, Zi]; half = stick * band_factor."""
    cost = np.asarray(cost, dtype=np.int32)
    X, Y, Zi = cost.shape
    half = stick * band_factor
    center = band_center(X, Y, Zi, landmarks)
    z = center[:, :, None].astype(np.int64) - half + np.arange(2 * half + 1)[None, None, :]
    inside = (z >= 0) & (z < Zi)
    vals = np.take_along_axis(cost, np.clip(z, 0, Zi - 1), axis=2)
    return np.where(inside, vals, np.int32(outside_cost)).astype(np.int32), center


def band_heights(h_band, center, half: int) -> np.ndarray:
    """Image heights of a band surface: center - half + h_band."""
    return (np.asarray(center, dtype=np.int64) - half + np.asarray(h_band, dtype=np.int64)).astype(np.int32)
