"""Independent reference answers that pin the oracle (pure numpy, no graph, no max-flow).

Each function computes the optimal surface of Eq. 1 by a route that shares nothing
with the oracle's explicit-edge Dinic:

* ``brute_force``   enumerates every surface h: columns -> [0, Z) of a tiny volume,
                    keeps the delta-feasible ones and takes the minimum energy; the
                    answer is the componentwise minimum over the optimal surfaces
                    (optimal surfaces form a lattice because the energy is submodular).
* ``row_dp``        exact dynamic program over a single row of columns (X = 1 or Y = 1).
* ``closed_form``   delta >= Z - 1 with alpha = 0 decouples the columns.
* ``identity_offset`` the constant K with max-flow = E*(h) + K, derived from the cut
                    capacity of the closed set below h (Eq. 6) after the node weights
                    telescope along each column (Section 1.2).
"""
from __future__ import annotations

import itertools

import numpy as np


def energy(cost: np.ndarray, h: np.ndarray, alpha: int) -> int:
    """E(h) = sum_col c(col, h(col)) + alpha * sum over unordered 4-neighbour pairs |h_p - h_q|."""
    X, Y, _ = cost.shape
    h = np.asarray(h, dtype=np.int64).reshape(X, Y)
    e = int(np.take_along_axis(cost.astype(np.int64), h[:, :, None], axis=2).sum())
    e += alpha * int(np.abs(np.diff(h, axis=0)).sum() + np.abs(np.diff(h, axis=1)).sum())
    return e


def feasible(h: np.ndarray, delta: int) -> bool:
    h = np.asarray(h, dtype=np.int64)
    ok_x = np.all(np.abs(np.diff(h, axis=0)) <= delta) if h.shape[0] > 1 else True
    ok_y = np.all(np.abs(np.diff(h, axis=1)) <= delta) if h.shape[1] > 1 else True
    return bool(ok_x and ok_y)


def brute_force(cost: np.ndarray, delta: int, alpha: int):
    """(E_min, h_min, optimal surfaces) by enumeration of all Z^(X*Y) surfaces."""
    X, Y, Z = cost.shape
    n = X * Y
    assert Z ** n <= 200_000, "volume too large for enumeration"
    hs = np.array(list(itertools.product(range(Z), repeat=n)), dtype=np.int64).reshape(-1, X, Y)
    ok = np.ones(len(hs), dtype=bool)
    if X > 1:
        ok &= np.all(np.abs(np.diff(hs, axis=1)) <= delta, axis=(1, 2))
    if Y > 1:
        ok &= np.all(np.abs(np.diff(hs, axis=2)) <= delta, axis=(1, 2))
    hs = hs[ok]
    c = cost.astype(np.int64)
    cols = np.arange(n)
    feat = c.reshape(n, Z)[cols[None, :], hs.reshape(len(hs), n)].sum(axis=1)
    prior = np.zeros(len(hs), dtype=np.int64)
    if X > 1:
        prior += np.abs(np.diff(hs, axis=1)).sum(axis=(1, 2))
    if Y > 1:
        prior += np.abs(np.diff(hs, axis=2)).sum(axis=(1, 2))
    e = feat + alpha * prior
    emin = int(e.min())
    opt = hs[e == emin]
    return emin, opt.min(axis=0), opt


def row_dp(cost: np.ndarray, delta: int, alpha: int):
    """(E_min, h_min) for a single row of columns (X == 1 or Y == 1).

    Forward A_i(h) = c_i(h) + min_{|h-h'| <= delta} [A_{i-1}(h') + alpha |h - h'|], backward
    B_i likewise from the other end; E* = min_h A_last(h), and the lowest optimal height
    of column i is min{h : A_i(h) + B_i(h) - c_i(h) = E*}.
    """
    X, Y, Z = cost.shape
    assert X == 1 or Y == 1
    c = cost.reshape(-1, Z).astype(np.int64)
    L = c.shape[0]
    hh = np.arange(Z)
    dist = np.abs(hh[:, None] - hh[None, :])
    big = np.int64(1) << 60
    trans = np.where(dist <= delta, alpha * dist, big)  # trans[h, h']

    def sweep(rows):
        out = np.empty_like(rows)
        out[0] = rows[0]
        for i in range(1, len(rows)):
            out[i] = rows[i] + np.min(out[i - 1][None, :] + trans, axis=1)
        return out

    A = sweep(c)
    B = sweep(c[::-1])[::-1]
    emin = int(A[-1].min())
    total = A + B - c
    h = np.array([int(np.flatnonzero(total[i] == emin)[0]) for i in range(L)], dtype=np.int64)
    return emin, h.reshape(X, Y)


def closed_form(cost: np.ndarray) -> np.ndarray:
    """delta >= Z-1 and alpha = 0: each column independently takes its lowest argmin."""
    return np.argmin(cost, axis=2).astype(np.int64)  # argmin returns the first (lowest) index


def node_weights(cost: np.ndarray) -> np.ndarray:
    """w(x,y,z) = c(z) - c(z-1) for z > 0, w(x,y,0) = c(x,y,0), w(0,0,0) -= 1 + sum c(.,.,0)."""
    c = cost.astype(np.int64)
    w = np.empty_like(c)
    w[:, :, 0] = c[:, :, 0]
    w[:, :, 1:] = c[:, :, 1:] - c[:, :, :-1]
    w[0, 0, 0] -= 1 + int(c[:, :, 0].sum())
    return w


def identity_offset(cost: np.ndarray) -> int:
    """K such that the cut below a feasible surface h has capacity E(h) + K.

    cut = sum_{v in S} w(v) + sum_{w(v) < 0} (-w(v)) + alpha * (soft arcs cut); the
    weights telescope to sum_col c(col, h) - 1 - sum_col c(col, 0), and the soft arcs
    cut between p and q number |h_p - h_q|.
    """
    w = node_weights(cost)
    return int(-1 - int(cost[:, :, 0].astype(np.int64).sum()) + int(-w[w < 0].sum()))


# --------------------------------------------------------------------------------------
# Convex pairwise costs: E(h) = sum_col c(col, h(col)) + sum over unordered 4-neighbour
# pairs f(|h_p - h_q|), |h_p - h_q| <= delta. `fv` holds f(0..delta) (fv[0] = 0).
# --------------------------------------------------------------------------------------

def energy_pairwise(cost: np.ndarray, h: np.ndarray, fv) -> int:
    X, Y, _ = cost.shape
    h = np.asarray(h, dtype=np.int64).reshape(X, Y)
    fv = np.asarray(fv, dtype=np.int64)
    e = int(np.take_along_axis(cost.astype(np.int64), h[:, :, None], axis=2).sum())
    e += int(fv[np.abs(np.diff(h, axis=0))].sum() + fv[np.abs(np.diff(h, axis=1))].sum())
    return e


def brute_force_pairwise(cost: np.ndarray, delta: int, fv):
    """(E_min, h_min, optimal surfaces) over all Z^(X*Y) surfaces, pairwise cost table fv."""
    X, Y, Z = cost.shape
    n = X * Y
    assert Z ** n <= 200_000, "volume too large for enumeration"
    fv = np.asarray(fv, dtype=np.int64)
    hs = np.array(list(itertools.product(range(Z), repeat=n)), dtype=np.int64).reshape(-1, X, Y)
    ok = np.ones(len(hs), dtype=bool)
    if X > 1:
        ok &= np.all(np.abs(np.diff(hs, axis=1)) <= delta, axis=(1, 2))
    if Y > 1:
        ok &= np.all(np.abs(np.diff(hs, axis=2)) <= delta, axis=(1, 2))
    hs = hs[ok]
    c = cost.astype(np.int64)
    cols = np.arange(n)
    e = c.reshape(n, Z)[cols[None, :], hs.reshape(len(hs), n)].sum(axis=1)
    if X > 1:
        e = e + fv[np.abs(np.diff(hs, axis=1))].sum(axis=(1, 2))
    if Y > 1:
        e = e + fv[np.abs(np.diff(hs, axis=2))].sum(axis=(1, 2))
    emin = int(e.min())
    opt = hs[e == emin]
    return emin, opt.min(axis=0), opt


def row_dp_pairwise(cost: np.ndarray, delta: int, fv):
    """(E_min, h_min) for one row of columns with pairwise cost table fv, by the forward /
    backward recursion of ``row_dp`` with f(|h - h'|) in place of alpha |h - h'|."""
    X, Y, Z = cost.shape
    assert X == 1 or Y == 1
    c = cost.reshape(-1, Z).astype(np.int64)
    L = c.shape[0]
    hh = np.arange(Z)
    dist = np.abs(hh[:, None] - hh[None, :])
    big = np.int64(1) << 60
    fv = np.asarray(fv, dtype=np.int64)
    trans = np.where(dist <= delta, fv[np.minimum(dist, delta)], big)

    def sweep(rows):
        out = np.empty_like(rows)
        out[0] = rows[0]
        for i in range(1, len(rows)):
            out[i] = rows[i] + np.min(out[i - 1][None, :] + trans, axis=1)
        return out

    A = sweep(c)
    B = sweep(c[::-1])[::-1]
    emin = int(A[-1].min())
    total = A + B - c
    h = np.array([int(np.flatnonzero(total[i] == emin)[0]) for i in range(L)], dtype=np.int64)
    return emin, h.reshape(X, Y)


def convex_profiles(delta: int):
    """A few convex f(1..delta) (f(0) = 0) of different shapes: linear, quadratic,
    truncated-linear-then-steep, zero, and a single kink."""
    t = np.arange(1, delta + 1, dtype=np.int64)
    out = {
        "linear3": 3 * t,
        "quadratic": 2 * t * t,
        "hinge": np.maximum(0, t - 1) * 7,
        "zero": 0 * t,
        "quad_plus_linear": t * t + 5 * t,
    }
    return {k: v for k, v in out.items()}
