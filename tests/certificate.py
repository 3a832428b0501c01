"""Host-side optimality certificate for a solved volume (numpy/scipy, independent of the
CUDA code and of the oracle's Dinic).

Given the cost volume and the residual state exported by ``pog_export_state``:

1. the exported preflow is feasible: every arc flow within its capacity (Eq. 2) and the
   excess of every node equals inflow - outflow and is non-negative (Section 2,
   preflow);
2. its value (net flow into t, Eq. 5) equals the reported flow;
3. the reported surface is the cut below it, whose capacity (Eq. 6, computed by the
   caller with the oracle's ``cut_capacity``) must equal the flow — then both are
   optimal by Theorem 1.1;
4. the exported cut is exactly the set reachable in the residual graph from the nodes
   with excess (the minimal minimum cut).

The state describes the graph in which the bottom layer z = 0 is merged into the source
(see include/pog.h): arcs into z = 0 carry no flow and the bottom layer's sink arcs add
the constant sum_{z=0, w>0} w to the flow value.
"""
from __future__ import annotations

import numpy as np

CAP_INF = 0x7FFFFFFF


def _weights(cost):
    c = cost.astype(np.int64)
    w = np.empty_like(c)
    w[:, :, 0] = c[:, :, 0]
    w[:, :, 1:] = c[:, :, 1:] - c[:, :, :-1]
    w[0, 0, 0] -= 1 + int(c[:, :, 0].sum())
    return w


def _arc_lists(X, Y, Z, delta, alpha, st):
    """(tail, head, flow, cap) arrays of every arc of the merged graph, from the state."""
    N = X * Y * Z
    idx = np.arange(N, dtype=np.int64).reshape(X, Y, Z)
    z = np.broadcast_to(np.arange(Z), (X, Y, Z))
    tails, heads, flows, caps = [], [], [], []

    def add(mask, t, h, f, cap):
        tails.append(t[mask])
        heads.append(h[mask])
        flows.append(f[mask].astype(np.int64))
        caps.append(np.broadcast_to(np.asarray(cap, dtype=np.int64), t.shape)[mask])

    fdn = st["fdown"].reshape(X, Y, Z)
    add(z >= 2, idx, idx - 1, fdn, CAP_INF)
    fh = st["fhard"].reshape(4, X, Y, Z)
    shifts = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    for d, (dx, dy) in enumerate(shifts):
        xs = np.arange(X)[:, None, None] + dx
        ys = np.arange(Y)[None, :, None] + dy
        ok = (xs >= 0) & (xs < X) & (ys >= 0) & (ys < Y) & (z - delta >= 1)
        ok = np.broadcast_to(ok, (X, Y, Z))
        head = idx + dx * Y * Z + dy * Z - delta
        add(ok, idx, head, fh[d], CAP_INF)
    if alpha > 0:
        gs = st["gsoft"].reshape(2, X, Y, Z)
        for k, (dx, dy) in enumerate([(1, 0), (0, 1)]):
            ok = np.broadcast_to((np.arange(X)[:, None, None] + dx < X) & (np.arange(Y)[None, :, None] + dy < Y)
                                 & (z >= 1), (X, Y, Z))
            head = idx + dx * Y * Z + dy * Z
            # one arc each way; the net flow g splits as max(g,0) forward, max(-g,0) back
            add(ok, idx, head, np.maximum(gs[k], 0), alpha)
            add(ok, head, idx, np.maximum(-gs[k], 0), alpha)
    return (np.concatenate(tails), np.concatenate(heads), np.concatenate(flows), np.concatenate(caps))


def check(cost, delta, alpha, st, flow, heights):
    """Raise AssertionError unless the exported state certifies (flow, heights)."""
    X, Y, Z = cost.shape
    N = X * Y * Z
    w = _weights(cost)
    z = np.broadcast_to(np.arange(Z), (X, Y, Z)).reshape(-1)
    wf = w.reshape(-1)
    upper = z >= 1
    exc0 = np.where(upper & (wf < 0), -wf, 0)
    snk0 = np.where(upper & (wf > 0), wf, 0)
    snk = st["sink"].astype(np.int64)
    exc = st["excess"].astype(np.int64)
    assert np.all(snk >= 0) and np.all(snk <= snk0), "sink arc over capacity"
    t, h, f, cap = _arc_lists(X, Y, Z, delta, alpha, st)
    assert np.all(f >= 0) and np.all(f <= cap), "arc flow outside [0, capacity]"
    # arcs that do not exist must carry nothing
    assert np.all(st["fdown"].reshape(X, Y, Z)[:, :, :2] == 0)
    net = exc0 - (snk0 - snk)
    net = net - np.bincount(t, weights=f, minlength=N).astype(np.int64)
    net = net + np.bincount(h, weights=f, minlength=N).astype(np.int64)
    assert np.array_equal(net[upper], exc[upper]), "excess != inflow - outflow"
    assert np.all(exc[upper] >= 0), "negative excess"
    bottom = w[:, :, 0]
    value = int((snk0 - snk).sum()) + int(bottom[bottom > 0].sum())
    assert value == flow, f"flow value of the exported preflow {value} != reported {flow}"
    # minimal cut: reachability from excess nodes over residual arcs (bottom = source side)
    res = cap - f  # forward residual
    rt = np.concatenate([t[res > 0], h[f > 0]])
    rh = np.concatenate([h[res > 0], t[f > 0]])
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order

    seeds = np.flatnonzero(upper & (exc > 0))
    src = N  # super source feeding every excess node
    rows = np.concatenate([rt, np.full(seeds.size, src)])
    cols = np.concatenate([rh, seeds])
    graph = sp.csr_matrix((np.ones(rows.size, dtype=np.int8), (rows, cols)), shape=(N + 1, N + 1))
    order = breadth_first_order(graph, src, directed=True, return_predecessors=False)
    reach = np.zeros(N + 1, dtype=bool)
    reach[order] = True
    reach = reach[:N] & upper
    in_cut = st["in_cut"].astype(bool) & upper
    assert np.array_equal(reach, in_cut), "exported cut is not the residual reach of the excess nodes"
    top = np.where(in_cut.reshape(X, Y, Z), np.arange(Z), 0).max(axis=2)
    assert np.array_equal(top, np.asarray(heights).reshape(X, Y)), "heights are not the top of the cut"
