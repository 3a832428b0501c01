"""The oracle pinned to answers that do not come from itself (CPU only).

Pins: brute-force enumeration, the single-row dynamic program, the delta >= Z-1
closed form, the flow/energy identity, the invariants of Section 1.3 (Eq. 2-4
and Theorem 1.1) checked inside the C code, and a library max-flow (scipy's
Edmonds-Karp) on the same literal graph. ``test_planted_mistakes`` compiles the
oracle with one deliberate error at a time and shows that the pins catch it.
"""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import certificate
import oracle
import pins
from paper_2601_17026_gb300 import synth


def _rand_cost(rng, X, Y, Z, lo=-20, hi=40):
    return rng.integers(lo, hi + 1, size=(X, Y, Z)).astype(np.int32)


TINY = [(1, 1, 5), (2, 3, 4), (3, 2, 4), (1, 6, 4), (6, 1, 4), (2, 2, 5), (3, 2, 3), (2, 3, 5)]


def _check_against_brute(cost, delta, alpha, lib=None):
    res = oracle.solve(cost, delta, alpha, check=lib is None, lib=lib)
    emin, hmin, opt = pins.brute_force(cost, delta, alpha)
    # the lattice property: the componentwise minimum of optimal surfaces is optimal
    assert pins.feasible(hmin, delta)
    assert pins.energy(cost, hmin, alpha) == emin
    np.testing.assert_array_equal(res.heights, hmin)
    assert res.flow == emin + pins.identity_offset(cost)


@pytest.mark.parametrize("shape", TINY)
@pytest.mark.parametrize("delta,alpha", [(0, 0), (1, 0), (1, 3), (2, 1), (0, 2), (9, 0), (9, 4)])
def test_brute_force(shape, delta, alpha):
    rng = np.random.default_rng(hash((shape, delta, alpha)) % (2**32))
    for _ in range(3):
        _check_against_brute(_rand_cost(rng, *shape), delta, alpha)


def test_brute_force_horizon_like():
    """Costs of the horizon kind (large away from a minimum, small near it)."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        X, Y, Z = 2, 3, 5
        h = rng.integers(0, Z, size=(X, Y))
        z = np.arange(Z)[None, None, :]
        cost = (np.minimum(100, 30 * np.abs(z - h[:, :, None])) + rng.integers(0, 25, (X, Y, Z))).astype(np.int32)
        _check_against_brute(cost, int(rng.integers(0, 3)), int(rng.integers(0, 8)))


@pytest.mark.parametrize("orient", ["x_row", "y_row"])
def test_row_dp(orient):
    rng = np.random.default_rng(11 if orient == "x_row" else 12)
    for trial in range(25):
        L = int(rng.integers(1, 12))
        Z = int(rng.integers(2, 14))
        shape = (L, 1, Z) if orient == "x_row" else (1, L, Z)
        cost = _rand_cost(rng, *shape, lo=-50, hi=200)
        delta = int(rng.integers(0, 4))
        alpha = int(rng.integers(0, 30))
        emin, h = pins.row_dp(cost, delta, alpha)
        res = oracle.solve(cost, delta, alpha, check=True)
        np.testing.assert_array_equal(res.heights, h)
        assert res.flow == emin + pins.identity_offset(cost)


def test_closed_form():
    rng = np.random.default_rng(3)
    for X, Y, Z in [(6, 7, 9), (1, 5, 12), (4, 1, 3), (5, 5, 1)]:
        cost = _rand_cost(rng, X, Y, Z, lo=-100, hi=100)
        for delta in (Z - 1, Z, Z + 3):
            res = oracle.solve(cost, max(delta, 0), 0, check=True)
            h = pins.closed_form(cost)
            np.testing.assert_array_equal(res.heights, h)
            assert res.flow == pins.energy(cost, h, 0) + pins.identity_offset(cost)


def test_ties_take_lowest_surface():
    """Equal costs everywhere: every surface with equal heights ties; the minimal cut
    is the lowest surface (all zeros)."""
    cost = np.full((3, 4, 6), 7, dtype=np.int32)
    for delta, alpha in [(0, 0), (2, 5), (5, 0)]:
        res = oracle.solve(cost, delta, alpha, check=True)
        assert np.all(res.heights == 0)


def test_small_workload_identity_and_invariants():
    v = synth.small_volume()
    res = oracle.solve(v.cost, v.delta, v.alpha, check=True)
    e, ok = oracle.energy(v.cost, res.heights, v.delta, v.alpha)
    assert ok
    assert e == pins.energy(v.cost, res.heights, v.alpha)
    assert res.flow == e + pins.identity_offset(v.cost)
    assert oracle.cut_capacity(v.cost, res.heights, v.delta, v.alpha) == res.flow


def test_cut_capacity_matches_identity_on_random_surfaces():
    """Eq. 6 counted arc by arc equals E(h) + K for any feasible h, and flags infeasible h."""
    rng = np.random.default_rng(8)
    for _ in range(30):
        X, Y, Z = 3, 4, 7
        cost = _rand_cost(rng, X, Y, Z)
        delta, alpha = int(rng.integers(0, 3)), int(rng.integers(0, 5))
        h = rng.integers(0, Z, size=(X, Y))
        cap = oracle.cut_capacity(cost, h, delta, alpha)
        if pins.feasible(h, delta):
            assert cap == pins.energy(cost, h, alpha) + pins.identity_offset(cost)
        else:
            assert cap == -1


def test_random_invariants_medium():
    rng = np.random.default_rng(21)
    for X, Y, Z, d, a in [(9, 11, 17, 2, 0), (10, 7, 20, 3, 5), (12, 12, 8, 1, 2)]:
        cost = _rand_cost(rng, X, Y, Z, lo=-300, hi=300)
        res = oracle.solve(cost, d, a, check=True)
        e, ok = oracle.energy(cost, res.heights, d, a)
        assert ok and res.flow == e + pins.identity_offset(cost)


# --------------------------------------------------------------------------------------
# Planted mistakes: each mutant of the oracle source must fail at least one pin.
# --------------------------------------------------------------------------------------

MUTANTS = {
    "bottom offset dropped": ("w -= 1 + bottom_sum;", "w -= bottom_sum;"),
    "source arc sign": ("if (w < 0) add_arc(g, mode, s, v, -w);", "if (w < 0) add_arc(g, mode, s, v, w + 2 * -w - 1);"),
    "hard arc lands at z": ("add_arc(g, mode, v, idx3(Y, Z, xq, yq, zq), ORC_INF);",
                            "add_arc(g, mode, v, idx3(Y, Z, xq, yq, z), ORC_INF);"),
    "hard arc off by one": ("const int64_t zq = (z - delta > 0) ? z - delta : 0;",
                            "const int64_t zq = (z - delta - 1 > 0) ? z - delta - 1 : 0;"),
    "x/y transposed": ("return (x * Y + y) * Z + z;", "return (y * Y + x) * Z + z;"),
    "soft arcs dropped": ("if (kcap[l] > 0 && z - l >= 0) add_arc(g, mode, v, idx3(Y, Z, xq, yq, z - l), kcap[l]);",
                          ";"),
    "down arc dropped": ("if (z >= 1) add_arc(g, mode, v, idx3(Y, Z, x, y, z - 1), ORC_INF);", ";"),
    "weight difference reversed": ("(int64_t)c[idx3(Y, Z, x, y, z)] - (int64_t)c[idx3(Y, Z, x, y, z - 1)]",
                                   "(int64_t)c[idx3(Y, Z, x, y, z - 1)] - (int64_t)c[idx3(Y, Z, x, y, z)]"),
    "surface takes lowest node": ("if (in_s[col * Z + z]) h = (int32_t)z;",
                                  "if (in_s[col * Z + z] && h < 0) h = (int32_t)z;"),
}


def _pins_pass(lib) -> bool:
    rng = np.random.default_rng(77)
    try:
        for shape in [(2, 3, 4), (3, 2, 4), (1, 5, 4)]:
            for delta, alpha in [(0, 0), (1, 2), (2, 0)]:
                for _ in range(2):
                    cost = _rand_cost(rng, *shape)
                    res = oracle.solve(cost, delta, alpha, lib=lib)
                    emin, hmin, _ = pins.brute_force(cost, delta, alpha)
                    if not np.array_equal(res.heights, hmin):
                        return False
                    if res.flow != emin + pins.identity_offset(cost):
                        return False
    except RuntimeError:
        return False
    return True


_MUTANT_RUNNER = """
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle, test_oracle_pins as t
sys.exit(0 if t._pins_pass(oracle.load_library({so!r})) else 3)
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes(name, tmp_path):
    """A mutant that crashes (an out-of-range index) counts as caught, so each one runs
    in a child process."""
    src = open(os.path.join(os.path.dirname(oracle.__file__), "pog_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation site for {name!r} not found"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new, 1))  # the first site is the graph construction
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-w", "-o", str(so), str(path)])
    here = os.path.dirname(os.path.abspath(__file__))
    code = _MUTANT_RUNNER.format(root=os.path.dirname(here), tests=here, so=str(so))
    rc = subprocess.run([sys.executable, "-c", code], capture_output=True, timeout=300).returncode
    assert rc != 0, f"pins did not catch: {name}"


def test_unmutated_passes_mutant_pins():
    assert _pins_pass(oracle._load())


# --------------------------------------------------------------------------------------
# The O(N) certificate used at sizes Dinic cannot reach, pinned on states whose status is
# known: the empty preflow (feasible; optimal exactly when no node starts with excess).
# --------------------------------------------------------------------------------------

def _zero_state(cost, delta, alpha):
    """The preflow before any push, in the exported layout, and its value."""
    X, Y, Z = cost.shape
    N = X * Y * Z
    w = pins.node_weights(cost).reshape(-1)
    upper = (np.arange(N) % Z) != 0
    exc = np.where(upper & (w < 0), -w, 0).astype(np.int32)
    snk = np.where(upper & (w > 0), w, 0).astype(np.int32)
    st = dict(excess=exc, sink=snk, fdown=np.zeros(N, np.int32), fhard=np.zeros(4 * N, np.int32),
              gsoft=np.zeros(2 * N, np.int32), in_cut=np.zeros(N, np.int32))
    b = pins.node_weights(cost)[:, :, 0]
    return st, int(b[b > 0].sum())


def _reach_zero_state(cost, delta, alpha, st):
    """Residual reach of the excess nodes in the untouched graph (python BFS, tiny only)."""
    X, Y, Z = cost.shape
    idx = lambda x, y, z: (x * Y + y) * Z + z  # noqa: E731
    seen = set(int(v) for v in np.flatnonzero(st["excess"] > 0))
    todo = list(seen)
    while todo:
        u = todo.pop()
        z, col = u % Z, u // Z
        x, y = col // Y, col % Y
        nxt = [u - 1] if z >= 2 else []
        for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
            xq, yq = x + dx, y + dy
            if 0 <= xq < X and 0 <= yq < Y:
                if z - delta >= 1:
                    nxt.append(idx(xq, yq, z - delta))
                if alpha > 0:
                    nxt.append(idx(xq, yq, z))
        for v in nxt:
            if v not in seen:
                seen.add(v)
                todo.append(v)
    cut = np.zeros(X * Y * Z, np.int32)
    cut[list(seen)] = 1
    return cut


def test_certificate_accepts_optimal_empty_preflow():
    rng = np.random.default_rng(31)
    for _ in range(5):
        cost = np.sort(rng.integers(-50, 50, size=(3, 4, 6)), axis=2).astype(np.int32)  # non-decreasing columns
        st, value = _zero_state(cost, 2, 3)
        heights = np.zeros((3, 4), np.int32)
        assert oracle.solve(cost, 2, 3).flow == value
        assert oracle.certify(cost, 2, 3, st, value, heights) == 0


def test_certificate_rejects_broken_states():
    rng = np.random.default_rng(32)
    cost = rng.integers(-50, 50, size=(3, 4, 6)).astype(np.int32)
    d, a = 1, 4
    st, value = _zero_state(cost, d, a)
    st["in_cut"] = _reach_zero_state(cost, d, a, st)
    top = np.where(st["in_cut"].reshape(3, 4, 6).astype(bool), np.arange(6), 0).max(axis=2).astype(np.int32)
    # feasible but not optimal: everything holds except the cut capacity
    assert oracle.certify(cost, d, a, st, value, top) == 15
    assert oracle.certify(cost, d, a, st, value + 1, top) == 12
    bad = {k: v.copy() for k, v in st.items()}
    bad["excess"][np.flatnonzero(bad["excess"])[0]] += 1
    assert oracle.certify(cost, d, a, bad, value, top) == 11
    bad = {k: v.copy() for k, v in st.items()}
    bad["fdown"][0] = 1  # a bottom node has no down arc
    assert oracle.certify(cost, d, a, bad, value, top) == 10
    bad = {k: v.copy() for k, v in st.items()}
    bad["gsoft"][7] = a + 1
    assert oracle.certify(cost, d, a, bad, value, top) in (10, 11)
    bad = {k: v.copy() for k, v in st.items()}
    off = np.flatnonzero((bad["in_cut"] == 1) & (np.arange(72) % 6 != 0))[0]
    bad["in_cut"][off] = 0
    assert oracle.certify(cost, d, a, bad, value, top) == 13
    wrong = top.copy()
    wrong[0, 0] = (wrong[0, 0] + 1) % 6
    assert oracle.certify(cost, d, a, st, value, wrong) == 14


def _literal_graph_csr(cost, delta, alpha, inf):
    """The s-t graph of Section 1.2 as a scipy CSR capacity matrix (parallel arcs summed):
    node weights w(z) = c(z) - c(z-1), w(x,y,0) = c(x,y,0), w(0,0,0) -= 1 + sum c(.,.,0);
    s->v with -w for w < 0, v->t with w for w > 0; `inf` arcs down the column and to
    (x',y',max(0,z-delta)) for every 4-neighbour; alpha arcs both ways between neighbours."""
    import scipy.sparse as sp

    X, Y, Z = cost.shape
    c = cost.astype(np.int64)
    w = np.diff(c, axis=2, prepend=0)
    w[:, :, 0] = c[:, :, 0]
    w[0, 0, 0] -= 1 + c[:, :, 0].sum()
    idx = lambda x, y, z: (x * Y + y) * Z + z  # noqa: E731
    n = X * Y * Z
    s, t = n, n + 1
    rows, cols, caps = [], [], []

    def arc(a, b, cap):
        rows.append(a)
        cols.append(b)
        caps.append(cap)

    for x in range(X):
        for y in range(Y):
            for z in range(Z):
                v = idx(x, y, z)
                if w[x, y, z] < 0:
                    arc(s, v, -w[x, y, z])
                elif w[x, y, z] > 0:
                    arc(v, t, w[x, y, z])
                if z >= 1:
                    arc(v, idx(x, y, z - 1), inf)
                for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                    x2, y2 = x + dx, y + dy
                    if 0 <= x2 < X and 0 <= y2 < Y:
                        arc(v, idx(x2, y2, max(0, z - delta)), inf)
                        if alpha > 0:
                            arc(v, idx(x2, y2, z), alpha)
    return sp.csr_matrix((np.array(caps, dtype=np.int32), (rows, cols)), shape=(n + 2, n + 2)), s, t


@pytest.mark.parametrize("seed", range(6))
def test_dinic_matches_library_edmonds_karp(seed):
    """The oracle's Dinic against scipy's Edmonds-Karp max-flow on the same literal graph
    (a different algorithm from a library; small costs keep every capacity in int32)."""
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(700 + seed)
    X, Y, Z = (int(v) for v in rng.integers(2, 6, size=3))
    delta, alpha = int(rng.integers(0, Z + 1)), int(rng.integers(0, 6))
    cost = _rand_cost(rng, X, Y, Z, lo=-15, hi=30)
    if cost[:, :, 0].sum() > 1000:
        cost[:, :, 0] //= 4
    inf = 1 << 28
    g, s, t = _literal_graph_csr(cost, delta, alpha, inf)
    ref = csgraph.maximum_flow(g, s, t, method="edmonds_karp").flow_value
    assert ref < inf  # no infinite path from s to t
    assert oracle.solve(cost, delta, alpha).flow == ref


# --- the certificate's accept path on states known to be optimal -----------------------

CERT_CASES = [((3, 4, 6), 0, 0), ((3, 4, 6), 1, 3), ((4, 3, 7), 2, 17), ((5, 5, 8), 2, 0), ((2, 6, 5), 5, 4),
              ((6, 2, 9), 3, 50), ((4, 4, 4), 1, 1)]


@pytest.mark.parametrize("shape,delta,alpha", CERT_CASES)
def test_certificate_accepts_the_oracles_own_optimal_state(shape, delta, alpha):
    """The oracle's final Dinic flow, written in the exported-state layout (bottom layer
    as part of the source), is a maximum preflow whose cut is the minimal one: the
    certificate must accept it, and so must the independent numpy certificate."""
    rng = np.random.default_rng(hash((shape, delta, alpha)) % (2**32))
    nontrivial = 0
    for kind in ("uniform", "horizon"):
        if kind == "uniform":
            cost = rng.integers(-40, 81, size=shape).astype(np.int32)
        else:
            cost = synth.horizon_cost(synth.scaled_spec(*shape, seed=int(rng.integers(1 << 30)), stream=3))
        flow, h, st = oracle.solve_state(cost, delta, alpha)
        ref = oracle.solve(cost, delta, alpha)
        assert flow == ref.flow
        np.testing.assert_array_equal(h, ref.heights)
        assert oracle.certify(cost, delta, alpha, st, flow, h) == 0
        certificate.check(cost, delta, alpha, st, flow, h)
        nontrivial += int(st["excess"].any() and (st["fdown"].any() or st["fhard"].any() or st["gsoft"].any()))
    assert nontrivial >= 1, "the states should carry excess and arc flow"


def test_certificate_rejects_one_word_perturbations_of_an_optimal_state():
    """Each check of the certificate catches a one-word change of an optimal state."""
    cost = synth.horizon_cost(synth.scaled_spec(6, 5, 12, seed=77, stream=5))
    d, a = 2, 5
    flow, h, st = oracle.solve_state(cost, d, a)
    assert oracle.certify(cost, d, a, st, flow, h) == 0
    X, Y, Z = cost.shape
    w = np.diff(cost.astype(np.int64), axis=2, prepend=0).reshape(-1)  # w(z) for z >= 1
    above = np.arange(X * Y * Z) % Z != 0

    def perturbed(key, i, delta_word):
        bad = {k: v.copy() for k, v in st.items()}
        bad[key][i] += delta_word
        return bad

    # 10: a sink residual above the sink arc's capacity
    v = int(np.flatnonzero(above & (w > 0))[0])
    assert oracle.certify(cost, d, a, perturbed("sink", v, int(w[v]) - int(st["sink"][v]) + 1), flow, h) == 10
    # 11: one unit of excess too many
    v = int(np.flatnonzero(above)[0])
    assert oracle.certify(cost, d, a, perturbed("excess", v, 1), flow, h) == 11
    # 12: the reported flow value off by one
    assert oracle.certify(cost, d, a, st, flow + 1, h) == 12
    # 13: one cut mark flipped
    v = int(np.flatnonzero(above & (st["in_cut"] == 1))[0])
    assert oracle.certify(cost, d, a, perturbed("in_cut", v, -1), flow, h) == 13
    # 14: one height off the top of its column's cut
    bad_h = h.copy()
    bad_h.reshape(-1)[0] += 1 if h.reshape(-1)[0] + 1 < Z else -1
    assert oracle.certify(cost, d, a, st, flow, bad_h) == 14
    # 15: a feasible but not maximum preflow, one unit taken back from a saturated sink
    #     arc of a cut node into its excess: every other check still holds
    v = int(np.flatnonzero(above & (st["in_cut"] == 1) & (w > 0) & (st["sink"] < w))[0])
    bad = perturbed("sink", v, 1)
    bad["excess"][v] += 1
    assert oracle.certify(cost, d, a, bad, flow - 1, h) == 15
