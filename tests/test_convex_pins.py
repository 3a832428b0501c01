"""The oracle's convex pairwise-cost solve pinned to answers that do not come from it (CPU).

The general proper-order graph of Section 1.2 carries convex edge costs over an edge
interval: E(h) = sum_col c(col, h(col)) + sum over 4-neighbour pairs f(|h_p - h_q|). The
oracle builds it literally, one layer of soft arcs per height drop d < delta with the
second difference of f as capacity, and runs Dinic. Pins: enumeration of every surface
on tiny volumes, the single-row dynamic program with f in place of alpha |.|, the
flow/energy identity with the energy computed from its definition, the linear profile
against the alpha solve, and planted mistakes in the layer construction. The O(N)
certificate of a convex-cost state (for volumes too large for Dinic) is pinned by accepting
the oracle's own optimal state and rejecting one-word changes of it, one per check, and a
feasible preflow below the maximum.
"""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import oracle
import pins


def _rand_cost(rng, X, Y, Z, lo=-20, hi=40):
    return rng.integers(lo, hi + 1, size=(X, Y, Z)).astype(np.int32)


def _fv(f):
    return np.concatenate([[0], np.asarray(f, dtype=np.int64)])


TINY = [(1, 1, 5), (2, 3, 4), (3, 2, 4), (1, 6, 4), (6, 1, 4), (2, 2, 6), (2, 3, 5)]


@pytest.mark.parametrize("shape", TINY)
@pytest.mark.parametrize("delta", [0, 1, 2, 3, 5])
def test_brute_force_convex(shape, delta):
    rng = np.random.default_rng(hash((shape, delta, "convex")) % (2**32))
    for name, f in pins.convex_profiles(delta).items():
        for _ in range(2):
            cost = _rand_cost(rng, *shape)
            res = oracle.solve_convex(cost, delta, f, check=True)
            emin, hmin, _ = pins.brute_force_pairwise(cost, delta, _fv(f))
            assert pins.feasible(hmin, delta)
            assert pins.energy_pairwise(cost, hmin, _fv(f)) == emin, name
            np.testing.assert_array_equal(res.heights, hmin, err_msg=name)
            assert res.flow == emin + pins.identity_offset(cost), name


def test_brute_force_convex_random_profiles():
    """Random convex profiles: non-negative second differences drawn at random."""
    rng = np.random.default_rng(12)
    for _ in range(40):
        delta = int(rng.integers(1, 5))
        k = rng.integers(0, 9, size=delta)          # k_0 = f(1), k_d = second differences
        f = np.array([sum(k[d] * (t - d) for d in range(t)) for t in range(1, delta + 1)], dtype=np.int64)
        shape = TINY[int(rng.integers(0, len(TINY)))]
        cost = _rand_cost(rng, *shape)
        res = oracle.solve_convex(cost, delta, f, check=True)
        emin, hmin, _ = pins.brute_force_pairwise(cost, delta, _fv(f))
        np.testing.assert_array_equal(res.heights, hmin)
        assert res.flow == emin + pins.identity_offset(cost)


@pytest.mark.parametrize("orient", ["x_row", "y_row"])
def test_row_dp_convex(orient):
    rng = np.random.default_rng(3 if orient == "x_row" else 4)
    for delta in (1, 2, 4, 7):
        for name, f in pins.convex_profiles(delta).items():
            L, Z = 9, 14
            shape = (1, L, Z) if orient == "x_row" else (L, 1, Z)
            cost = _rand_cost(rng, *shape, lo=-200, hi=200)
            res = oracle.solve_convex(cost, delta, f, check=True)
            emin, h = pins.row_dp_pairwise(cost, delta, _fv(f))
            np.testing.assert_array_equal(res.heights, h, err_msg=f"{delta} {name}")
            assert res.flow == emin + pins.identity_offset(cost)


def test_linear_profile_is_the_alpha_problem():
    rng = np.random.default_rng(8)
    for X, Y, Z, delta, alpha in [(5, 6, 9, 2, 3), (4, 7, 12, 4, 1), (6, 5, 8, 1, 6)]:
        cost = _rand_cost(rng, X, Y, Z, lo=-100, hi=100)
        a = oracle.solve(cost, delta, alpha)
        b = oracle.solve_convex(cost, delta, alpha * np.arange(1, delta + 1))
        assert a.flow == b.flow
        np.testing.assert_array_equal(a.heights, b.heights)


def test_energy_identity_medium():
    rng = np.random.default_rng(9)
    for X, Y, Z, delta in [(9, 11, 17, 3), (10, 7, 20, 5), (12, 12, 10, 2)]:
        for f in pins.convex_profiles(delta).values():
            cost = _rand_cost(rng, X, Y, Z, lo=-300, hi=300)
            res = oracle.solve_convex(cost, delta, f, check=True)
            e, ok = oracle.energy_convex(cost, res.heights, delta, f)
            assert ok and res.flow == e + pins.identity_offset(cost)
            assert e == pins.energy_pairwise(cost, res.heights, _fv(f))


def test_non_convex_profile_is_rejected():
    cost = np.zeros((2, 2, 4), np.int32)
    with pytest.raises(RuntimeError):
        oracle.solve_convex(cost, 3, [4, 5, 5])      # second difference 5 - 10 + 4 < 0
    with pytest.raises(RuntimeError):
        oracle.solve_convex(cost, 2, [-1, 0])        # f(1) < 0
    with pytest.raises(ValueError):
        oracle.solve_convex(cost, 2, [1])            # wrong length


# --------------------------------------------------------------------------------------
# Planted mistakes in the layer construction: each mutant must fail a convex pin.
# --------------------------------------------------------------------------------------

MUTANTS = {
    "layer lands one height too high": ("idx3(Y, Z, xq, yq, z - l), kcap[l]", "idx3(Y, Z, xq, yq, z - l + (l > 1)), kcap[l]"),
    "second difference sign": ("f[d] - 2 * fd + fm", "f[d] - 2 * fd - fm"),
    "first layer doubled": ("kcap[d] = d == 0 ? f[0]", "kcap[d] = d == 0 ? 2 * f[0]"),
    "only the first layer": ("for (int64_t l = 0; l < nk; ++l)", "for (int64_t l = 0; l < nk && l < 1; ++l)"),
    "layers shifted by one": ("kcap[d] = d == 0 ? f[0] : f[d] - 2 * fd + fm;",
                              "kcap[d] = d == 0 ? f[0] : (d + 1 < delta ? f[d + 1] - 2 * f[d] + fd : 0);"),
    "convex energy drops the pair cost": ("if (ad > 0) e += f[ad - 1];", "if (ad > 1) e += f[ad - 2];"),
}


def _convex_pins_pass(lib) -> bool:
    rng = np.random.default_rng(78)
    try:
        for shape in [(2, 3, 5), (3, 2, 5), (1, 5, 6)]:
            for delta in (2, 3):
                for f in pins.convex_profiles(delta).values():
                    cost = _rand_cost(rng, *shape)
                    res = oracle.solve_convex(cost, delta, f, lib=lib)
                    emin, hmin, _ = pins.brute_force_pairwise(cost, delta, _fv(f))
                    if not np.array_equal(res.heights, hmin):
                        return False
                    if res.flow != emin + pins.identity_offset(cost):
                        return False
                    if lib is not None:
                        feas = oracle.ctypes.c_int32(0)
                        fa = np.ascontiguousarray(f, dtype=np.int64)
                        h = np.ascontiguousarray(res.heights, dtype=np.int32)
                        e = lib.oracle_energy_convex(oracle._i32(cost), *cost.shape, delta,
                                                     fa.ctypes.data_as(oracle.ctypes.POINTER(oracle.ctypes.c_int64)),
                                                     oracle._i32(h), oracle.ctypes.byref(feas))
                        if e != emin or not feas.value:
                            return False
    except RuntimeError:
        return False
    return True


_MUTANT_RUNNER = """
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle, test_convex_pins as t
sys.exit(0 if t._convex_pins_pass(oracle.load_library({so!r})) else 3)
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_convex_mistakes(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "pog_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name!r} not found once"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-w", "-o", str(so), str(path)])
    here = os.path.dirname(os.path.abspath(__file__))
    code = _MUTANT_RUNNER.format(root=os.path.dirname(here), tests=here, so=str(so))
    rc = subprocess.run([sys.executable, "-c", code], capture_output=True, timeout=300).returncode
    assert rc != 0, f"pins did not catch: {name}"


def test_unmutated_passes_convex_mutant_pins():
    lib = oracle._load()
    assert _convex_pins_pass(lib)


# --------------------------------------------------------------------------------------
# The literal cut capacity and the O(N) certificate of a convex-cost state.
# --------------------------------------------------------------------------------------

def _kcap(delta, f):
    fv = _fv(f)
    return [int(fv[1])] + [int(fv[d + 1] - 2 * fv[d] + fv[d - 1]) for d in range(1, delta)] if delta else []


def test_cut_capacity_convex_is_energy_plus_offset():
    """Every feasible surface: literal arc count = E(h) + K; infeasible: -1."""
    rng = np.random.default_rng(41)
    for _ in range(60):
        delta = int(rng.integers(0, 5))
        f = list(pins.convex_profiles(delta).values())[int(rng.integers(0, 5))]
        X, Y, Z = int(rng.integers(1, 5)), int(rng.integers(1, 5)), int(rng.integers(2, 8))
        cost = _rand_cost(rng, X, Y, Z)
        h = rng.integers(0, Z, size=(X, Y))
        e, ok = oracle.energy_convex(cost, h, delta, f)
        cut = oracle.cut_capacity_convex(cost, h, delta, f)
        if ok:
            assert cut == e + pins.identity_offset(cost)
            assert e == pins.energy_pairwise(cost, h, _fv(f))
        else:
            assert cut == -1


CERT_CASES = [((2, 3, 5), 2), ((3, 2, 6), 3), ((4, 4, 7), 4), ((1, 5, 8), 1), ((5, 1, 6), 0), ((3, 3, 4), 7),
              ((4, 3, 9), 9)]


@pytest.mark.parametrize("shape,delta", CERT_CASES)
def test_certificate_convex_accepts_the_oracles_optimal_state(shape, delta):
    rng = np.random.default_rng(hash((shape, delta, "cert")) % (2**32))
    for name, f in pins.convex_profiles(delta).items():
        for lo, hi in ((-30, 50), (-400, 400)):
            cost = _rand_cost(rng, *shape, lo=lo, hi=hi)
            flow, h, st = oracle.solve_state_convex(cost, delta, f)
            ref = oracle.solve_convex(cost, delta, f)
            assert flow == ref.flow and np.array_equal(h, ref.heights)
            assert oracle.certify_convex(cost, delta, f, st, flow, h) == 0, name


def _zero_state_convex(cost, delta, f):
    """The convex graph's preflow before any push, its value, its residual reach and the
    heights of that cut (python BFS over the merged graph, tiny volumes only)."""
    X, Y, Z = cost.shape
    N = X * Y * Z
    w = pins.node_weights(cost).reshape(-1)
    upper = (np.arange(N) % Z) != 0
    k = _kcap(delta, f)
    st = {"excess": np.where(upper & (w < 0), -w, 0).astype(np.int32),
          "sink": np.where(upper & (w > 0), w, 0).astype(np.int32),
          "fdown": np.zeros(N, np.int32), "fhard": np.zeros(4 * N, np.int32), "gpair": np.zeros(2 * N, np.int32),
          "flayer": np.zeros(max(4 * (delta - 1), 1) * N, np.int32)}
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
            if not (0 <= xq < X and 0 <= yq < Y):
                continue
            if z - delta >= 1:
                nxt.append(idx(xq, yq, z - delta))
            for d in range(delta):
                if k[d] > 0 and z - d >= 1:
                    nxt.append(idx(xq, yq, z - d))
        for v in nxt:
            if v not in seen:
                seen.add(v)
                todo.append(v)
    st["in_cut"] = np.zeros(N, np.int32)
    st["in_cut"][list(seen)] = 1
    heights = np.where(st["in_cut"].reshape(X, Y, Z) > 0, np.arange(Z), 0).max(axis=2)
    b = pins.node_weights(cost)[:, :, 0]
    return st, int(b[b > 0].sum()), heights


def test_certificate_convex_rejects_one_word_changes():
    """One change per check (10-15) of an optimal state, and a feasible but non-maximum
    preflow (the state before any push) for the last check."""
    rng = np.random.default_rng(52)
    shape, delta = (3, 4, 7), 3
    f = pins.convex_profiles(delta)["quadratic"]
    X, Y, Z = shape
    N = X * Y * Z
    for _ in range(5):
        cost = _rand_cost(rng, *shape)
        flow, h, st = oracle.solve_state_convex(cost, delta, f)
        assert oracle.certify_convex(cost, delta, f, st, flow, h) == 0

        def with_change(key, i, val):
            s2 = {k: v.copy() for k, v in st.items()}
            s2[key][i] = val
            return s2

        v = (1 * Y + 2) * Z + 4                    # an interior node with every layer arc present
        d1 = ((1 - 1) * 4 + 1) * N + v             # its layer-1 arc towards x+1
        assert oracle.certify_convex(cost, delta, f, with_change("flayer", d1, 8 + 1), flow, h) == 10
        assert oracle.certify_convex(cost, delta, f, with_change("flayer", 0 * N + 0, 1), flow, h) == 10  # bottom
        assert oracle.certify_convex(cost, delta, f, with_change("gpair", v, 2 + 1), flow, h) == 10
        assert oracle.certify_convex(cost, delta, f, with_change("excess", v, st["excess"][v] + 1), flow, h) == 11
        assert oracle.certify_convex(cost, delta, f, st, flow + 1, h) == 12
        u = int(np.flatnonzero((np.arange(N) % Z != 0))[3])
        assert oracle.certify_convex(cost, delta, f, with_change("in_cut", u, 1 - st["in_cut"][u]), flow, h) == 13
        h2 = h.copy()
        h2[0, 0] = (h2[0, 0] + 1) % Z
        assert oracle.certify_convex(cost, delta, f, st, flow, h2) == 14
    # the state before any push is a feasible preflow; the certificate rejects it (check 15)
    # whenever its value is below the maximum
    rejected = 0
    for _ in range(6):
        cost = _rand_cost(rng, *shape)
        st0, value0, h0 = _zero_state_convex(cost, delta, f)
        best = oracle.solve_convex(cost, delta, f).flow
        code = oracle.certify_convex(cost, delta, f, st0, value0, h0)
        assert code == (0 if value0 == best else 15)
        rejected += code == 15
    assert rejected > 0
