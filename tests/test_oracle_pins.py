"""The oracle pinned to answers that do not come from itself (CPU only).

Pins: brute-force enumeration, the single-row dynamic program, the delta >= Z-1
closed form, the flow/energy identity, and the invariants of Section 1.3 (Eq. 2-4
and Theorem 1.1) checked inside the C code. ``test_planted_mistakes`` compiles the
oracle with one deliberate error at a time and shows that the pins catch it.
"""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

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
    "soft arcs dropped": ("if (alpha > 0) add_arc(g, mode, v, idx3(Y, Z, xq, yq, z), alpha);", ";"),
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
