"""Parity of the convex pairwise-cost solve (pog_solve_convex, through the C ABI) with the
CPU oracle's layered literal graph: flow value and surface heights bit for bit
(tolerance 0), on random and layered-horizon volumes, on the stored oracle results of two
mid-size volumes, and, at the benchmark size, against the tuned alpha path (linear
profile) and by the energy identity of the solved surface."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import pins
from paper_2601_17026_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts, skipped there
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2601_17026_gb300 import pog  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "convex.json")
MAX_ROUNDS = 2000   # a solve that does not converge fails fast instead of running on


def gpu_convex(cost_np, delta, f, **opt):
    cost = torch.from_numpy(np.ascontiguousarray(cost_np, dtype=np.int32)).cuda()
    opt.setdefault("max_rounds", MAX_ROUNDS)
    flow, energy, h, stats = pog.pog_solve_convex(cost, delta, f, options=pog.make_options(**opt))
    return flow, energy, h.cpu().numpy(), stats


def assert_convex_parity(cost, delta, f, **opt):
    flow, energy, h, stats = gpu_convex(cost, delta, f, **opt)
    ref = oracle.solve_convex(cost, delta, f)
    assert flow == ref.flow, f"flow {flow} != oracle {ref.flow}"
    np.testing.assert_array_equal(h, ref.heights)
    e, ok = oracle.energy_convex(cost, ref.heights, delta, f)
    assert ok and energy == e
    return stats


SHAPES = [(1, 1, 1), (1, 1, 6), (2, 3, 4), (3, 2, 5), (1, 7, 9), (6, 1, 8), (5, 4, 11), (7, 5, 13)]


@pytest.mark.parametrize("shape", SHAPES)
def test_random_volumes_all_profiles(shape):
    rng = np.random.default_rng(abs(hash(("cvx", shape))) % (2**32))
    Z = shape[2]
    for delta in sorted({0, 1, 2, 3, 5, min(Z + 1, 9)}):
        for name, f in pins.convex_profiles(delta).items():
            cost = rng.integers(-40, 81, size=shape).astype(np.int32)
            assert_convex_parity(cost, delta, f)


def test_random_convex_profiles():
    """Second differences drawn at random, including zero layers between positive ones."""
    rng = np.random.default_rng(33)
    for _ in range(25):
        delta = int(rng.integers(1, 10))
        k = rng.integers(0, 12, size=delta) * (rng.random(delta) < 0.6)
        f = np.array([sum(int(k[d]) * (t - d) for d in range(t)) for t in range(1, delta + 1)], dtype=np.int64)
        shape = (int(rng.integers(1, 9)), int(rng.integers(1, 9)), int(rng.integers(2, 20)))
        cost = rng.integers(-60, 121, size=shape).astype(np.int32)
        assert_convex_parity(cost, delta, f)


def test_matches_brute_force_directly():
    rng = np.random.default_rng(5)
    for _ in range(20):
        cost = rng.integers(-20, 41, size=(2, 3, 5)).astype(np.int32)
        delta = int(rng.integers(1, 5))
        f = pins.convex_profiles(delta)["quadratic"]
        _, _, h, _ = gpu_convex(cost, delta, f)
        emin, hmin, _ = pins.brute_force_pairwise(cost, delta, np.concatenate([[0], f]))
        np.testing.assert_array_equal(h, hmin)


@pytest.mark.parametrize("sweeps", [1, 3, 64])
def test_horizon_volume_matches_oracle(sweeps):
    """32 x 32 x 64 layered-horizon volume, edge interval 10, quadratic cost."""
    cost = synth.convex_cost(32, 32, 64)
    stats = assert_convex_parity(cost, synth.CONVEX_DELTA, synth.convex_profile(), sweeps_per_relabel=sweeps)
    assert stats["rounds"] >= 1 and stats["nodes"] == cost.size


def test_stored_oracle_results():
    with open(GOLDEN) as fh:
        gold = json.load(fh)
    for vol in gold["volumes"]:
        X, Y, Z = vol["shape"]
        cost = synth.convex_cost(X, Y, Z)
        flow, energy, h, _ = gpu_convex(cost, vol["delta"], np.array(vol["f"], dtype=np.int64))
        assert flow == vol["flow"] and energy == vol["energy"]
        h = np.ascontiguousarray(h, dtype=np.int32)
        assert hashlib.sha256(h.tobytes()).hexdigest() == vol["heights_sha256"]
        assert int(h.sum()) == vol["heights_sum"]


def test_edge_cases():
    rng = np.random.default_rng(6)
    f3 = synth.convex_profile(3)
    for shape in [(1, 1, 1), (4, 3, 1), (1, 1, 12), (9, 1, 2), (3, 3, 2)]:
        cost = rng.integers(-50, 51, size=shape).astype(np.int32)
        assert_convex_parity(cost, 3, f3)
    cost = rng.integers(-50, 51, size=(4, 5, 6)).astype(np.int32)
    assert_convex_parity(cost, 0, [])                      # delta 0: flat surfaces only
    assert_convex_parity(cost, 9, synth.convex_profile(9))  # delta >= Z
    assert_convex_parity(cost, 4, [0, 0, 0, 0])            # no soft arcs: hard limit only


def test_linear_profile_equals_alpha_path_full_size():
    """f(t) = 50 t on the benchmark volume equals the tuned alpha solve (bit for bit)."""
    X, Y, Z = synth.CONVEX_SHAPE
    cost_np = synth.convex_cost(X, Y, Z)
    cost = torch.from_numpy(cost_np).cuda()
    delta, alpha = 3, 50
    flow_a, h_a = pog.solve(cost, delta, alpha)
    flow_c, energy_c, h_c, _ = pog.pog_solve_convex(cost, delta, alpha * np.arange(1, delta + 1),
                                                    options=pog.make_options(max_rounds=MAX_ROUNDS))
    assert flow_c == flow_a
    assert torch.equal(h_c, h_a)
    e, ok = oracle.energy(cost_np, h_c.cpu().numpy(), delta, alpha)
    assert ok and energy_c == e


def test_full_size_energy_identity_and_local_optimality():
    """The benchmark workload: the surface is feasible, its energy (from the definition)
    equals flow - K, and no single-column move of +-1 lowers it (a property of every
    optimum)."""
    X, Y, Z = synth.CONVEX_SHAPE
    cost = synth.convex_cost(X, Y, Z)
    f = synth.convex_profile()
    flow, energy, h, stats = gpu_convex(cost, synth.CONVEX_DELTA, f)
    e, ok = oracle.energy_convex(cost, h, synth.CONVEX_DELTA, f)
    assert ok
    assert energy == e == flow - pins.identity_offset(cost)
    rng = np.random.default_rng(7)
    fv = np.concatenate([[0], f])
    for _ in range(200):
        x, y = int(rng.integers(0, X)), int(rng.integers(0, Y))
        for step in (-1, 1):
            h2 = h.copy()
            h2[x, y] += step
            if not (0 <= h2[x, y] < Z) or not pins.feasible(h2[max(0, x - 1):x + 2, max(0, y - 1):y + 2],
                                                            synth.CONVEX_DELTA):
                continue
            e2, ok2 = oracle.energy_convex(cost, h2, synth.CONVEX_DELTA, f)
            assert ok2 and e2 >= e
    assert pins.energy_pairwise(cost, h, fv) == e


def test_full_size_schedule_independence():
    """The minimal cut is unique: two very different sweep schedules on the benchmark volume
    give the same flow and the same surface, bit for bit."""
    X, Y, Z = synth.CONVEX_SHAPE
    cost = synth.convex_cost(X, Y, Z)
    f = synth.convex_profile()
    a = gpu_convex(cost, synth.CONVEX_DELTA, f, sweeps_per_relabel=16)
    b = gpu_convex(cost, synth.CONVEX_DELTA, f, sweeps_per_relabel=200, flags=pog.POG_FLAG_NO_PREPUSH)
    assert a[0] == b[0] and a[1] == b[1]
    np.testing.assert_array_equal(a[2], b[2])


def test_invalid_arguments_and_failures():
    cost = torch.zeros((3, 3, 5), dtype=torch.int32, device="cuda")
    with pytest.raises(pog.PogError) as ei:
        pog.pog_solve_convex(cost, 3, [4, 5, 5])            # second difference < 0
    assert ei.value.status == pog.POG_E_INVALID
    with pytest.raises(pog.PogError) as ei:
        pog.pog_solve_convex(cost, 2, [-1, 0])              # f(1) < 0
    assert ei.value.status == pog.POG_E_INVALID
    with pytest.raises(pog.PogError) as ei:
        pog.pog_solve_convex(cost, 33, np.arange(1, 34))    # delta above the maximum
    assert ei.value.status == pog.POG_E_INVALID
    with pytest.raises(pog.PogError) as ei:
        pog.pog_solve_convex(cost, 2, [1, 1 << 31])         # layer capacity >= 2^30
    assert ei.value.status == pog.POG_E_INVALID
    with pytest.raises(pog.PogError) as ei:
        pog.pog_solve_convex(cost, 2, [1, 4], options=pog.make_options(test_fail_alloc=1))
    assert ei.value.status == pog.POG_E_NOMEM
    big = torch.full((3, 3, 5), 1 << 30, dtype=torch.int32, device="cuda")
    with pytest.raises(pog.PogError) as ei:
        pog.pog_solve_convex(big, 2, [1, 4])
    assert ei.value.status == pog.POG_E_OVERFLOW
    with pytest.raises(pog.PogError):
        pog.pog_solve_convex(cost, 2, [1, 4], heights=torch.zeros((3, 4), dtype=torch.int32, device="cuda"))
    # the device is still usable after every failure above
    rng = np.random.default_rng(1)
    assert_convex_parity(rng.integers(-30, 31, size=(4, 4, 7)).astype(np.int32), 2, [1, 4])
