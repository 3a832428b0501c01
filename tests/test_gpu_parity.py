"""Parity of the CUDA path (through the C ABI) with the CPU oracle: flow value and
surface heights must match bit for bit (integer results; tolerance 0)."""
import numpy as np
import pytest

import certificate
import oracle
import pins
from paper_2601_17026_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts, skipped there
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2601_17026_gb300 import pog  # noqa: E402


def gpu_solve(cost_np, delta, alpha, **opt):
    cost = torch.from_numpy(np.ascontiguousarray(cost_np, dtype=np.int32)).cuda()
    options = pog.make_options(**opt) if opt else None
    flow, h = pog.solve(cost, delta, alpha, options)
    return flow, h.cpu().numpy()


def assert_parity(cost, delta, alpha, **opt):
    flow, h = gpu_solve(cost, delta, alpha, **opt)
    ref = oracle.solve(cost, delta, alpha)
    assert flow == ref.flow, f"flow {flow} != oracle {ref.flow}"
    np.testing.assert_array_equal(h, ref.heights)
    return flow, h


def test_small_workload():
    v = synth.small_volume()
    assert_parity(v.cost, v.delta, v.alpha)


SHAPES = [(1, 1, 1), (1, 1, 2), (1, 1, 7), (2, 3, 4), (3, 2, 5), (1, 6, 4), (6, 1, 4), (4, 4, 8), (5, 3, 9)]


@pytest.mark.parametrize("shape", SHAPES)
def test_tiny_random(shape):
    rng = np.random.default_rng(abs(hash(shape)) % (2**32))
    Z = shape[2]
    for delta in sorted({0, 1, 2, 3, Z}):
        for alpha in (0, 3, 17):
            cost = rng.integers(-40, 81, size=shape).astype(np.int32)
            assert_parity(cost, delta, alpha)


def test_matches_brute_force_directly():
    rng = np.random.default_rng(4)
    for _ in range(20):
        cost = rng.integers(-20, 41, size=(2, 3, 4)).astype(np.int32)
        d, a = int(rng.integers(0, 3)), int(rng.integers(0, 5))
        flow, h = gpu_solve(cost, d, a)
        emin, hmin, _ = pins.brute_force(cost, d, a)
        np.testing.assert_array_equal(h, hmin)
        assert flow == emin + pins.identity_offset(cost)


@pytest.mark.parametrize("delta", list(range(0, 11)))
def test_delta_sweep(delta):
    """All delta from 0 to beyond Z: the solver drops hard arcs that land in the bottom
    layer; the oracle keeps the literal arc set."""
    rng = np.random.default_rng(100 + delta)
    cost = rng.integers(0, 300, size=(5, 4, 9)).astype(np.int32)
    for alpha in (0, 7):
        assert_parity(cost, delta, alpha)


@pytest.mark.parametrize("X,Y,Z,delta,alpha", [(37, 23, 50, 2, 5), (33, 65, 70, 3, 50), (70, 31, 41, 1, 0),
                                                (64, 64, 96, 2, 0), (9, 17, 33, 0, 20), (5, 3, 130, 40, 3)])
@pytest.mark.parametrize("mode", ["tiles", "nodes", "shape1", "shape3"])
def test_ragged_horizon_volumes(X, Y, Z, delta, alpha, mode):
    cost = synth.horizon_cost(synth.scaled_spec(X, Y, Z, synth.BASE_SEED + X, stream=500 + Y))
    opt = {"nodes": {"flags": pog.POG_FLAG_NODE_SWEEPS}, "shape1": {"tile_shape": 1},
           "shape3": {"tile_shape": 3}}.get(mode, {})
    assert_parity(cost, delta, alpha, **opt)


def test_degenerate_volumes():
    # a single layer: only the bottom, heights all 0
    c = np.arange(12, dtype=np.int32).reshape(3, 4, 1)
    flow, h = assert_parity(c, 2, 3)
    assert np.all(h == 0)
    # equal costs everywhere: ties resolve to the lowest surface
    flow, h = assert_parity(np.full((6, 5, 7), 11, dtype=np.int32), 1, 4)
    assert np.all(h == 0)
    # strictly decreasing columns: the top node is optimal everywhere
    c = np.broadcast_to(np.arange(10, 0, -1, dtype=np.int32), (4, 4, 10)).copy()
    flow, h = assert_parity(c, 1, 0)
    assert np.all(h == 9)
    # large magnitudes near the limit
    rng = np.random.default_rng(9)
    c = rng.integers(-(1 << 29), 1 << 29, size=(4, 5, 6)).astype(np.int32)
    assert_parity(c, 2, 1000)


def test_repeatable():
    cost = synth.horizon_cost(synth.scaled_spec(40, 40, 64, 5, stream=9))
    r0 = gpu_solve(cost, 2, 25)
    for _ in range(3):
        r = gpu_solve(cost, 2, 25)
        assert r[0] == r0[0]
        np.testing.assert_array_equal(r[1], r0[1])


def test_options_do_not_change_results():
    cost = synth.horizon_cost(synth.scaled_spec(30, 20, 48, 3, stream=11))
    ref = oracle.solve(cost, 2, 10)
    for opt in [dict(sweeps_per_relabel=1), dict(sweeps_per_relabel=64, tile_sweeps=1),
                dict(flags=pog.POG_FLAG_NO_GAP), dict(tile_sweeps=16), dict(flags=pog.POG_FLAG_NODE_SWEEPS),
                dict(flags=pog.POG_FLAG_NO_PREPUSH), dict(bfs_blocks_per_sm=1), dict(tile_sweeps=64),
                dict(tile_shape=1), dict(tile_shape=2), dict(tile_shape=3), dict(bfs_bottom_up_ratio=-1),
                dict(bfs_bottom_up_ratio=1), dict(relabel_factor=0.25), dict(sweeps_per_relabel=3, tile_shape=3),
                dict(flags=pog.POG_FLAG_NO_TMA), dict(flags=pog.POG_FLAG_NO_TMA, tile_shape=1),
                dict(relabel_factor=3.0, tile_shape=1, bfs_bottom_up_ratio=-1)]:
        flow, h = gpu_solve(cost, 2, 10, **opt)
        assert flow == ref.flow
        np.testing.assert_array_equal(h, ref.heights)


def test_certificate_export_state():
    cost = synth.horizon_cost(synth.scaled_spec(48, 40, 96, 17, stream=12))
    for delta, alpha in [(3, 50), (2, 0)]:
        t = torch.from_numpy(cost).cuda()
        with pog.pog_build(t, delta, alpha) as g:
            flow = pog.pog_maxflow(g)
            h = pog.pog_surface(g).cpu().numpy()
            st = pog.pog_export_state(g)
        certificate.check(cost, delta, alpha, st, flow, h)
        assert oracle.certify(cost, delta, alpha, st, flow, h) == 0
        assert oracle.cut_capacity(cost, h, delta, alpha) == flow


def test_energy_identity():
    cost = synth.horizon_cost(synth.scaled_spec(20, 30, 40, 8, stream=13))
    t = torch.from_numpy(cost).cuda()
    with pog.pog_build(t, 2, 9) as g:
        flow = pog.pog_maxflow(g)
        h = pog.pog_surface(g).cpu().numpy()
        e = pog.pog_energy(g)
    e_ref, ok = oracle.energy(cost, h, 2, 9)
    assert ok and e == e_ref
    assert flow == e + pins.identity_offset(cost)


def test_float_build_matches_quantised_oracle():
    spec = synth.scaled_spec(24, 20, 32, 21, stream=14)
    fc = synth.float_horizon_cost(spec)
    cq = np.rint(fc.astype(np.float64) * 1024.0).astype(np.int32)
    ref = oracle.solve(cq, 2, 10240)
    t = torch.from_numpy(fc).cuda()
    with pog.pog_build_f32(t, 1024.0, 2, 10240) as g:
        flow = pog.pog_maxflow(g)
        h = pog.pog_surface(g).cpu().numpy()
    assert flow == ref.flow
    np.testing.assert_array_equal(h, ref.heights)
    q = pog.pog_quantise(t, 1024.0).cpu().numpy()
    np.testing.assert_array_equal(q, cq)


def test_quantise_round_half_even_and_range():
    x = torch.tensor([0.5, 1.5, 2.5, -0.5, -1.5, 1e-3, 3.0], device="cuda") / 1024.0
    q = pog.pog_quantise(x, 1024.0).cpu().numpy()
    np.testing.assert_array_equal(q, [0, 2, 2, 0, -2, 0, 3])
    with pytest.raises(pog.PogError) as ei:
        pog.pog_quantise(torch.tensor([2.0 ** 21], device="cuda"), 1024.0)
    assert ei.value.status == pog.POG_E_OVERFLOW
    with pytest.raises(pog.PogError):
        pog.pog_quantise(torch.tensor([float("nan")], device="cuda"), 1024.0)


def test_errors():
    bad = torch.full((3, 3, 4), 1 << 30, dtype=torch.int32, device="cuda")
    with pog.pog_build(bad, 1, 0) as g:
        with pytest.raises(pog.PogError) as ei:
            pog.pog_maxflow(g)
        assert ei.value.status == pog.POG_E_OVERFLOW
    ok = torch.zeros((3, 3, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(pog.PogError) as ei:
        pog.pog_build(ok, -1, 0)
    assert ei.value.status == pog.POG_E_INVALID
    with pytest.raises(pog.PogError) as ei:
        pog.pog_build(ok, 1, -2)
    assert ei.value.status == pog.POG_E_INVALID
    with pog.pog_build(ok, 1, 0) as g:
        with pytest.raises(pog.PogError) as ei:
            pog.pog_surface(g)
        assert ei.value.status == pog.POG_E_STATE
        pog.pog_maxflow(g)
        h = pog.pog_surface(g).cpu().numpy()
        assert np.all(h == 0)
    with pytest.raises(pog.PogError):
        pog.pog_build(ok.float(), 1, 0)  # wrong dtype is rejected before the ABI call


def test_noconverge_cap():
    cost = synth.horizon_cost(synth.scaled_spec(32, 32, 64, 3, stream=15))
    t = torch.from_numpy(cost).cuda()
    with pog.pog_build(t, 2, 0, pog.make_options(max_rounds=1, sweeps_per_relabel=1)) as g:
        with pytest.raises(pog.PogError) as ei:
            pog.pog_maxflow(g)
        assert ei.value.status == pog.POG_E_NOCONVERGE


def test_batch_uneven():
    vols = synth.batch_volumes(limit=6)
    # shrink to keep the oracle quick while keeping the uneven shapes and parameters
    costs = [v.cost[: v.cost.shape[0] // 2, : v.cost.shape[1] // 3, :] for v in vols]
    flows, hs = pog.pog_solve_batch([torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in costs],
                                    [v.delta for v in vols], [v.alpha for v in vols])
    for c, v, f, h in zip(costs, vols, flows, hs):
        ref = oracle.solve(c, v.delta, v.alpha)
        assert f == ref.flow
        np.testing.assert_array_equal(h.cpu().numpy(), ref.heights)


def test_batch_last_live_volume_is_not_the_first():
    """Small easy volumes finish first; the hard one that finishes last sits at a nonzero
    node and tile offset (the single-volume kernels then run on a slice of the union)."""
    rng = np.random.default_rng(51)
    easy = [np.sort(rng.integers(0, 50, size=(9, 7, 20)), axis=2).astype(np.int32) for _ in range(3)]
    hard = synth.horizon_cost(synth.scaled_spec(70, 40, 96, 99, stream=61))
    costs = easy[:2] + [hard] + easy[2:]
    deltas = [1, 2, 3, 1]
    alphas = [0, 5, 20, 0]
    opts = pog.make_options(max_rounds=5000)
    for shape in (0, 1):
        opts.tile_shape = shape
        flows, hs = pog.pog_solve_batch([torch.from_numpy(c).cuda() for c in costs], deltas, alphas, opts)
        for c, d, a, f, h in zip(costs, deltas, alphas, flows, hs):
            ref = oracle.solve(c, d, a)
            assert f == ref.flow
            np.testing.assert_array_equal(h.cpu().numpy(), ref.heights)
