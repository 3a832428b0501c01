"""Full-size cases. The 256^3 volume and the 64 uneven volumes of the batched workload
are compared with the oracle's stored results (tests/golden/medium.json and batch.json,
written by make_golden.py with the oracle alone). The
512x512x384 workload, too large for the oracle to solve in a test, is solved in the
launch configuration the benchmark times (the tuned options) and checked by properties
that hold at any size, with the oracle's linear-time routines: the exported final state
is a feasible preflow whose value is the reported flow, the cut below the surface has
capacity equal to the flow (weak duality, so both are optimal), and the cut is the
residual reach of the excess nodes (the minimal minimum cut)."""
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

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2601_17026_gb300 import autotune, pog  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _tuned(vol):
    X, Y, Z = vol.cost.shape
    return pog.make_options(**autotune.tuned_params(X, Y, Z, vol.delta, vol.alpha))


def test_medium_matches_stored_oracle():
    with open(os.path.join(GOLDEN, "medium.json")) as f:
        ref = json.load(f)
    vol = synth.medium_volume()
    assert list(vol.cost.shape) == ref["shape"] and (vol.delta, vol.alpha) == (ref["delta"], ref["alpha"])
    flow, h = pog.solve(torch.from_numpy(vol.cost).cuda(), vol.delta, vol.alpha, _tuned(vol))
    h = np.ascontiguousarray(h.cpu().numpy(), dtype=np.int32)
    assert flow == ref["flow"]
    assert int(h.sum()) == ref["heights_sum"]
    assert hashlib.sha256(h.tobytes()).hexdigest() == ref["heights_sha256"]


def test_seismic_full_size_certificate():
    vol = synth.seismic_volume()
    with pog.pog_build(torch.from_numpy(vol.cost).cuda(), vol.delta, vol.alpha, _tuned(vol)) as g:
        flow = pog.pog_maxflow(g)
        h = pog.pog_surface(g).cpu().numpy()
        st = pog.pog_export_state(g)
    assert oracle.certify(vol.cost, vol.delta, vol.alpha, st, flow, h) == 0
    assert oracle.cut_capacity(vol.cost, h, vol.delta, vol.alpha) == flow
    e, feasible = oracle.energy(vol.cost, h, vol.delta, vol.alpha)
    assert feasible
    assert flow == e + pins.identity_offset(vol.cost)  # max-flow = E*(h) + K for the construction


def test_uneven_batch_matches_stored_oracle():
    """The 64 uneven volumes (227M nodes) in one batched solve, against the oracle's
    stored flow and surface of every volume (tests/golden/batch.json)."""
    with open(os.path.join(GOLDEN, "batch.json")) as f:
        ref = json.load(f)["volumes"]
    vols = synth.batch_volumes()
    assert len(vols) == len(ref)
    costs = [torch.from_numpy(v.cost).cuda() for v in vols]
    flows, heights = pog.pog_solve_batch(costs, [v.delta for v in vols], [v.alpha for v in vols])
    for v, r, fl, h in zip(vols, ref, flows, heights):
        assert list(v.cost.shape) == r["shape"] and (v.delta, v.alpha) == (r["delta"], r["alpha"])
        assert fl == r["flow"], v.name
        h = np.ascontiguousarray(h.cpu().numpy(), dtype=np.int32)
        assert hashlib.sha256(h.tobytes()).hexdigest() == r["heights_sha256"], v.name
