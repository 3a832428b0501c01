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


def test_differentiable_workload_matches_stored_oracle():
    """The 16 float volumes of 128^3 (delta 2, alpha 10, hinge margin 1 against a flat
    target): energies, optimal and loss-augmented surfaces, hinge losses and the gradient
    of E* + L, against the oracle's stored results (tests/golden/diff.json). The
    loss-augmented solve runs warm (from the energy solve's state) in the autograd path and
    cold through the raw entry point; both must give the oracle's values."""
    from paper_2601_17026_gb300 import autograd as pag

    with open(os.path.join(GOLDEN, "diff.json")) as f:
        ref = json.load(f)["volumes"]
    fc = synth.diff_volumes_f32()
    ht = synth.diff_target()
    B, X, Y, Z = fc.shape
    assert len(ref) == B
    x = torch.from_numpy(fc).cuda().requires_grad_(True)
    htd = torch.from_numpy(ht).cuda()
    e, loss, h, hh = pag.solve_with_hinge(x, htd, synth.DIFF_DELTA, synth.DIFF_ALPHA, synth.DIFF_MARGIN)
    (e.sum() + loss.sum()).backward()

    def sha(t):
        return hashlib.sha256(np.ascontiguousarray(t.cpu().numpy(), dtype=np.int32).tobytes()).hexdigest()

    for b, r in enumerate(ref):
        assert e[b].item() * 1024 == r["energy"], b
        assert loss[b].item() * 1024 == r["hinge_q"], b
        assert sha(h[b]) == r["heights_sha256"], b
        assert sha(hh[b]) == r["aug_heights_sha256"], b
    # gradient of E* + L: onehot(h*) + onehot(h_t) - onehot(h_hat), exactly
    zs = torch.arange(Z, device="cuda", dtype=torch.int32)
    want = ((h[..., None] == zs).float() + (htd[..., None] == zs).float() - (hh[..., None] == zs).float())
    assert torch.equal(x.grad, want)
    # the raw entry point, warm and cold: flow values of both graphs as well
    xc = torch.from_numpy(fc).cuda()
    for flags in (0, pog.POG_FLAG_COLD_HINGE):
        out = pog.pog_solve_batch_f32_hinge(xc, 1024.0, htd, 1024, synth.DIFF_DELTA, 10240,
                                            pog.make_options(flags=flags))
        for b, r in enumerate(ref):
            assert out["flows"][b] == r["flow"] and out["aug_flows"][b] == r["aug_flow"], (flags, b)
            assert out["energies"][b] == r["energy"] and out["aug_energies"][b] == r["aug_energy"], (flags, b)
            assert out["hinge"][b] == r["hinge_q"], (flags, b)
            assert sha(out["h_hat"][b]) == r["aug_heights_sha256"], (flags, b)
