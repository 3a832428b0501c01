"""Narrow-band construction on the GPU (pog_narrow_band, pog_band_heights) against the
oracle's numpy construction, bit for bit, and a band solve against the oracle's Dinic
on the same band, mapped back to image heights."""
import numpy as np
import pytest

import oracle
from oracle import band as oband
from paper_2601_17026_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2601_17026_gb300 import pog  # noqa: E402


def _gpu_band(cost, lm, stick, factor, outside):
    b, c = pog.pog_narrow_band(torch.from_numpy(cost).cuda(), torch.from_numpy(np.asarray(lm, np.int32)).cuda(),
                               stick, factor, outside)
    return b, c


def test_band_construction_full_size():
    """The 512x512x384 volume with landmarks on its central horizon (8x8 lattice),
    stick 16, band factor 2: 65 rows per column, 17M band nodes, every one equal."""
    spec = synth.spec_seismic()
    cost = synth.horizon_cost(spec)
    lm = synth.horizon_landmarks(spec, 8)
    b, c = _gpu_band(cost, lm, synth.BAND_STICK, synth.BAND_FACTOR, synth.BAND_OUTSIDE)
    rb, rc = oband.narrow_band(cost, lm, synth.BAND_STICK, synth.BAND_FACTOR, synth.BAND_OUTSIDE)
    np.testing.assert_array_equal(c.cpu().numpy(), rc)
    assert torch.equal(b.cpu(), torch.from_numpy(rb))


def test_band_solve_full_size_matches_stored_oracle():
    """The benchmark's band (17M nodes, delta 3, alpha 50) solved in the bench's launch
    configuration: flow, band surface and image heights against the oracle's stored Dinic
    result (tests/golden/band.json)."""
    import hashlib
    import json
    import os

    from paper_2601_17026_gb300 import autotune

    gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "band.json")
    if not os.path.exists(gold):
        pytest.skip("no stored oracle result for the full-size band")
    with open(gold) as fh:
        ref = json.load(fh)
    spec = synth.spec_seismic()
    cost = synth.horizon_cost(spec)
    lm = synth.horizon_landmarks(spec, 8)
    half = synth.BAND_STICK * synth.BAND_FACTOR
    b, c = _gpu_band(cost, lm, synth.BAND_STICK, synth.BAND_FACTOR, synth.BAND_OUTSIDE)
    X, Y, Zb = b.shape
    opts = pog.make_options(**autotune.tuned_params(X, Y, Zb, 3, 50))
    with pog.pog_build(b, 3, 50, opts) as g:
        flow = pog.pog_maxflow(g)
        hb = pog.pog_surface(g)
        himg = pog.pog_band_heights(hb, c, half)
    sha = lambda t: hashlib.sha256(t.cpu().numpy().astype(np.int32).tobytes()).hexdigest()  # noqa: E731
    assert sha(b) == ref["band_sha256"] and sha(c) == ref["center_sha256"]
    assert flow == ref["flow"]
    assert sha(hb) == ref["heights_sha256"] and int(hb.sum().item()) == ref["heights_sum"]
    assert sha(himg) == ref["image_heights_sha256"]


@pytest.mark.parametrize("grid,stick,factor", [(4, 6, 2), (3, 5, 1), (1, 20, 3)])
def test_band_solve_matches_oracle(grid, stick, factor):
    spec = synth.scaled_spec(48, 40, 96, 29, stream=30)
    cost = synth.horizon_cost(spec)
    lm = synth.horizon_landmarks(spec, grid)
    b, c = _gpu_band(cost, lm, stick, factor, 1200)
    half = stick * factor
    flow, hb = pog.solve(b, 2, 25)
    himg = pog.pog_band_heights(hb, c, half).cpu().numpy()
    rb, rc = oband.narrow_band(cost, lm, stick, factor, 1200)
    ref = oracle.solve(rb, 2, 25)
    assert flow == ref.flow
    np.testing.assert_array_equal(hb.cpu().numpy(), ref.heights)
    np.testing.assert_array_equal(himg, oband.band_heights(ref.heights, rc, half))


def test_band_edge_cases_and_errors():
    rng = np.random.default_rng(8)
    cost = rng.integers(0, 100, size=(5, 6, 10)).astype(np.int32)
    # landmarks at the image's bottom and top rows; half larger than the image
    lm = [(0, 0, 0), (4, 5, 9), (2, 2, 5), (2, 2, 1)]
    b, c = _gpu_band(cost, lm, 7, 2, -3)
    rb, rc = oband.narrow_band(cost, lm, 7, 2, -3)
    np.testing.assert_array_equal(c.cpu().numpy(), rc)
    np.testing.assert_array_equal(b.cpu().numpy(), rb)
    t = torch.from_numpy(cost).cuda()
    with pytest.raises(pog.PogError) as ei:
        pog.pog_narrow_band(t, torch.zeros((0, 3), dtype=torch.int32, device="cuda"), 2, 1, 0)
    assert ei.value.status == pog.POG_E_INVALID
    with pytest.raises(pog.PogError) as ei:
        pog.pog_narrow_band(t, torch.zeros((1, 3), dtype=torch.int32, device="cuda"), 2, 0, 0)
    assert ei.value.status == pog.POG_E_INVALID
