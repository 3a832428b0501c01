"""pog_solve_noalloc, the entry point for callers that may not allocate, against the
ordinary pog_build / pog_maxflow / pog_surface path (tolerance 0: integer results).

It lives in a file of its own that pytest collects last, so that a run stopping at the
first failure has already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2601_17026_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2601_17026_gb300 import pog  # noqa: E402


def _reference(cost, delta, alpha):
    flow, h = pog.solve(cost, delta, alpha)
    return flow, h.cpu().numpy()


def _noalloc(cost, delta, alpha):
    heights = torch.full(cost.shape[:2], -7, dtype=torch.int32, device="cuda")
    flow = pog.pog_solve_noalloc(cost, delta, alpha, heights)
    return flow, heights.cpu().numpy()


def test_noalloc_matches_allocating_path_twice_in_a_row():
    # two different volumes back to back: the second call must not see the first's state
    a = torch.from_numpy(synth.horizon_cost(synth.scaled_spec(40, 30, 48, 31, stream=41))).cuda()
    b = torch.from_numpy(synth.horizon_cost(synth.scaled_spec(33, 20, 64, 32, stream=42))).cuda()
    cases = [(a, 2, 25), (b, 3, 0), (a, 2, 25)]
    for cost, delta, alpha in cases:
        ref = _reference(cost, delta, alpha)
        got = _noalloc(cost, delta, alpha)
        assert got[0] == ref[0]
        np.testing.assert_array_equal(got[1], ref[1])


def test_noalloc_matches_the_oracle():
    """Against the CPU oracle directly, not only against the allocating GPU path."""
    import oracle

    for seed, (X, Y, Z), delta, alpha in [(43, (24, 20, 40), 2, 25), (44, (17, 33, 36), 1, 0)]:
        cost = synth.horizon_cost(synth.scaled_spec(X, Y, Z, seed, stream=seed))
        got = _noalloc(torch.from_numpy(cost).cuda(), delta, alpha)
        ref = oracle.solve(cost, delta, alpha)
        assert got[0] == ref.flow
        np.testing.assert_array_equal(got[1], ref.heights)


def test_noalloc_rejects_a_heights_buffer_of_the_wrong_shape():
    cost = torch.zeros((6, 5, 8), dtype=torch.int32, device="cuda")
    for bad in (torch.empty((6, 4), dtype=torch.int32, device="cuda"), torch.empty((30,), dtype=torch.int32,
                                                                                   device="cuda")):
        with pytest.raises(pog.PogError) as ei:
            pog.pog_solve_noalloc(cost, 1, 0, bad)
        assert ei.value.status == pog.POG_E_INVALID


def test_noalloc_rejects_volumes_beyond_the_scratch():
    big = torch.zeros((128, 128, 64), dtype=torch.int32, device="cuda")  # 1M nodes > limit
    heights = torch.empty((128, 128), dtype=torch.int32, device="cuda")
    with pytest.raises(pog.PogError) as ei:
        pog.pog_solve_noalloc(big, 1, 5, heights)
    assert ei.value.status == pog.POG_E_INVALID
