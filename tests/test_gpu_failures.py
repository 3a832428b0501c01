"""Failure detection without a GPU fault: a bounded device wait that runs out, and an
allocation that fails on the host. Each failure must come back as its status code, leak
nothing, and leave the device usable (a normal solve right after matches the oracle)."""
import numpy as np
import pytest

import oracle
from paper_2601_17026_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2601_17026_gb300 import pog  # noqa: E402


def _volume():
    cost = synth.horizon_cost(synth.scaled_spec(40, 36, 48, 71, stream=71))
    return cost, torch.from_numpy(cost).cuda()


def _assert_matches_oracle(cost, flow, heights, delta, alpha):
    ref = oracle.solve(cost, delta, alpha)
    assert flow == ref.flow
    np.testing.assert_array_equal(heights, ref.heights)


def test_grid_barrier_timeout_is_reported_and_the_device_recovers():
    """The searches' grid barrier with a wait limit of one poll: blocks that arrive early
    give up, raise the timeout word and leave; every other block leaves at its next
    barrier. The call returns POG_E_TIMEOUT; the graph frees cleanly."""
    cost, t = _volume()
    for _ in range(2):
        with pog.pog_build(t, 2, 9, pog.make_options(test_wait_limit=1)) as g:
            with pytest.raises(pog.PogError) as ei:
                pog.pog_maxflow(g)
            assert ei.value.status == pog.POG_E_TIMEOUT
        torch.cuda.synchronize()
        flow, h = pog.solve(t, 2, 9)
        _assert_matches_oracle(cost, flow, h.cpu().numpy(), 2, 9)


def test_grid_barrier_timeout_in_the_no_allocation_path():
    cost, t = _volume()
    heights = torch.empty(cost.shape[:2], dtype=torch.int32, device="cuda")
    with pytest.raises(pog.PogError) as ei:
        pog.pog_solve_noalloc(t, 2, 9, heights, pog.make_options(test_wait_limit=1))
    assert ei.value.status == pog.POG_E_TIMEOUT
    flow = pog.pog_solve_noalloc(t, 2, 9, heights)
    _assert_matches_oracle(cost, flow, heights.cpu().numpy(), 2, 9)


@pytest.mark.parametrize("site", [1, 2, 3])
def test_allocation_failure_returns_nomem_and_keeps_nothing(site):
    """Allocation k of a build fails (1 device state, 2 tensor-map table, 3 pinned
    counters): POG_E_NOMEM, and the device memory allocated before it is released."""
    cost = synth.horizon_cost(synth.scaled_spec(128, 128, 64, 72, stream=72))  # ~50 MB of state
    t = torch.from_numpy(cost).cuda()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        with pytest.raises(pog.PogError) as ei:
            pog.pog_build(t, 2, 5, pog.make_options(test_fail_alloc=site))
        assert ei.value.status == pog.POG_E_NOMEM
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    flow, h = pog.solve(t, 2, 5)
    _assert_matches_oracle(cost, flow, h.cpu().numpy(), 2, 5)
