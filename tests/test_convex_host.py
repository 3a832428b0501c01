"""Host-side argument checks of pog_solve_convex (CPU only): every rejection below happens
before the call touches the device, so no GPU is needed and no device memory is used."""
import ctypes

import numpy as np
import pytest

from paper_2601_17026_gb300 import build as build_mod
from paper_2601_17026_gb300 import pog

FAKE_DEV = ctypes.c_void_p(0x1000)  # never dereferenced: each call below is rejected first


@pytest.fixture(scope="module")
def lib():
    return pog.load(build_mod.build())


def _call(lib, X, Y, Z, delta, f, cost=FAKE_DEV, heights=FAKE_DEV):
    fa = np.ascontiguousarray(np.asarray(f, dtype=np.int64))
    fptr = ctypes.c_void_p(fa.ctypes.data) if fa.size else None
    flow, energy = ctypes.c_int64(0), ctypes.c_int64(0)
    return lib.pog_solve_convex(cost, X, Y, Z, delta, fptr, None, None, ctypes.byref(flow), ctypes.byref(energy),
                                heights, None)


@pytest.mark.parametrize("f, why", [
    ([4, 5, 5], "second difference 5 - 10 + 4 < 0"),
    ([-1, 0], "f(1) < 0"),
    ([1, 1 << 31], "layer capacity >= 2^30"),
    ([1 << 30], "f(1) = 2^30"),
    ([0, 0, 3, 4], "second difference at d = 3: 4 - 6 + 0 < 0"),
])
def test_non_convex_or_oversized_profiles_are_rejected(lib, f, why):
    assert _call(lib, 4, 4, 8, len(f), f) == pog.POG_E_INVALID, why


def test_bad_sizes_and_pointers_are_rejected(lib):
    f = [4, 16]
    assert _call(lib, 0, 4, 8, 2, f) == pog.POG_E_INVALID
    assert _call(lib, 4, 4, -1, 2, f) == pog.POG_E_INVALID
    assert _call(lib, 4, 4, 8, -1, []) == pog.POG_E_INVALID
    assert _call(lib, 4, 4, 8, pog.POG_CONVEX_MAX_DELTA + 1, np.arange(1, 34)) == pog.POG_E_INVALID
    assert _call(lib, 4, 4, 8, 2, f, cost=None) == pog.POG_E_INVALID
    assert _call(lib, 4, 4, 8, 2, f, heights=None) == pog.POG_E_INVALID
    assert _call(lib, 2048, 2048, 1024, 2, f) == pog.POG_E_INVALID   # 2^32 nodes
    # delta > 0 without a profile
    flow, energy = ctypes.c_int64(0), ctypes.c_int64(0)
    assert lib.pog_solve_convex(FAKE_DEV, 4, 4, 8, 2, None, None, None, ctypes.byref(flow), ctypes.byref(energy),
                                FAKE_DEV, None) == pog.POG_E_INVALID


def test_binding_checks_profile_length():
    torch = pytest.importorskip("torch")
    with pytest.raises(pog.PogError):
        pog.pog_solve_convex(torch.zeros((2, 2, 4), dtype=torch.int32), 2, [1])
