"""CPU oracle for the proper-order multi-column min-cut — TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg
of ``bench.py`` may import this package. The product path (the CUDA library and its
binding) never does, and this package imports nothing from it.

``solve`` builds the literal explicit-edge s-t graph of Section 1.2 and runs Dinic's
blocking-flow max-flow (Section 2) in plain C (``pog_oracle.c``), int64 throughout.
Its result is the max-flow value (Eq. 5), the minimal minimum cut (nodes reachable
from s in the final residual graph; the cut of Theorem 1.1) and the surface height
of each column, the top node of the cut in that column.

Pins (see ``tests/test_oracle_pins.py``): brute-force enumeration of all feasible
surfaces on tiny volumes, the closed form for delta >= Z-1 without soft penalty,
an exact dynamic program over one row of columns, the energy/flow identity, and the
capacity / conservation / max-flow = min-cut invariants checked inside the C code.

``solve_convex`` builds the same literal graph with a convex pairwise cost f over the
edge interval (one layer of soft arcs per height drop, capacity the second difference of
f) and runs the same Dinic; ``energy_convex`` is that energy from its definition. Pins in
``tests/test_convex_pins.py``: enumeration, the single-row dynamic program with f, the
energy identity, the linear profile against ``solve``, and planted mistakes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pog_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", 1: "bad arguments", 2: "out of memory", 3: "capacity violated",
          4: "conservation violated", 5: "flow != cut capacity", 6: "empty column in cut"}

CERTIFY_ERRORS = {0: "ok", 2: "out of memory", 10: "arc capacity violated", 11: "excess != inflow - outflow",
                  12: "preflow value != reported flow", 13: "cut != residual reach of the excess nodes",
                  14: "heights != top of the cut", 15: "cut capacity of the surface != flow"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-Wextra",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_solve.restype = ctypes.c_int
    lib.oracle_solve.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                 ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, i64p, i32p, i64p]
    lib.oracle_solve_convex.restype = ctypes.c_int
    lib.oracle_solve_convex.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, i64p, ctypes.c_int32, i64p, i32p, i64p]
    lib.oracle_energy_convex.restype = ctypes.c_int64
    lib.oracle_energy_convex.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, i64p, i32p, i32p]
    lib.oracle_cut_capacity_convex.restype = ctypes.c_int64
    lib.oracle_cut_capacity_convex.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_int32, i64p, i32p]
    lib.oracle_solve_state_convex.restype = ctypes.c_int
    lib.oracle_solve_state_convex.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              i64p, i64p, i32p, i32p, i32p, i32p, i32p, i32p, i32p, i32p]
    lib.oracle_certify_convex.restype = ctypes.c_int
    lib.oracle_certify_convex.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          i64p, i32p, i32p, i32p, i32p, i32p, i32p, i32p, i32p, ctypes.c_int64]
    lib.oracle_energy.restype = ctypes.c_int64
    lib.oracle_energy.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.c_int64, i32p, i32p]
    lib.oracle_cut_capacity.restype = ctypes.c_int64
    lib.oracle_cut_capacity.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int64, i32p]
    lib.oracle_solve_state.restype = ctypes.c_int
    lib.oracle_solve_state.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int64, i64p, i32p] + [i32p] * 6
    lib.oracle_certify.restype = ctypes.c_int
    lib.oracle_certify.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int64] + [i32p] * 7 + [ctypes.c_int64]
    return lib


def load_library(path: str):
    """Load an oracle build from an explicit path (used to test planted mistakes)."""
    return _configure(ctypes.CDLL(path))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _i32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _cost(cost) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(cost), dtype=np.int32)
    if c.ndim != 3:
        raise ValueError("cost must be [X, Y, Z]")
    return c


class OracleResult:
    def __init__(self, flow, heights, phases, augmentations, nodes, half_arcs):
        self.flow = flow
        self.heights = heights
        self.phases = phases
        self.augmentations = augmentations
        self.nodes = nodes
        self.half_arcs = half_arcs

    def __repr__(self):
        return (f"OracleResult(flow={self.flow}, phases={self.phases}, "
                f"augmentations={self.augmentations}, nodes={self.nodes})")


def solve(cost, delta: int, alpha: int, check: bool = False, lib=None) -> OracleResult:
    """Max-flow value and minimal-cut surface of one int32 [X, Y, Z] cost volume."""
    lib = lib or _load()
    c = _cost(cost)
    X, Y, Z = c.shape
    heights = np.empty((X, Y), dtype=np.int32)
    flow = ctypes.c_int64(0)
    stats = (ctypes.c_int64 * 4)()
    rc = lib.oracle_solve(_i32(c), X, Y, Z, int(delta), int(alpha), 1 if check else 0,
                          ctypes.byref(flow), _i32(heights), stats)
    if rc != 0:
        raise RuntimeError(f"oracle_solve failed: {ERRORS.get(rc, rc)}")
    return OracleResult(int(flow.value), heights, *[int(v) for v in stats])


def _profile(delta: int, f) -> np.ndarray:
    fa = np.ascontiguousarray(np.asarray(f if f is not None else [], dtype=np.int64).reshape(-1))
    if fa.size != delta:
        raise ValueError("f must hold f(1..delta)")
    return fa


def solve_convex(cost, delta: int, f, check: bool = False, lib=None) -> OracleResult:
    """Max-flow value and minimal-cut surface with the convex pairwise cost f
    (f[d-1] = f(d) for d = 1..delta, f(0) = 0): the literal graph with one layer of soft
    arcs per height drop d < delta, capacity the second difference of f (Section 1.2's
    convex edge costs over an edge interval), solved by the same Dinic."""
    lib = lib or _load()
    c = _cost(cost)
    X, Y, Z = c.shape
    fa = _profile(delta, f)
    heights = np.empty((X, Y), dtype=np.int32)
    flow = ctypes.c_int64(0)
    stats = (ctypes.c_int64 * 4)()
    rc = lib.oracle_solve_convex(_i32(c), X, Y, Z, int(delta), fa.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 1 if check else 0, ctypes.byref(flow), _i32(heights), stats)
    if rc != 0:
        raise RuntimeError(f"oracle_solve_convex failed: {ERRORS.get(rc, rc)}")
    return OracleResult(int(flow.value), heights, *[int(v) for v in stats])


def energy_convex(cost, heights, delta: int, f):
    """(E, feasible): sum_col c(col, h) + sum over unordered 4-neighbour pairs f(|h_p - h_q|)."""
    lib = _load()
    c = _cost(cost)
    X, Y, Z = c.shape
    fa = _profile(delta, f)
    h = np.ascontiguousarray(heights, dtype=np.int32).reshape(X, Y)
    feas = ctypes.c_int32(0)
    e = lib.oracle_energy_convex(_i32(c), X, Y, Z, int(delta), fa.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 _i32(h), ctypes.byref(feas))
    return int(e), bool(feas.value)


CONVEX_STATE_KEYS = ("excess", "sink", "fdown", "fhard", "gpair", "flayer", "in_cut")


def _i64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def cut_capacity_convex(cost, heights, delta: int, f) -> int:
    """Eq. 6 for the cut below the surface, arc by arc over the literal layered graph; -1 when
    an infinite arc crosses it."""
    lib = _load()
    c = _cost(cost)
    X, Y, Z = c.shape
    fa = _profile(delta, f)
    h = np.ascontiguousarray(heights, dtype=np.int32).reshape(X, Y)
    return int(lib.oracle_cut_capacity_convex(_i32(c), X, Y, Z, int(delta), _i64(fa), _i32(h)))


def solve_state_convex(cost, delta: int, f, lib=None):
    """(flow, heights, state): the oracle's max flow of the convex-cost graph in a solver-state
    layout (the dict ``certify_convex`` takes; flayer holds (delta - 1) * 4 arrays of N words,
    layer d = 1.. and direction 0..3)."""
    lib = lib or _load()
    c = _cost(cost)
    X, Y, Z = c.shape
    N = X * Y * Z
    fa = _profile(delta, f)
    heights = np.empty((X, Y), dtype=np.int32)
    st = {k: np.empty(N, dtype=np.int32) for k in ("excess", "sink", "fdown", "in_cut")}
    st["fhard"] = np.empty(4 * N, dtype=np.int32)
    st["gpair"] = np.empty(2 * N, dtype=np.int32)
    st["flayer"] = np.zeros(max(4 * (delta - 1), 1) * N, dtype=np.int32)
    flow = ctypes.c_int64(0)
    rc = lib.oracle_solve_state_convex(_i32(c), X, Y, Z, int(delta), _i64(fa), ctypes.byref(flow), _i32(heights),
                                       _i32(st["excess"]), _i32(st["sink"]), _i32(st["fdown"]), _i32(st["fhard"]),
                                       _i32(st["gpair"]), _i32(st["flayer"]), _i32(st["in_cut"]))
    if rc != 0:
        raise RuntimeError(f"oracle_solve_state_convex failed: {ERRORS.get(rc, rc)}")
    return int(flow.value), heights, st


def certify_convex(cost, delta: int, f, state: dict, flow: int, heights, lib=None) -> int:
    """O(N) certificate of a convex-cost state (see ``solve_state_convex``); 0 means the
    preflow is feasible with value `flow`, the cut below `heights` has capacity `flow`, and the
    cut is the residual reach of the excess nodes. See CERTIFY_ERRORS."""
    lib = lib or _load()
    c = _cost(cost)
    X, Y, Z = c.shape
    N = X * Y * Z
    fa = _profile(delta, f)
    arr = {k: np.ascontiguousarray(state[k], dtype=np.int32) for k in CONVEX_STATE_KEYS}
    if arr["flayer"].size < max(4 * (delta - 1), 1) * N:
        raise ValueError("flayer must hold 4 * (delta - 1) arrays of N words")
    h = np.ascontiguousarray(heights, dtype=np.int32).reshape(X, Y)
    return int(lib.oracle_certify_convex(_i32(c), X, Y, Z, int(delta), _i64(fa), _i32(arr["excess"]),
                                         _i32(arr["sink"]), _i32(arr["fdown"]), _i32(arr["fhard"]),
                                         _i32(arr["gpair"]), _i32(arr["flayer"]), _i32(arr["in_cut"]), _i32(h),
                                         int(flow)))


def solve_state(cost, delta: int, alpha: int, lib=None):
    """(flow, heights, state): the oracle's max flow described in the layout of a solver's
    exported state (the dict ``certify`` takes: excess, sink, fdown, fhard, gsoft, in_cut;
    the bottom layer counted as part of the source), for checking the certificate on a
    state known to be optimal."""
    lib = lib or _load()
    c = _cost(cost)
    X, Y, Z = c.shape
    N = X * Y * Z
    heights = np.empty((X, Y), dtype=np.int32)
    st = {k: np.empty(N, dtype=np.int32) for k in ("excess", "sink", "fdown", "in_cut")}
    st["fhard"] = np.empty(4 * N, dtype=np.int32)
    st["gsoft"] = np.empty(2 * N, dtype=np.int32)
    flow = ctypes.c_int64(0)
    rc = lib.oracle_solve_state(_i32(c), X, Y, Z, int(delta), int(alpha), ctypes.byref(flow), _i32(heights),
                                _i32(st["excess"]), _i32(st["sink"]), _i32(st["fdown"]), _i32(st["fhard"]),
                                _i32(st["gsoft"]), _i32(st["in_cut"]))
    if rc != 0:
        raise RuntimeError(f"oracle_solve_state failed: {ERRORS.get(rc, rc)}")
    return int(flow.value), heights, st


def energy(cost, heights, delta: int, alpha: int):
    """(E, feasible): Eq. 1 with E_feature = sum_col c(col, h) and E_prior =
    alpha * sum over unordered 4-neighbour pairs |h_p - h_q|."""
    lib = _load()
    c = _cost(cost)
    X, Y, Z = c.shape
    h = np.ascontiguousarray(heights, dtype=np.int32).reshape(X, Y)
    feas = ctypes.c_int32(0)
    e = lib.oracle_energy(_i32(c), X, Y, Z, int(delta), int(alpha), _i32(h), ctypes.byref(feas))
    return int(e), bool(feas.value)


def cut_capacity(cost, heights, delta: int, alpha: int) -> int:
    """Eq. 6 for the cut below the surface (z <= h in every column), arc by arc over the
    literal graph; -1 when an infinite arc crosses it."""
    lib = _load()
    c = _cost(cost)
    X, Y, Z = c.shape
    h = np.ascontiguousarray(heights, dtype=np.int32).reshape(X, Y)
    return int(lib.oracle_cut_capacity(_i32(c), X, Y, Z, int(delta), int(alpha), _i32(h)))


def certify(cost, delta: int, alpha: int, state: dict, flow: int, heights) -> int:
    """Check a solver's exported final state (the dict of ``pog_export_state``: excess,
    sink, fdown, fhard, gsoft, in_cut) against (flow, heights) in O(N); 0 means the
    preflow is feasible, its value is `flow`, the cut below `heights` has capacity
    `flow`, and the cut is the residual reach of the excess nodes. See CERTIFY_ERRORS."""
    lib = _load()
    c = _cost(cost)
    X, Y, Z = c.shape
    arr = {k: np.ascontiguousarray(state[k], dtype=np.int32) for k in
           ("excess", "sink", "fdown", "fhard", "gsoft", "in_cut")}
    h = np.ascontiguousarray(heights, dtype=np.int32).reshape(X, Y)
    return int(lib.oracle_certify(_i32(c), X, Y, Z, int(delta), int(alpha), _i32(arr["excess"]),
                                  _i32(arr["sink"]), _i32(arr["fdown"]), _i32(arr["fhard"]),
                                  _i32(arr["gsoft"]), _i32(arr["in_cut"]), _i32(h), int(flow)))
