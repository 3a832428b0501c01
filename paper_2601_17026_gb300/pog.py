"""Thin Python binding of the C ABI in ``include/pog.h`` (``libpog.so``).

The functions carry the C names and only marshal arguments: every step of the solve
runs in the library's CUDA kernels. Tensors are torch CUDA tensors (torch provides
device memory and streams); the library is loaded from this package directory and
there is no fallback — a missing or unloadable library raises ``PogError``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpog.so")

POG_OK = 0
POG_E_INVALID = 1
POG_E_OVERFLOW = 2
POG_E_NOMEM = 3
POG_E_CUDA = 4
POG_E_NOCONVERGE = 5
POG_E_TIMEOUT = 6
POG_E_STATE = 7
POG_FLAG_NO_GAP = 1
POG_FLAG_TIMING = 2
POG_FLAG_NO_PREPUSH = 4
POG_FLAG_NODE_SWEEPS = 8
POG_FLAG_NO_TMA = 16
POG_FLAG_COLD_HINGE = 32
POG_CONVEX_MAX_DELTA = 32

EXPORTED = ["pog_build", "pog_build_f32", "pog_build_f32_augmented", "pog_maxflow", "pog_surface", "pog_energy",
            "pog_stats", "pog_export_state", "pog_trace", "pog_free", "pog_strerror", "pog_quantise", "pog_backward",
            "pog_surface_energy", "pog_solve_batch", "pog_solve_batch_f32", "pog_solve_batch_f32_hinge",
            "pog_narrow_band", "pog_band_heights", "pog_solve_noalloc", "pog_solve_convex"]


class PogError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {pog_strerror(status)} (status {status})")


class pog_options(ctypes.Structure):
    _fields_ = [("sweeps_per_relabel", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("tile_sweeps", ctypes.c_int32), ("flags", ctypes.c_int32), ("bfs_blocks_per_sm", ctypes.c_int32),
                ("relabel_factor", ctypes.c_float), ("tile_shape", ctypes.c_int32),
                ("bfs_bottom_up_ratio", ctypes.c_int32), ("test_wait_limit", ctypes.c_int32),
                ("test_fail_alloc", ctypes.c_int32)]


class pog_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("rounds", "sweeps", "bfs_passes", "cut_passes", "gaps",
                                               "active_initial", "nodes", "state_bytes", "launches", "tiles_visited")] + \
               [(n, ctypes.c_double) for n in ("sweep_ms", "bfs_ms", "cut_ms", "build_ms")]


class pog_volume(ctypes.Structure):
    _fields_ = [("cost_dev", ctypes.c_void_p), ("X", ctypes.c_int32), ("Y", ctypes.c_int32),
                ("Z", ctypes.c_int32), ("delta", ctypes.c_int32), ("alpha", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libpog.so (once) and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise PogError(POG_E_CUDA, f"{path} is missing; build it with __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        i64p = ctypes.POINTER(ctypes.c_int64)
        opts = ctypes.POINTER(pog_options)
        sig = {
            "pog_build": [vp, i32, i32, i32, i32, i32, opts, vp, ctypes.POINTER(vp)],
            "pog_build_f32": [vp, f32, i32, i32, i32, i32, i32, opts, vp, ctypes.POINTER(vp)],
            "pog_build_f32_augmented": [vp, f32, vp, i32, i32, i32, i32, i32, i32, opts, vp, ctypes.POINTER(vp)],
            "pog_maxflow": [vp, i64p],
            "pog_energy": [vp, i64p],
            "pog_surface_energy": [vp, f32, vp, i32, i32, i32, i32, i32, vp, vp],
            "pog_surface": [vp, vp],
            "pog_stats": [vp, ctypes.POINTER(pog_stats_t)],
            "pog_export_state": [vp, vp, vp, vp, vp, vp, vp],
            "pog_trace": [vp, vp, i32, ctypes.POINTER(i32)],
            "pog_quantise": [vp, vp, i64, f32, vp],
            "pog_backward": [vp, vp, vp, vp, vp, vp, i32, i32, i32, i32, vp],
            "pog_solve_batch": [i32, ctypes.POINTER(pog_volume), opts, vp, i64p, ctypes.POINTER(vp)],
            "pog_solve_noalloc": [vp, i32, i32, i32, i32, i32, opts, vp, i64p, vp],
            "pog_solve_batch_f32": [i32, vp, f32, vp, i32, i32, i32, i32, i32, i32, opts, vp, i64p, i64p, vp],
            "pog_solve_batch_f32_hinge": [i32, vp, f32, vp, i32, i32, i32, i32, i32, i32, opts, vp, i64p, i64p, i64p,
                                          i64p, i64p, vp, vp],
            "pog_narrow_band": [vp, i32, i32, i32, vp, i32, i32, i32, i32, vp, vp, vp],
            "pog_band_heights": [vp, vp, i32, i32, i32, vp, vp],
            "pog_solve_convex": [vp, i32, i32, i32, i32, vp, opts, vp, i64p, i64p, vp, ctypes.POINTER(pog_stats_t)],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.pog_free.argtypes = [vp]
        lib.pog_free.restype = None
        lib.pog_strerror.argtypes = [ctypes.c_int]
        lib.pog_strerror.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != POG_OK:
        raise PogError(status, where)


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise PogError(POG_E_INVALID, f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise PogError(POG_E_INVALID, f"{name} must be a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def make_options(sweeps_per_relabel=0, max_rounds=0, tile_sweeps=0, flags=0, bfs_blocks_per_sm=0,
                 relabel_factor=0.0, tile_shape=0, bfs_bottom_up_ratio=0, test_wait_limit=0,
                 test_fail_alloc=0) -> pog_options:
    return pog_options(sweeps_per_relabel, max_rounds, tile_sweeps, flags, bfs_blocks_per_sm, relabel_factor,
                       tile_shape, bfs_bottom_up_ratio, test_wait_limit, test_fail_alloc)


def pog_strerror(status: int) -> str:
    try:
        return load().pog_strerror(int(status)).decode()
    except PogError:
        return f"status {status}"


class Graph:
    """Owner of one pog_graph handle (freed on close / garbage collection)."""

    def __init__(self, handle, shape, delta, alpha, keepalive=None):
        self.handle = handle
        self.shape = shape
        self.delta = delta
        self.alpha = alpha
        self._keep = keepalive

    def close(self):
        if self.handle:
            load().pog_free(self.handle)
            self.handle = None
            self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def pog_build(cost, delta: int, alpha: int, options: pog_options | None = None, stream=None) -> Graph:
    """cost: int32 CUDA tensor [X, Y, Z] (z fastest)."""
    import torch

    lib = load()
    ptr = _dev(cost, torch.int32, "cost")
    if cost.dim() != 3:
        raise PogError(POG_E_INVALID, "cost must be [X, Y, Z]")
    X, Y, Z = cost.shape
    h = ctypes.c_void_p()
    _check(lib.pog_build(ptr, X, Y, Z, int(delta), int(alpha), ctypes.byref(options) if options else None,
                         _stream(stream), ctypes.byref(h)), "pog_build")
    return Graph(h, (X, Y, Z), delta, alpha, keepalive=cost)


def pog_build_f32(cost, scale: float, delta: int, alpha: int, options: pog_options | None = None,
                  stream=None) -> Graph:
    """cost: float32 CUDA tensor [X, Y, Z]; quantised on the device to rint(scale * c)."""
    import torch

    lib = load()
    ptr = _dev(cost, torch.float32, "cost")
    if cost.dim() != 3:
        raise PogError(POG_E_INVALID, "cost must be [X, Y, Z]")
    X, Y, Z = cost.shape
    h = ctypes.c_void_p()
    _check(lib.pog_build_f32(ptr, float(scale), X, Y, Z, int(delta), int(alpha),
                             ctypes.byref(options) if options else None, _stream(stream), ctypes.byref(h)),
           "pog_build_f32")
    return Graph(h, (X, Y, Z), delta, alpha, keepalive=cost)


def pog_build_f32_augmented(cost, scale: float, h_aug, margin: int, delta: int, alpha: int,
                            options: pog_options | None = None, stream=None) -> Graph:
    """As pog_build_f32 with `margin` added at node (x, y, h_aug[x, y]) of every column."""
    import torch

    lib = load()
    ptr = _dev(cost, torch.float32, "cost")
    X, Y, Z = cost.shape
    h = ctypes.c_void_p()
    _check(lib.pog_build_f32_augmented(ptr, float(scale), _dev(h_aug, torch.int32, "h_aug"), int(margin), X, Y, Z,
                                       int(delta), int(alpha), ctypes.byref(options) if options else None,
                                       _stream(stream), ctypes.byref(h)), "pog_build_f32_augmented")
    return Graph(h, (X, Y, Z), delta, alpha, keepalive=(cost, h_aug))


def pog_energy(g: Graph) -> int:
    """Optimal energy E*(h) of the last pog_maxflow (from the flow identity)."""
    e = ctypes.c_int64(0)
    _check(load().pog_energy(g.handle, ctypes.byref(e)), "pog_energy")
    return int(e.value)


def pog_surface_energy(cost, scale: float, h, alpha: int, out=None, stream=None):
    """int64 [B] energies of surfaces h [B, X, Y] on quantised float costs [B, X, Y, Z]."""
    import torch

    B, X, Y, Z = cost.shape
    if out is None:
        out = torch.empty(B, dtype=torch.int64, device=cost.device)
    _check(load().pog_surface_energy(_dev(cost, torch.float32, "cost"), float(scale), _dev(h, torch.int32, "h"),
                                     B, X, Y, Z, int(alpha), _dev(out, torch.int64, "out"), _stream(stream)),
           "pog_surface_energy")
    return out


def pog_maxflow(g: Graph) -> int:
    flow = ctypes.c_int64(0)
    _check(load().pog_maxflow(g.handle, ctypes.byref(flow)), "pog_maxflow")
    return int(flow.value)


def pog_surface(g: Graph, heights=None):
    """Heights into an int32 CUDA tensor [X, Y] (allocated when not given)."""
    import torch

    if heights is None:
        heights = torch.empty(g.shape[:2], dtype=torch.int32, device="cuda")
    _check(load().pog_surface(g.handle, _dev(heights, torch.int32, "heights")), "pog_surface")
    return heights


def pog_stats(g: Graph) -> dict:
    s = pog_stats_t()
    _check(load().pog_stats(g.handle, ctypes.byref(s)), "pog_stats")
    return {n: getattr(s, n) for n, _ in pog_stats_t._fields_}


def pog_export_state(g: Graph) -> dict:
    """Host copies of the final residual state (numpy int32), see pog.h."""
    X, Y, Z = g.shape
    N = X * Y * Z
    out = {k: np.empty(N, dtype=np.int32) for k in ("excess", "sink", "fdown", "in_cut")}
    out["fhard"] = np.empty(4 * N, dtype=np.int32)
    out["gsoft"] = np.zeros(2 * N, dtype=np.int32)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    _check(load().pog_export_state(g.handle, p(out["excess"]), p(out["sink"]), p(out["fdown"]), p(out["fhard"]),
                                   p(out["gsoft"]) if g.alpha > 0 else None, p(out["in_cut"])), "pog_export_state")
    return out


def pog_trace(g: Graph, max_levels: int = 4096) -> np.ndarray:
    """int64 [levels, 3]: (frontier size, mode, device ns) per level of the last global relabel."""
    out = np.zeros(3 * max_levels, dtype=np.int64)
    n = ctypes.c_int32(0)
    _check(load().pog_trace(g.handle, ctypes.c_void_p(out.ctypes.data), max_levels, ctypes.byref(n)), "pog_trace")
    return out[: 3 * n.value].reshape(-1, 3)


def pog_free(g: Graph) -> None:
    g.close()


def pog_quantise(x, scale: float, out=None, stream=None):
    """int32 = round_half_even(scale * x) on the device; raises PogError on overflow."""
    import torch

    if out is None:
        out = torch.empty(x.shape, dtype=torch.int32, device=x.device)
    _check(load().pog_quantise(_dev(x, torch.float32, "x"), _dev(out, torch.int32, "out"), x.numel(),
                               float(scale), _stream(stream)), "pog_quantise")
    return out


def pog_backward(grad, h, g_energy, h_target=None, h_hat=None, g_hinge=None, stream=None):
    """grad float32 [B,X,Y,Z] <- g_energy[b]*onehot(h) + g_hinge[b]*(onehot(h_target) - onehot(h_hat))."""
    import torch

    B, X, Y, Z = grad.shape
    opt = lambda t, dt, n: None if t is None else _dev(t, dt, n)  # noqa: E731
    _check(load().pog_backward(_dev(grad, torch.float32, "grad"), _dev(h, torch.int32, "h"),
                               opt(h_target, torch.int32, "h_target"), opt(h_hat, torch.int32, "h_hat"),
                               _dev(g_energy, torch.float32, "g_energy"), opt(g_hinge, torch.float32, "g_hinge"),
                               B, X, Y, Z, _stream(stream)), "pog_backward")
    return grad


def pog_solve_batch(costs, deltas, alphas, options: pog_options | None = None, stream=None):
    """Solve a list of int32 CUDA volumes; returns (flows list, heights list)."""
    import torch

    n = len(costs)
    vols = (pog_volume * max(n, 1))()
    heights = []
    for i, c in enumerate(costs):
        X, Y, Z = c.shape
        vols[i] = pog_volume(_dev(c, torch.int32, f"costs[{i}]").value, X, Y, Z, int(deltas[i]), int(alphas[i]))
        heights.append(torch.empty((X, Y), dtype=torch.int32, device=c.device))
    hptrs = (ctypes.c_void_p * max(n, 1))(*[h.data_ptr() for h in heights])
    flows = (ctypes.c_int64 * max(n, 1))()
    _check(load().pog_solve_batch(n, vols, ctypes.byref(options) if options else None, _stream(stream), flows,
                                  hptrs), "pog_solve_batch")
    return [int(flows[i]) for i in range(n)], heights


def pog_solve_batch_f32(cost, scale: float, delta: int, alpha: int, h_aug=None, margin: int = 0,
                        options: pog_options | None = None, stream=None):
    """float32 CUDA [B, X, Y, Z] -> (flows list, energies list, heights int32 CUDA [B, X, Y])."""
    import torch

    B, X, Y, Z = cost.shape
    heights = torch.empty((B, X, Y), dtype=torch.int32, device=cost.device)
    flows = (ctypes.c_int64 * max(B, 1))()
    energies = (ctypes.c_int64 * max(B, 1))()
    _check(load().pog_solve_batch_f32(B, _dev(cost, torch.float32, "cost"), float(scale),
                                      None if h_aug is None else _dev(h_aug, torch.int32, "h_aug"), int(margin),
                                      X, Y, Z, int(delta), int(alpha), ctypes.byref(options) if options else None,
                                      _stream(stream), flows, energies, _dev(heights, torch.int32, "heights")),
           "pog_solve_batch_f32")
    return [int(flows[i]) for i in range(B)], [int(energies[i]) for i in range(B)], heights


def pog_solve_batch_f32_hinge(cost, scale: float, h_target, margin: int, delta: int, alpha: int,
                              options: pog_options | None = None, stream=None) -> dict:
    """Energy solve, loss-augmented solve and structured-hinge loss of float32 CUDA volumes
    [B, X, Y, Z] against target surfaces h_target (int32 CUDA [B, X, Y]); quantised units.
    Returns a dict: energies, aug_energies, hinge, flows, aug_flows (lists of int), heights,
    h_hat (int32 CUDA [B, X, Y])."""
    import torch

    if cost.dim() != 4:
        raise PogError(POG_E_INVALID, "cost must be [B, X, Y, Z]")
    B, X, Y, Z = cost.shape
    if tuple(h_target.shape) != (B, X, Y) or h_target.device != cost.device:
        raise PogError(POG_E_INVALID, "h_target must be an int32 tensor [B, X, Y] on the device of cost")
    heights = torch.empty((B, X, Y), dtype=torch.int32, device=cost.device)
    h_hat = torch.empty((B, X, Y), dtype=torch.int32, device=cost.device)
    arr = {k: (ctypes.c_int64 * max(B, 1))() for k in ("energies", "aug_energies", "hinge", "flows", "aug_flows")}
    _check(load().pog_solve_batch_f32_hinge(B, _dev(cost, torch.float32, "cost"), float(scale),
                                            _dev(h_target, torch.int32, "h_target"), int(margin), X, Y, Z, int(delta),
                                            int(alpha), ctypes.byref(options) if options else None, _stream(stream),
                                            arr["energies"], arr["aug_energies"], arr["hinge"], arr["flows"],
                                            arr["aug_flows"], _dev(heights, torch.int32, "heights"),
                                            _dev(h_hat, torch.int32, "h_hat")), "pog_solve_batch_f32_hinge")
    out = {k: [int(v[i]) for i in range(B)] for k, v in arr.items()}
    out["heights"] = heights
    out["h_hat"] = h_hat
    return out


def pog_narrow_band(cost, landmarks, stick: int, band_factor: int, outside_cost: int, stream=None):
    """Band cost volume int32 CUDA [X, Y, 2*half+1] and center surface int32 CUDA [X, Y] of
    an image cost volume [X, Y, Zi] around landmarks (int32 CUDA [L, 3] of x, y, z);
    half = stick * band_factor."""
    import torch

    if cost.dim() != 3 or landmarks.dim() != 2 or landmarks.shape[1] != 3 or landmarks.device != cost.device:
        raise PogError(POG_E_INVALID, "cost must be [X, Y, Zi] and landmarks [L, 3] on the same device")
    X, Y, Zi = cost.shape
    half = int(stick) * int(band_factor)
    band = torch.empty((X, Y, 2 * half + 1), dtype=torch.int32, device=cost.device)
    center = torch.empty((X, Y), dtype=torch.int32, device=cost.device)
    _check(load().pog_narrow_band(_dev(cost, torch.int32, "cost"), X, Y, Zi, _dev(landmarks, torch.int32, "landmarks"),
                                  landmarks.shape[0], int(stick), int(band_factor), int(outside_cost), _stream(stream),
                                  _dev(band, torch.int32, "band"), _dev(center, torch.int32, "center")),
           "pog_narrow_band")
    return band, center


def pog_band_heights(h_band, center, half: int, out=None, stream=None):
    """Image heights center - half + h_band (int32 CUDA [X, Y])."""
    import torch

    if tuple(h_band.shape) != tuple(center.shape) or h_band.dim() != 2:
        raise PogError(POG_E_INVALID, "h_band and center must both be [X, Y]")
    X, Y = center.shape
    if out is None:
        out = torch.empty((X, Y), dtype=torch.int32, device=center.device)
    _check(load().pog_band_heights(_dev(h_band, torch.int32, "h_band"), _dev(center, torch.int32, "center"), X, Y,
                                   int(half), _stream(stream), _dev(out, torch.int32, "out")), "pog_band_heights")
    return out


def pog_solve_noalloc(cost, delta: int, alpha: int, heights, options: pog_options | None = None, stream=None) -> int:
    """Whole solve with the library's fixed scratch array (no allocation inside the call);
    `heights` is a caller-owned int32 CUDA tensor [X, Y]. Returns the flow value."""
    import torch

    if not isinstance(cost, torch.Tensor) or cost.dim() != 3:
        raise PogError(POG_E_INVALID, "cost must be a CUDA tensor [X, Y, Z]")
    X, Y, Z = cost.shape
    # the library writes X*Y heights through this pointer and cannot check its size
    if (not isinstance(heights, torch.Tensor) or tuple(heights.shape) != (X, Y)
            or heights.device != cost.device):
        raise PogError(POG_E_INVALID, "heights must be an int32 tensor [X, Y] on the device of cost")
    flow = ctypes.c_int64(0)
    _check(load().pog_solve_noalloc(_dev(cost, torch.int32, "cost"), X, Y, Z, int(delta), int(alpha),
                                    ctypes.byref(options) if options else None, _stream(stream), ctypes.byref(flow),
                                    _dev(heights, torch.int32, "heights")), "pog_solve_noalloc")
    return int(flow.value)


def pog_solve_convex(cost, delta: int, f, heights=None, options: pog_options | None = None, stream=None):
    """Solve with the convex pairwise cost f (f[d-1] = f(d), d = 1..delta, f(0) = 0).
    Returns (flow, energy, heights, stats): the max-flow value, E*(h), the int32 CUDA
    tensor [X, Y] of the minimal cut's surface and the solve's counters (dict)."""
    import torch

    if not isinstance(cost, torch.Tensor) or cost.dim() != 3:
        raise PogError(POG_E_INVALID, "cost must be a CUDA tensor [X, Y, Z]")
    X, Y, Z = cost.shape
    fa = np.ascontiguousarray(np.asarray(f if f is not None else [], dtype=np.int64).reshape(-1))
    if fa.size != int(delta):
        raise PogError(POG_E_INVALID, "f must hold f(1..delta)")
    if heights is None:
        heights = torch.empty((X, Y), dtype=torch.int32, device=cost.device)
    elif (not isinstance(heights, torch.Tensor) or tuple(heights.shape) != (X, Y)
            or heights.device != cost.device):
        raise PogError(POG_E_INVALID, "heights must be an int32 tensor [X, Y] on the device of cost")
    flow, energy, st = ctypes.c_int64(0), ctypes.c_int64(0), pog_stats_t()
    fptr = ctypes.c_void_p(fa.ctypes.data) if fa.size else None
    _check(load().pog_solve_convex(_dev(cost, torch.int32, "cost"), X, Y, Z, int(delta), fptr,
                                   ctypes.byref(options) if options else None, _stream(stream), ctypes.byref(flow),
                                   ctypes.byref(energy), _dev(heights, torch.int32, "heights"), ctypes.byref(st)),
           "pog_solve_convex")
    return int(flow.value), int(energy.value), heights, {n: getattr(st, n) for n, _ in pog_stats_t._fields_}


def solve(cost, delta: int, alpha: int, options: pog_options | None = None, stream=None):
    """Max-flow value (int) and surface heights (int32 CUDA tensor [X, Y]) of one volume."""
    with pog_build(cost, delta, alpha, options, stream) as g:
        flow = pog_maxflow(g)
        return flow, pog_surface(g)
