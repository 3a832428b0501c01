"""Autotuner for the solver's launch parameters.

Picks, per volume class (shape, delta, alpha), the sweeps per global relabel (fixed, or
adaptive with a relabel factor: sweep time per round against global-relabel time), the
tile shape, the local sweeps per tile visit, the BFS
grid (resident blocks per SM) and the BFS frontier mode (bottom-up threshold) by timing
whole solves through the C ABI: coordinate descent from the defaults, best of
`repeats` solves per candidate (the push schedule is nondeterministic, so single timings
are noisy). Results are kept in ``tuned.json`` beside this file.

    python -m paper_2601_17026_gb300.autotune --workload seismic
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TUNED_PATH = os.path.join(HERE, "tuned.json")

SPACE = {
    "sweeps_per_relabel": [0, 32, 64, 128],  # 0: adaptive (relabel_factor)
    "tile_shape": [0, 1, 2, 3],
    "tile_sweeps": [4, 8, 16, 32],
    "relabel_factor": [0.5, 1.0, 2.0, 4.0],
    "bfs_blocks_per_sm": [1, 2, 4],
    "bfs_bottom_up_ratio": [4, 8, 16, -1],
}
DEFAULTS = {"sweeps_per_relabel": 0, "tile_shape": 0, "tile_sweeps": 8, "relabel_factor": 1.0,
            "bfs_blocks_per_sm": 4, "bfs_bottom_up_ratio": 8}


def volume_key(X: int, Y: int, Z: int, delta: int, alpha: int) -> str:
    return f"{X}x{Y}x{Z}/d{delta}/a{alpha}"


def load_table(path: str = TUNED_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tuned_params(X, Y, Z, delta, alpha, path: str = TUNED_PATH) -> dict:
    """Tuned parameters for this volume class; else those of the tuned class with the same
    delta and alpha whose node count is closest in ratio; else the defaults."""
    table = load_table(path)
    entry = table.get(volume_key(X, Y, Z, delta, alpha))
    if entry is None:
        n = X * Y * Z
        near = []
        for key, e in table.items():
            try:
                shape, d, a = key.split("/")
                dims = [int(v) for v in shape.split("x")]
            except ValueError:
                continue
            if d == f"d{delta}" and a == f"a{alpha}" and len(dims) == 3:
                near.append((abs(math.log(dims[0] * dims[1] * dims[2] / n)), key))
        if near:
            entry = table[min(near)[1]]
    params = dict(DEFAULTS)
    if entry:
        params.update(entry["params"])
    return params


def batch_params(name: str = "uneven-64", path: str = TUNED_PATH) -> dict:
    """Parameters recorded for a batched workload (key ``batch/<name>``), else the defaults."""
    params = dict(DEFAULTS)
    entry = load_table(path).get(f"batch/{name}")
    if entry:
        params.update(entry["params"])
    return params


def options_for(X, Y, Z, delta, alpha, flags: int = 0, path: str = TUNED_PATH):
    from . import pog

    return pog.make_options(flags=flags, **tuned_params(X, Y, Z, delta, alpha, path))


def _time_solve(cost, delta, alpha, params, repeats):
    import torch

    from . import pog

    best = float("inf")
    flow = None
    for _ in range(repeats):
        torch.cuda.synchronize()
        t = time.perf_counter()
        f, _ = pog.solve(cost, delta, alpha, pog.make_options(**params))
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t)
        if flow is not None and f != flow:
            raise RuntimeError("solves with different parameters disagree")
        flow = f
    return best, flow


def tune(cost, delta: int, alpha: int, repeats: int = 2, passes: int = 1, log=print) -> dict:
    """Coordinate descent over SPACE from DEFAULTS; returns the best parameters found."""
    params = dict(DEFAULTS)
    best, flow0 = _time_solve(cost, delta, alpha, params, repeats)
    log(f"defaults: {best:.3f} s")
    for _ in range(passes):
        for name, values in SPACE.items():
            for v in values:
                if v == params[name]:
                    continue
                trial = dict(params, **{name: v})
                t, flow = _time_solve(cost, delta, alpha, trial, repeats)
                if flow != flow0:
                    raise RuntimeError(f"{trial} changed the flow value")
                log(f"{name}={v}: {t:.3f} s")
                if t < best:
                    best, params = t, trial
    log(f"best {params}: {best:.3f} s")
    return {"params": params, "seconds": round(best, 4)}


def main():
    import torch

    from . import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="seismic", choices=["seismic", "medium", "small"])
    ap.add_argument("--repeats", type=int, default=2)
    ap.add_argument("--out", default=TUNED_PATH)
    args = ap.parse_args()
    vol = {"seismic": synth.seismic_volume, "medium": synth.medium_volume, "small": synth.small_volume}[args.workload]()
    cost = torch.from_numpy(vol.cost).cuda()
    X, Y, Z = vol.cost.shape
    result = tune(cost, vol.delta, vol.alpha, repeats=args.repeats)
    result["device"] = torch.cuda.get_device_name()
    table = load_table(args.out)
    table[volume_key(X, Y, Z, vol.delta, vol.alpha)] = result
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print(json.dumps(result))


if __name__ == "__main__":
    main()
