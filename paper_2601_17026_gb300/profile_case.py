"""A short, fixed-size run of the solver for profiler captures.

    python -m paper_2601_17026_gb300.profile_case --workload seismic-crop --sweeps 1

Builds one volume with its tuned options and runs the initial global relabel, `--sweeps`
tiled sweeps and a second global relabel, then stops (the round cap is reached on
purpose). It prints one JSON line with the volume's node count and the tile visits of
those sweeps, so that a capture of the first tile-kernel launch (`--sweeps 1`) or of a
global relabel can be divided by the units of work it processed. The result of the
solve is not used.

The convex workloads (``convex``: 256x256x128, ``convex-crop``: 128x128x128; delta 9,
f(t) = 4 t^2) run pog_solve_convex the same way: a global relabel, `--sweeps` node sweeps
and a second relabel; the line gives the active nodes listed by those sweeps.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="seismic-crop",
                    choices=["seismic", "seismic-crop", "medium", "convex", "convex-crop"])
    ap.add_argument("--sweeps", type=int, default=1)
    args = ap.parse_args()

    import torch

    import __graft_entry__
    from paper_2601_17026_gb300 import autotune, pog, synth

    __graft_entry__.build()
    torch.cuda.set_device(0)
    if args.workload.startswith("convex"):
        shape = synth.CONVEX_SHAPE if args.workload == "convex" else (128, 128, 128)
        cost = torch.from_numpy(synth.convex_cost(*shape)).cuda()
        import ctypes

        import numpy as np

        opts = pog.make_options(max_rounds=2, sweeps_per_relabel=args.sweeps)
        f = np.ascontiguousarray(synth.convex_profile(), dtype=np.int64)
        heights = torch.empty(shape[:2], dtype=torch.int32, device="cuda")
        flow, energy, st = ctypes.c_int64(0), ctypes.c_int64(0), pog.pog_stats_t()
        # the C call directly: its counters are filled also when the round cap stops it
        rc = pog.load().pog_solve_convex(ctypes.c_void_p(cost.data_ptr()), *shape, synth.CONVEX_DELTA,
                                         ctypes.c_void_p(f.ctypes.data), ctypes.byref(opts),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                         ctypes.byref(flow), ctypes.byref(energy),
                                         ctypes.c_void_p(heights.data_ptr()), ctypes.byref(st))
        if rc not in (pog.POG_OK, pog.POG_E_NOCONVERGE):
            raise pog.PogError(rc, "pog_solve_convex")
        torch.cuda.synchronize()
        print(json.dumps({"workload": f"{shape} delta {synth.CONVEX_DELTA} f(t) = 4 t^2", "nodes": int(cost.numel()),
                          "status": "converged" if rc == pog.POG_OK else "stopped after two global relabels",
                          "sweeps": st.sweeps, "listed_nodes": st.tiles_visited, "bfs_levels": st.bfs_passes,
                          "rounds": st.rounds}), flush=True)
        return
    vol = {"seismic": synth.seismic_volume, "seismic-crop": synth.seismic_crop,
           "medium": synth.medium_volume}[args.workload]()
    X, Y, Z = vol.cost.shape
    params = autotune.tuned_params(X, Y, Z, vol.delta, vol.alpha)
    params["sweeps_per_relabel"] = args.sweeps
    opts = pog.make_options(max_rounds=2, **params)
    cost = torch.from_numpy(vol.cost).cuda()
    with pog.pog_build(cost, vol.delta, vol.alpha, opts) as g:
        try:
            pog.pog_maxflow(g)
            status = "converged"
        except pog.PogError as e:
            if e.status != pog.POG_E_NOCONVERGE:
                raise
            status = "stopped after two global relabels"
        st = pog.pog_stats(g)
    torch.cuda.synchronize()
    print(json.dumps({"workload": vol.name, "nodes": vol.n, "sweeps": st["sweeps"], "rounds": st["rounds"],
                      "tiles_visited": st["tiles_visited"], "bfs_levels": st["bfs_passes"], "status": status,
                      "params": params}), flush=True)


if __name__ == "__main__":
    main()
