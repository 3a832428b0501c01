"""A short, fixed-size run of the solver for profiler captures.

    python -m paper_2601_17026_gb300.profile_case --workload seismic-crop --sweeps 1

Builds one volume with its tuned options and runs the initial global relabel, `--sweeps`
tiled sweeps and a second global relabel, then stops (the round cap is reached on
purpose). It prints one JSON line with the volume's node count and the tile visits of
those sweeps, so that a capture of the first tile-kernel launch (`--sweeps 1`) or of a
global relabel can be divided by the units of work it processed. The result of the
solve is not used.
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
    ap.add_argument("--workload", default="seismic-crop", choices=["seismic", "seismic-crop", "medium"])
    ap.add_argument("--sweeps", type=int, default=1)
    args = ap.parse_args()

    import torch

    import __graft_entry__
    from paper_2601_17026_gb300 import autotune, pog, synth

    __graft_entry__.build()
    torch.cuda.set_device(0)
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
