"""Write the stored expected values under tests/golden/ with the CPU oracle only.

    python tests/golden/make_golden.py small      # seconds
    python tests/golden/make_golden.py medium     # about an hour on one core
    python tests/golden/make_golden.py batch [K]  # the first K volumes of the uneven batch

Each file records the workload, the oracle's max-flow value and its surface (in full for
the small volume; as a SHA-256 of the int32 heights plus their sum otherwise). Nothing
here touches the CUDA path.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2601_17026_gb300 import synth  # noqa: E402


def record(vol, full_heights=False):
    t = time.time()
    r = oracle.solve(vol.cost, vol.delta, vol.alpha)
    h = np.ascontiguousarray(r.heights, dtype=np.int32)
    out = {"workload": vol.name, "shape": list(vol.cost.shape), "delta": vol.delta, "alpha": vol.alpha,
           "flow": r.flow, "heights_sha256": hashlib.sha256(h.tobytes()).hexdigest(), "heights_sum": int(h.sum()),
           "oracle": "explicit-edge Dinic (oracle/pog_oracle.c)", "oracle_seconds": round(time.time() - t, 1),
           "generator": f"paper_2601_17026_gb300.synth, seed {synth.BASE_SEED}"}
    if full_heights:
        out["heights"] = h.tolist()
    return out


def main():
    which = sys.argv[1] if len(sys.argv) > 1 else "small"
    if which == "small":
        data = record(synth.small_volume(), full_heights=True)
    elif which == "medium":
        data = record(synth.medium_volume())
    elif which == "batch":
        from concurrent.futures import ThreadPoolExecutor

        k = int(sys.argv[2]) if len(sys.argv) > 2 else 64
        workers = int(sys.argv[3]) if len(sys.argv) > 3 else 1
        vols = synth.batch_volumes(limit=k)
        with ThreadPoolExecutor(workers) as ex:  # the oracle releases the GIL inside C
            data = {"volumes": list(ex.map(record, vols))}
    else:
        raise SystemExit(f"unknown set {which}")
    path = os.path.join(HERE, f"{which}.json")
    with open(path, "w") as f:
        json.dump(data, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
