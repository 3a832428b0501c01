"""Write the stored expected values under tests/golden/ with the CPU oracle only.

    python tests/golden/make_golden.py small      # seconds
    python tests/golden/make_golden.py medium     # about an hour on one core
    python tests/golden/make_golden.py batch [K]  # the first K volumes of the uneven batch
    python tests/golden/make_golden.py diff [W]   # the 16 float volumes of 128^3, W threads
    python tests/golden/make_golden.py convex     # convex pairwise costs, two mid-size volumes
    python tests/golden/make_golden.py band       # the benchmark's narrow band (about an hour)

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


def record_diff(args):
    """One volume of the differentiable workload: the energy solve and the loss-augmented
    solve of the structured hinge, on the quantised costs round_half_even(1024 * c)."""
    b, fc, ht = args
    t = time.time()
    scale, aq, mq = 1024.0, int(synth.DIFF_ALPHA * 1024), int(synth.DIFF_MARGIN * 1024)
    cq = np.rint(fc.astype(np.float64) * scale).astype(np.int32)  # exact: x1024 is exact in fp32
    X, Y, Z = cq.shape
    ref = oracle.solve(cq, synth.DIFF_DELTA, aq)
    e, ok = oracle.energy(cq, ref.heights, synth.DIFF_DELTA, aq)
    assert ok
    aug = cq.copy()
    idx = ht[:, :, None]
    np.put_along_axis(aug, idx, np.take_along_axis(cq, idx, 2) + mq, axis=2)
    ra = oracle.solve(aug, synth.DIFF_DELTA, aq)
    ea, ok = oracle.energy(aug, ra.heights, synth.DIFF_DELTA, aq)
    assert ok
    et, ok = oracle.energy(cq, ht, synth.DIFF_DELTA, aq)
    assert ok
    h = np.ascontiguousarray(ref.heights, dtype=np.int32)
    hh = np.ascontiguousarray(ra.heights, dtype=np.int32)
    return {"volume": b, "shape": [X, Y, Z], "delta": synth.DIFF_DELTA, "alpha_q": aq, "margin_q": mq,
            "flow": ref.flow, "energy": e, "heights_sha256": hashlib.sha256(h.tobytes()).hexdigest(),
            "heights_sum": int(h.sum()), "aug_flow": ra.flow, "aug_energy": ea,
            "aug_heights_sha256": hashlib.sha256(hh.tobytes()).hexdigest(), "aug_heights_sum": int(hh.sum()),
            "target_energy": et, "hinge_q": et - (ea - mq * X * Y),
            "oracle_seconds": round(time.time() - t, 1)}


def record_convex(shape):
    """One volume of the convex workload (edge interval of 10, f(t) = 4 t^2)."""
    X, Y, Z = shape
    cost = synth.convex_cost(X, Y, Z)
    f = synth.convex_profile()
    t = time.time()
    r = oracle.solve_convex(cost, synth.CONVEX_DELTA, f)
    e, ok = oracle.energy_convex(cost, r.heights, synth.CONVEX_DELTA, f)
    assert ok
    h = np.ascontiguousarray(r.heights, dtype=np.int32)
    return {"shape": [X, Y, Z], "delta": synth.CONVEX_DELTA, "f": [int(v) for v in f], "flow": r.flow,
            "energy": e, "heights_sha256": hashlib.sha256(h.tobytes()).hexdigest(), "heights_sum": int(h.sum()),
            "oracle_seconds": round(time.time() - t, 1)}


def record_band():
    """The narrow band of the 512x512x384 volume around its 64 landmarks (stick 16, band
    factor 2): band volume and center surface from oracle/band.py, then the band's solve."""
    from oracle import band as oband

    spec = synth.spec_seismic()
    cost = synth.horizon_cost(spec)
    lm = synth.horizon_landmarks(spec, 8)
    half = synth.BAND_STICK * synth.BAND_FACTOR
    rb, rc = oband.narrow_band(cost, lm, synth.BAND_STICK, synth.BAND_FACTOR, synth.BAND_OUTSIDE)
    t = time.time()
    r = oracle.solve(rb, 3, 50)
    hb = np.ascontiguousarray(r.heights, dtype=np.int32)
    himg = np.ascontiguousarray(oband.band_heights(hb, rc, half), dtype=np.int32)
    sha = lambda a: hashlib.sha256(np.ascontiguousarray(a, dtype=np.int32).tobytes()).hexdigest()  # noqa: E731
    return {"workload": "narrow band of the 512x512x384 volume (delta 3, alpha 50): 64 landmarks "
                        "(synth.horizon_landmarks, 8x8), stick 16, band factor 2, outside cost 1200",
            "oracle": "oracle/band.py construction; explicit-edge Dinic (oracle/pog_oracle.c)",
            "generator": f"paper_2601_17026_gb300.synth, seed {synth.BASE_SEED}",
            "band_shape": list(rb.shape), "band_sha256": sha(rb), "center_sha256": sha(rc),
            "flow": r.flow, "heights_sha256": sha(hb), "heights_sum": int(hb.sum()),
            "image_heights_sha256": sha(himg), "oracle_seconds": round(time.time() - t, 1)}


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
    elif which == "diff":
        from concurrent.futures import ThreadPoolExecutor

        workers = int(sys.argv[2]) if len(sys.argv) > 2 else 1
        fc = synth.diff_volumes_f32()
        ht = synth.diff_target()
        with ThreadPoolExecutor(workers) as ex:
            vols = list(ex.map(record_diff, [(b, fc[b], ht[b]) for b in range(fc.shape[0])]))
        data = {"workload": "16 float32 volumes of 128^3, N(0,1) + horizon pattern, quantised by 1024; "
                            "hinge target flat at height 64, margin 1024",
                "oracle": "explicit-edge Dinic (oracle/pog_oracle.c)",
                "generator": f"paper_2601_17026_gb300.synth, seed {synth.BASE_SEED}", "volumes": vols}
    elif which == "band":
        data = record_band()
    elif which == "convex":
        data = {"workload": "layered-horizon volumes (synth.convex_cost), convex pairwise cost f(t) = 4 t^2, "
                            "delta 9 (edge interval of 10)",
                "oracle": "explicit-edge Dinic on the layered graph (oracle/pog_oracle.c)",
                "generator": f"paper_2601_17026_gb300.synth, seed {synth.BASE_SEED}",
                "volumes": [record_convex(s) for s in [(64, 64, 128), (80, 48, 96)]]}
    else:
        raise SystemExit(f"unknown set {which}")
    path = os.path.join(HERE, f"{which}.json")
    with open(path, "w") as f:
        json.dump(data, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
