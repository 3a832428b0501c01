"""Host logic of the tuned-parameter table (no GPU)."""
import json

from paper_2601_17026_gb300 import autotune


def test_exact_nearest_and_default(tmp_path):
    path = tmp_path / "tuned.json"
    table = {
        "512x512x384/d3/a50": {"params": {"tile_shape": 1, "tile_sweeps": 16}},
        "64x64x64/d3/a50": {"params": {"tile_shape": 2}},
        "256x256x256/d2/a0": {"params": {"tile_shape": 3}},
        "garbage": {"params": {"tile_shape": 0}},
    }
    path.write_text(json.dumps(table))
    exact = autotune.tuned_params(512, 512, 384, 3, 50, path=str(path))
    assert exact["tile_shape"] == 1 and exact["tile_sweeps"] == 16
    assert exact["bfs_blocks_per_sm"] == autotune.DEFAULTS["bfs_blocks_per_sm"]
    # closest node count (in ratio) among the same (delta, alpha)
    assert autotune.tuned_params(256, 256, 384, 3, 50, path=str(path))["tile_shape"] == 1
    assert autotune.tuned_params(48, 48, 64, 3, 50, path=str(path))["tile_shape"] == 2
    # no class with this delta and alpha: defaults
    assert autotune.tuned_params(256, 256, 384, 2, 50, path=str(path)) == autotune.DEFAULTS
    # missing table: defaults
    assert autotune.tuned_params(8, 8, 8, 1, 0, path=str(tmp_path / "none.json")) == autotune.DEFAULTS


def test_batch_params(tmp_path):
    path = tmp_path / "tuned.json"
    path.write_text(json.dumps({"batch/uneven-64": {"params": {"tile_sweeps": 16}},
                                "512x512x384/d3/a50": {"params": {"tile_shape": 1}}}))
    got = autotune.batch_params("uneven-64", path=str(path))
    assert got["tile_sweeps"] == 16 and got["tile_shape"] == autotune.DEFAULTS["tile_shape"]
    assert autotune.batch_params("other", path=str(path)) == autotune.DEFAULTS
    # the batch entry is not a volume class: the nearest-class lookup skips it
    assert autotune.tuned_params(256, 256, 384, 3, 50, path=str(path))["tile_shape"] == 1


def test_coordinate_descent_keeps_the_fastest(monkeypatch):
    """tune() walks SPACE one parameter at a time from DEFAULTS and keeps a change only when
    it is faster; a candidate that changes the flow value is an error."""
    cost_of = {"tile_sweeps": {16: -0.3, 32: -0.1}, "tile_shape": {1: -0.2}, "bfs_blocks_per_sm": {2: +0.5}}

    def fake_time(cost, delta, alpha, params, repeats):
        t = 1.0
        for name, table in cost_of.items():
            t += table.get(params[name], 0.0)
        return t, 12345

    monkeypatch.setattr(autotune, "_time_solve", fake_time)
    out = autotune.tune(None, 3, 50, log=lambda *_: None)
    assert out["params"]["tile_sweeps"] == 16 and out["params"]["tile_shape"] == 1
    assert out["params"]["bfs_blocks_per_sm"] == autotune.DEFAULTS["bfs_blocks_per_sm"]
    assert abs(out["seconds"] - 0.5) < 1e-9

    def wrong_flow(cost, delta, alpha, params, repeats):
        return 1.0, 1 if params == autotune.DEFAULTS else 2

    monkeypatch.setattr(autotune, "_time_solve", wrong_flow)
    import pytest

    with pytest.raises(RuntimeError):
        autotune.tune(None, 3, 50, log=lambda *_: None)
