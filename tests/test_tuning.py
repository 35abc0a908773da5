"""The grouped contraction's tile table (tuning.py): the committed table is well formed (every
bucket's choice is one of the timed shapes and the fastest of them), the buckets follow the start
counts, and `choose` reads the table or falls back to the library's default.  The timing itself
(`tune`) needs a GPU and runs in `bench.py --tune`; here a fake group stands in for it."""
import json

from paper_1212_4137_gb300 import tuning


def test_committed_table_is_well_formed():
    table = tuning.load_table()
    assert table.get("buckets"), "the measured table is committed beside tuning.py"
    shapes = {f"{n},{s}" for n, s in tuning.TILE_SHAPES}
    for name, entry in table["buckets"].items():
        assert name in ("r<=16", "r<=64", "r<=256", "r>256")
        assert set(entry["ms"]) <= shapes and entry["ms"]
        best = min(entry["ms"], key=entry["ms"].get)
        assert entry["choice"] == [int(t) for t in best.split(",")]


def test_buckets_and_choose(tmp_path):
    assert [tuning.bucket(r) for r in (1, 16, 17, 64, 65, 256, 257)] == \
        ["r<=16", "r<=16", "r<=64", "r<=64", "r<=256", "r<=256", "r>256"]
    table = {"buckets": {"r<=64": {"ms": {"64,4": 1.0, "128,3": 2.0}, "choice": [64, 4]}}}
    assert tuning.choose(40, table) == (64, 4)
    assert tuning.choose(200, table) is None          # a bucket the table lacks: the default
    path = tmp_path / "t.json"
    path.write_text(json.dumps(table))
    assert tuning.load_table(str(path)) == table
    assert tuning.load_table(str(tmp_path / "missing.json")) == {}


def test_tune_times_every_shape_and_picks_the_fastest(monkeypatch):
    import sys
    import types

    class FakeTorchCuda:
        @staticmethod
        def synchronize():
            pass

    monkeypatch.setitem(sys.modules, "torch", types.SimpleNamespace(cuda=FakeTorchCuda))
    cost = {(64, 2): 0.004, (64, 3): 0.003, (64, 4): 0.002, (128, 2): 0.005, (128, 3): 0.006}
    calls = []

    class FakeGroup:
        def solve(self, problems, tiles=None):
            calls.append(tiles)
            import time
            time.sleep(cost[tiles])

    out = tuning.tune(FakeGroup(), [("p",)], reps=2)
    assert set(out["ms"]) == {f"{n},{s}" for n, s in tuning.TILE_SHAPES}
    assert out["choice"] == [64, 4]
    assert len(calls) == 3 * len(tuning.TILE_SHAPES)   # a warm-up and two timed solves per shape
