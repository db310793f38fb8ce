"""The autotune cache of the binding (a JSON file of launch shapes keyed by
grid, FC, kernel, precision, scheme and device): store and reload, a hit
applies the stored shape without timing anything, and the key separates
contexts that differ in any of those.  Host logic only: the context is a
stand-in with the binding's own key and cache methods."""
import pytest

b = pytest.importorskip("paper_2606_06247_gb300.binding")


class StandIn(b.Context):
    def __init__(self, nx, ny, batch, prec, n_cont=25):
        # the binding's parameter structs, no library context
        self.grid = b.fcsph_grid(nx, ny, 1.0, 1.0, 1, batch, 1, 0.0)
        self.fc = b.fcsph_fc(b.FC_GRAM, 5, n_cont, 0)
        self.kernel = b.fcsph_kernel(b.FAMILY["G8"], 1.3)
        self.prec = b.fcsph_precision(b.PREC[prec], 0)
        self.h = None
        self.applied = None
        self.tuned = 0

    def apply_tune_state(self, st):
        self.applied = st

    def tune_state(self):
        return {"tiling": [1, 1], "cta_threads": [32, 64], "groups": 2, "persistent": False}

    def get_tiling(self):
        return tuple(self.applied["tiling"]) if self.applied else (1, 1)

    def _params(self, *a):
        return b.fcsph_step_params()


def test_cache_round_trip_and_hit(tmp_path, monkeypatch):
    path = str(tmp_path / "tune.json")
    assert b.load_tune_cache(path) == {}
    calls = []
    monkeypatch.setattr(b.lib, "fcsph_autotune", lambda *a: calls.append(a) or 0, raising=False)
    ctx = StandIn(256, 256, 32, "f32x2")
    r, c, ms = ctx.autotune(steps=2, cache=path, device_name="GB300")
    assert len(calls) == 1 and ms is not None
    stored = b.load_tune_cache(path)
    assert list(stored.values()) == [ctx.tune_state()]
    again = StandIn(256, 256, 32, "f32x2")
    r, c, ms = again.autotune(steps=2, cache=path, device_name="GB300")
    assert len(calls) == 1 and ms is None and again.applied == ctx.tune_state()


def test_cache_key_separates_contexts():
    base = StandIn(256, 256, 32, "f32x2").tune_key("rk3", "GB300")
    others = [StandIn(256, 256, 16, "f32x2").tune_key("rk3", "GB300"),
              StandIn(256, 256, 32, "f64").tune_key("rk3", "GB300"),
              StandIn(256, 256, 32, "f32x2", n_cont=24).tune_key("rk3", "GB300"),
              StandIn(128, 256, 32, "f32x2").tune_key("rk3", "GB300"),
              StandIn(256, 256, 32, "f32x2").tune_key("fop", "GB300"),
              StandIn(256, 256, 32, "f32x2").tune_key("rk3", "B200")]
    assert len(set(others + [base])) == len(others) + 1


def test_unreadable_cache_is_empty(tmp_path):
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    assert b.load_tune_cache(str(p)) == {}
