"""Host logic of bench.py's opt-in sweeps (separator size, merging), run
through a stand-in for the library binding that returns fixed device times:
the rows, the launch count of the per-message path and the launch-overhead
shares.  CPU only; the device times themselves come from the GPU runs."""
import sys
import types

import numpy as np
import pytest

import paper_1202_3777_gb300


class _Handle:
    class info:
        depth = 3

    def free(self):
        pass


@pytest.fixture
def fake_jt(monkeypatch):
    fake = types.ModuleType("paper_1202_3777_gb300.jt")
    fake.JT_F32, fake.JT_OK, fake.JT_MATERIALIZE_CLIQUES = 0, 0, 1
    fake.jt_load_synth = lambda t, **k: _Handle()
    fake.jt_load_tree = lambda *a, **k: _Handle()
    fake.jt_init_from_cpts = lambda *a, **k: 0.1
    fake.jt_profile_propagate = lambda h, a, b: np.array([0.25, 0.05], np.float32)
    fake.jt_get_status = lambda h, a, b: np.zeros(1, np.int32)
    # per-message time: 1 ms on the floor tree, 10 ms on the others
    fake.jt_propagate_per_message = lambda h, c, layout: 1.0 if getattr(h, "floor", False) else 10.0
    monkeypatch.setitem(sys.modules, "paper_1202_3777_gb300.jt", fake)
    monkeypatch.setattr(paper_1202_3777_gb300, "jt", fake, raising=False)
    return fake


def test_separator_sweep_rows_and_shares(fake_jt):
    import bench
    floor = {"n": 0}

    def load(t, **k):
        h = _Handle()
        h.floor = floor["n"] == 0          # the first tree loaded is the floor tree
        floor["n"] += 1
        return h
    fake_jt.jt_load_synth = load
    out = bench.separator_sweep()
    rows = out["rows"]
    assert [r["avg_separator_entries"] for r in rows] == [2.0] + [4.0 ** s for s in range(1, 8)]
    assert all(r["launches_per_message_path"] == 4 * 31 + 8 for r in rows)
    assert out["tau_us"] == pytest.approx(1e3 * 1.0 / (4 * 31 + 8))
    assert rows[0]["launch_overhead_share"] == pytest.approx(1.0)
    assert all(r["launch_overhead_share"] == pytest.approx(0.1) for r in rows[1:])
    assert all(r["fused_ms"] == pytest.approx(0.3) for r in rows)


def test_merging_sweep_rows(fake_jt):
    import bench
    rows = bench.merging_sweep()["rows"]
    small = [r for r in rows if r["tree"].startswith("small")]
    binary = [r for r in rows if r["tree"].startswith("binary")]
    assert [r["cliques"] for r in small] == [32, 22]
    assert binary[0]["cliques"] == 1024 and all(r["cliques"] < 1024 for r in binary[1:])
    assert [r["cliques"] for r in binary[1:]] == sorted((r["cliques"] for r in binary[1:]), reverse=True)
