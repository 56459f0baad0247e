"""Context.checkpoint() / restore() and their Ising counterparts on the host, with the C calls
faked (no GPU): what a checkpoint holds, the order in which restore() loads it (spins, widths
where the sample adapts, then the MCS counter) and the refusal of a checkpoint of another
shape. The GPU side of resuming is tests/test_gpu_resume.py."""

import numpy as np
import pytest

from paper_1803_07030_gb300 import vegas as vb


@pytest.fixture
def fake_ctx(monkeypatch):
    calls = []
    state = {"spins": {i: np.full((5, 3), float(i)) for i in range(4)}, "mcs": 40,
             "widths": np.array([0.0, 0.3, 0.0, 0.7])}
    monkeypatch.setattr(vb, "vegas_get_spins", lambda ptr, inst, n: state["spins"][inst].copy())
    monkeypatch.setattr(vb, "vegas_set_spins", lambda ptr, inst, x: calls.append(("spins", inst, np.array(x))))
    monkeypatch.setattr(vb, "vegas_stats", lambda ptr: {"mcs_done": state["mcs"]})
    monkeypatch.setattr(vb, "vegas_adaptive_width", lambda ptr, n: state["widths"].copy())
    monkeypatch.setattr(vb, "vegas_set_adaptive_width", lambda ptr, w: calls.append(("widths", np.array(w))))
    monkeypatch.setattr(vb, "vegas_set_mcs_counter", lambda ptr, t: calls.append(("mcs", t)))
    c = object.__new__(vb.Context)
    c.samples, c.replicas, c.n_sites, c.ptr = [object(), object()], 2, [5, 5], 1
    yield c, calls
    c.ptr = None


def test_checkpoint_holds_spins_counter_and_widths(fake_ctx):
    c, _ = fake_ctx
    st = c.checkpoint()
    assert len(st["spins"]) == 4 and all(np.all(x == i) for i, x in enumerate(st["spins"]))
    assert st["mcs"] == 40 and np.array_equal(st["widths"], [0.0, 0.3, 0.0, 0.7])


def test_restore_loads_spins_then_widths_then_the_counter(fake_ctx):
    c, calls = fake_ctx
    c.restore(c.checkpoint())
    assert [k[0] for k in calls] == ["spins"] * 4 + ["widths", "mcs"]
    assert [k[1] for k in calls[:4]] == [0, 1, 2, 3]
    assert np.array_equal(calls[4][1], [1.0, 0.3, 1.0, 0.7])  # non-adaptive slots get a valid filler
    assert calls[5] == ("mcs", 40)


def test_restore_without_adaptive_widths_skips_them(fake_ctx):
    c, calls = fake_ctx
    st = c.checkpoint()
    st["widths"] = np.zeros(4)
    c.restore(st)
    assert [k[0] for k in calls] == ["spins"] * 4 + ["mcs"]


def test_restore_refuses_another_shape(fake_ctx):
    c, calls = fake_ctx
    st = c.checkpoint()
    st["spins"] = st["spins"][:3]
    with pytest.raises(ValueError):
        c.restore(st)
    assert not calls


def test_ising_checkpoint_and_restore(monkeypatch):
    calls = []
    c = object.__new__(vb.IsingContext)
    c.replicas, c.ptr = 4, None
    monkeypatch.setattr(c, "spins", lambda r: np.full(8, r, dtype=np.int8), raising=False)
    monkeypatch.setattr(c, "stats", lambda: {"mcs_done": 12}, raising=False)
    monkeypatch.setattr(c, "set_spins", lambda r, x: calls.append(("spins", r)), raising=False)
    monkeypatch.setattr(c, "set_mcs_counter", lambda t: calls.append(("mcs", t)), raising=False)
    st = c.checkpoint()
    assert st["mcs"] == 12 and [int(x[0]) for x in st["spins"]] == [0, 1, 2, 3]
    c.restore(st)
    assert calls == [("spins", 0), ("spins", 1), ("spins", 2), ("spins", 3), ("mcs", 12)]
    with pytest.raises(ValueError):
        c.restore({"spins": st["spins"][:2], "mcs": 12})
