"""The benchmark line's host logic on the CPU, with the device and the context faked.

The fakes stand in for torch.cuda (events on a fake clock that each run advances) and for
vg.Context (counts launches, returns an empty history); nothing of the method runs except
the oracle's CPU baseline. The checks are the fields the line must carry, the arithmetic
that turns the counted attempts and the timed milliseconds into `value`, the roofline
fraction, and that the secondary workloads give every sample, with its instance ids, to the
context.
"""

import json
import sys
import types

import numpy as np
import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402

RUN_MS = 7.0      # fake device time of one run
SWEEP_MS = 0.25   # fake device time of one sweep launch


class Clock:
    now = 0.0


class FakeEvent:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = Clock.now

    def elapsed_time(self, other):
        return other.t - self.t


class FakeContext:
    made = []

    def __init__(self, samples, precision=32, replicas=1, seed=1, inst_base=0, device=-1, stream=None,
                 timing=False, variant=-1, type_stats=False, snapshots=False, resident_smem=0, graphs=1,
                 cluster_blocks=0, cluster_threads=0, cluster_split=0, group_threads=0, group_sites=0):
        self.samples, self.R, self.inst_base, self.precision = list(samples), replicas, inst_base, precision
        self.launches = self.sweeps = 0
        self.sweep_ms = 0.0
        self.hist_rows = 0
        FakeContext.made.append(self)

    @property
    def n_inst(self):
        return len(self.samples) * self.R

    def run(self, T, B, mcs):
        T, B = np.asarray(T), np.asarray(B)
        assert T.shape == B.shape and T.shape[0] == self.n_inst
        Clock.now += RUN_MS
        n = T.shape[1] * mcs
        self.launches += 3 * n
        self.sweeps += 2 * n
        self.sweep_ms += 2 * n * SWEEP_MS
        self.hist_rows += n

    def history(self):
        return np.zeros((self.n_inst, self.hist_rows, 4))

    def spins(self, inst):
        """Every spin along +z (the history says E = 0, so the precision figure is |E_up| / N)."""
        n = self.samples[inst // self.R].n_sites
        return np.tile([0.0, 0.0, 1.0], (n, 1))

    def stats(self):
        return {"kernel_launches": self.launches, "sweep_launches": self.sweeps, "sweep_ms": self.sweep_ms,
                "variant": 0, "block_threads": 256, "cluster_blocks": 0, "split_sites": 0, "group_threads": 0,
                "group_sites": 0}

    def close(self):
        pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


@pytest.fixture
def fake_device(monkeypatch):
    torch = pytest.importorskip("torch")
    import paper_1803_07030_gb300 as vg

    Clock.now = 0.0
    FakeContext.made = []
    for name, fn in (("set_device", lambda d: None), ("current_device", lambda: 0), ("synchronize", lambda: None),
                     ("current_stream", lambda: types.SimpleNamespace(cuda_stream=0)), ("Event", FakeEvent)):
        monkeypatch.setattr(torch.cuda, name, fn)
    monkeypatch.setattr(vg, "build", lambda *a, **k: None)
    monkeypatch.setattr(vg, "Context", FakeContext)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    return vg


def args(**kw):
    a = dict(gpus=1, steps=3, warmup=2, mcs=bench.MCS, impl="ours", side=bench.L_SIDE, depth=0, workload="sg256x32",
             policy="", variant=-1, analysis=False, ising=False, type_stats=False, snapshots=False, quick=False,
             resident_smem=0, graphs=1, cluster_blocks=0, cluster_threads=0, cluster_split=0, group_threads=0)
    a.update(kw)
    return types.SimpleNamespace(**a)


def last_json(capsys):
    return json.loads(capsys.readouterr().out.strip().splitlines()[-1])


def test_headline_line_fields_and_arithmetic(fake_device, capsys, monkeypatch):
    side, mcs = 8, 4
    monkeypatch.setattr(bench, "L_SIDE", side)
    bench.run_ours(args(mcs=mcs, side=side))
    line = last_json(capsys)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    n = side ** 3
    attempts = bench.REPLICAS * n * mcs * 3
    assert line["value"] == pytest.approx(attempts / (3 * RUN_MS / 1000.0))
    assert line["ms_per_step"] == pytest.approx(RUN_MS)
    assert line["n_gpus"] == 1 and line["steps"] == 3 and line["warmup"] == 2 and line["higher_is_better"]
    assert line["gpu_launches"] == 3 * 3 * mcs and line["vs_baseline"] is None
    r = line["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["kernel"] == "pass32_r32"
    assert r["attempts_per_launch"] == bench.REPLICAS * n // 2
    assert r["achieved"] == pytest.approx(bench.BYTES_PER_ATTEMPT * r["attempts_per_launch"] / (SWEEP_MS / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] is None  # the committed counters describe the 256^3 lattice only
    # the whole-step fraction: bytes per attempt x attempts/s of the line
    assert r["headline_achieved"] == pytest.approx(bench.BYTES_PER_ATTEMPT * line["value"] / 1e9)
    assert r["headline_frac"] == pytest.approx(r["headline_achieved"] / r["peak"])
    # precision: the history's E/N (the fake's is 0) against the oracle's energy of the spins
    import oracle
    from lattices import sc_periodic

    p = line["precision"]
    up = np.tile([0.0, 0.0, 1.0], (n, 1))
    e_up = abs(oracle.energy(sc_periodic(side, bimodal_seed=bench.SEED), up, 0.0)) / n
    assert p["bound"] == 1e-3 and [c["instance"] for c in p["checked"]] == [0, 16, 31]
    assert p["d_e_per_site"] == pytest.approx(e_up) and p["ok"] == (e_up < 1e-3)
    c = line["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] >= 1 and c["value"] > 0 and "host" in c
    e = line["e2e"]
    assert e["h2d_bytes_per_step"] == bench.REPLICAS * 2 * 8 + 40
    assert e["d2h_bytes_per_step"] == bench.REPLICAS * mcs * 4 * 8 + 4
    made = FakeContext.made
    assert made[0].R == bench.REPLICAS and made[0].inst_base == 0
    assert [m.inst_base for m in made[1:]] == [0, bench.REPLICAS - 1]  # the plain leg's two replicas


def test_quick_line(fake_device, capsys, monkeypatch):
    monkeypatch.setattr(bench, "L_SIDE", 6)
    bench.run_ours(args(mcs=1, steps=1, warmup=0, quick=True, side=6))
    line = last_json(capsys)
    assert line["quick"] and line["gpu_launches"] == 3 and line["avg_launch_ms"] == pytest.approx(SWEEP_MS)


def test_traffic_is_read_only_while_the_summary_matches_the_source(tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    summary = tmp_path / "k.txt"
    summary.write_text(f"kernel_source_sha256_16: {bench.kernel_hash([str(src)])}\ndram_bytes_per_launch: 1234\n")
    assert bench.profiled_traffic(str(summary), [str(src)]) == 1234.0
    src.write_text("kernel v2")
    assert bench.profiled_traffic(str(summary), [str(src)]) is None
    assert bench.profiled_traffic(str(tmp_path / "none.txt"), [str(src)]) is None
    for name, (kernel, path, sources, classes) in bench.SWEEP_KERNELS.items():
        text = open(path).read()
        assert kernel in text and "kernel_source_sha256_16:" in text and "dram_bytes_per_launch:" in text, name


@pytest.mark.parametrize("name", ["np256", "sc8_fp64"])
def test_secondary_workload_line(fake_device, capsys, name):
    secondary_line(capsys, name)


def secondary_line(capsys, name):
    from lattices import workload

    bench.run_workload(args(workload=name, steps=2, warmup=1))
    line = last_json(capsys)
    w = workload(name)
    main = FakeContext.made[0]
    assert len(main.samples) == len(w.samples) and main.inst_base == 0 and main.precision == w.precision
    assert line["value"] == pytest.approx(w.attempts() * 2 / (2 * RUN_MS / 1000.0))
    assert line["config"]["attempts_per_step"] == w.attempts()
    assert line["scaling"] == ("strong" if name == "np256" else "weak")
    assert line["dtype"] == ("f64" if name == "sc8_fp64" else "f32")
    assert line["gpu_launches"] == 3 * 2 * w.n_steps * w.mcs
    c = line["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] == 1 and c["value"] > 0 and c["unit"] == bench.UNIT
    p = line["precision"]
    assert p["bound"] == 1e-3 and p["checked"] and p["checked"][0]["instance"] == 0
    import oracle

    smp0 = w.samples[0]
    e_up = abs(oracle.energy(smp0, np.tile([0.0, 0.0, 1.0], (smp0.n_sites, 1)), float(w.B[0, -1]))) / smp0.n_sites
    assert p["checked"][0]["d_e_per_site"] == pytest.approx(e_up)
    r = line["effective_roofline"]
    assert r["achieved"] == pytest.approx(r["bytes_per_attempt"] * line["value"] / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    if name == "np256":
        plain = FakeContext.made[1:]
        assert [m.inst_base for m in plain] == list(range(len(w.samples)))
        assert line["batched_over_plain"] > 0
    return line


def test_workload_bytes_per_attempt_follow_the_size_table():
    """Spin read + write plus the links shared by the replicas: 32 + 48 B for a periodic sc
    lattice swept alone in FP32, 64 + 72 B in FP64, 32 + 48/32 B for 32 replicas."""
    from lattices import workload

    assert bench.workload_bytes_per_attempt(workload("sc64_hyst", scale=0.125)) == pytest.approx(80.0)
    assert bench.workload_bytes_per_attempt(workload("sc8_fp64")) == pytest.approx(136.0)
    assert bench.workload_bytes_per_attempt(workload("sg256x32", scale=1 / 32)) == pytest.approx(33.5)
    assert bench.BYTES_PER_ATTEMPT == pytest.approx(33.5)
    w = workload("np256", scale=0.05)
    z = sum(s.n_edges for s in w.samples) / sum(s.n_sites for s in w.samples)
    assert 8 < z < 12 and bench.workload_bytes_per_attempt(w) == pytest.approx(32 + 8 * z)


def test_reference_arm_on_a_secondary_workload(fake_device, capsys):
    """`--impl reference --workload NAME`: the oracle on the same config as the GPU line."""
    ours = secondary_line(capsys, "sc8_fp64")
    bench.run_reference(args(impl="reference", workload="sc8_fp64", steps=2, warmup=0))
    ref = last_json(capsys)
    assert ref["impl"] == "reference" and ref["value"] > 0 and ref["dtype"] == "f64"
    assert ref["metric"] == ours["metric"] and ref["unit"] == ours["unit"]
    assert ref["config"] == ours["config"] and ref["scaling"] == ours["scaling"]
    assert ref["e2e"]["h2d_bytes_per_step"] == 0 and ref["cpu_baseline"]["value"] == ref["value"]


def test_peak_falls_back_without_a_usable_measurement(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"bf16_tflops": 1900}')
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text("not json")
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6788.6}')
    assert bench.peaks() == (6788.6, "measured")


def test_reference_arm_is_not_silently_the_headline_for_other_lines(capsys):
    for kw in ({"analysis": True}, {"ising": True}):
        bench.run_reference(args(impl="reference", **kw))
        line = last_json(capsys)
        assert line["impl"] == "reference" and "unavailable" in line and "value" not in line
