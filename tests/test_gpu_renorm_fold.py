"""The end-of-step renormalisation |S_i| = s_i folded into the step's last class-1 pass of the
replica-batched (R = 32) FP32 sweep (option renorm_fold), through the C-ABI.

Every class-1 spin is stored renormalised by its own last attempt of the step, and every
class-0 block by the warp that finishes the last class-1 block reading it, so the spins,
energy/magnetisation histories, accepted counts and snapshots must equal, bit for bit, those
of the same sweep with the renormalisation in a pass of its own: on every launch path (one
graph per run, per step, per MCS, direct launches with timing events), with ragged blocks,
per-site spin norms (the FP64 formula) and anisotropy, and for a single MCS per step.
"""

import numpy as np
import pytest

import paper_1803_07030_gb300 as vg
from paper_1803_07030_gb300 import vegas as vb
from lattices import sc_periodic

pytestmark = pytest.mark.gpu

R = 32


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    vg.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def ctx(samples, **kw):
    kw.setdefault("stream", None)
    kw.setdefault("replicas", R)
    return vg.Context(samples, **kw)


def schedule(n_steps, seed=0):
    rng = np.random.default_rng(seed)
    T = np.geomspace(0.2, 2.5, R)[:, None] * np.linspace(1.0, 0.7, n_steps)[None, :]
    B = rng.uniform(-0.3, 0.3, size=(R, n_steps))
    return T, B


def glass(shape=8, seed=1, **kw):
    return sc_periodic(shape, bimodal_seed=seed, **kw)


def run_pair(s, n_steps=3, mcs=4, **kw):
    """The same run with and without the fold; returns both results and both stats."""
    T, B = schedule(n_steps)
    out = []
    for fold in (0, -1):
        with ctx([s], seed=11, renorm_fold=fold, accept_log_mcs=2, **kw) as c:
            c.run(T, B, mcs)
            out.append({"spins": np.stack([c.spins(i) for i in range(R)]), "hist": c.history(),
                        "acc": c.accept_history(), "alog": c.accept_log(), "stats": c.stats(),
                        "snap": c.snapshot(R - 1, n_steps - 1) if kw.get("snapshots") else None})
    return out


def assert_same(a, b):
    assert np.array_equal(a["spins"], b["spins"])
    assert np.array_equal(a["hist"], b["hist"])
    assert np.array_equal(a["acc"], b["acc"])
    assert np.array_equal(a["alog"], b["alog"])
    if a["snap"] is not None:
        assert np.array_equal(a["snap"], b["snap"])


def kernels(st):
    return vb.sweep_kernel_names(st["sweep_kernels"])


@pytest.mark.parametrize("graphs,timing", [(1, False), (2, False), (0, False), (0, True)])
def test_fold_matches_separate_pass_on_every_launch_path(graphs, timing):
    a, b = run_pair(glass(), variant=0, graphs=graphs, timing=timing)
    assert "pass32_r32_renorm" in kernels(a["stats"]) and "pass32_r32" in kernels(a["stats"])
    assert "pass32_r32_renorm" not in kernels(b["stats"])
    assert_same(a, b)
    # one kernel fewer per step: no renormalisation pass
    assert a["stats"]["kernel_launches"] == b["stats"]["kernel_launches"] - 3


@pytest.mark.parametrize("shape", [(6, 6, 10), (6, 6, 6), (6, 10, 14)])
def test_fold_ragged_blocks(shape):
    """Classes whose size is not a multiple of the kernel's 8-site blocks."""
    s = glass(shape, seed=4)
    a, b = run_pair(s, n_steps=2, mcs=3, variant=0)
    assert "pass32_r32_renorm" in kernels(a["stats"])
    assert_same(a, b)


def test_fold_single_mcs_steps_and_snapshots():
    a, b = run_pair(glass(6, seed=2), n_steps=4, mcs=1, variant=0, snapshots=True)
    assert "pass32_r32_renorm" in kernels(a["stats"])
    assert_same(a, b)


def test_fold_per_site_norms_and_anisotropy():
    """Spin norms other than 1 take the FP64 formula inside the fold; per-site parameters."""
    s = glass(8, seed=5, k_uni=0.4)
    rng = np.random.default_rng(5)
    s.spin_norm = rng.uniform(0.5, 2.5, size=s.n_sites)
    a, b = run_pair(s, variant=0)
    assert "pass32_r32_renorm" in kernels(a["stats"])
    assert_same(a, b)
    norms = np.linalg.norm(a["spins"], axis=2)
    assert np.allclose(norms, s.spin_norm[None, :], rtol=2e-7, atol=0)


def test_fold_with_automatic_sweep_choice():
    """Whatever sweep the autotuner keeps, the two contexts give the same spins."""
    a, b = run_pair(glass(8, seed=6), n_steps=3, mcs=16)
    assert_same(a, b)


def test_fold_not_used_where_it_does_not_apply():
    """FP64, fewer replicas, more than two colour classes, another sweep: a pass of its own."""
    s = glass(6, seed=3)
    T, B = schedule(2)
    for kw in ({"precision": 64}, {"replicas": 16}, {"variant": 1}):
        with ctx([s], seed=3, **kw) as c:
            Tk, Bk = T[:c.n_instances], B[:c.n_instances]
            c.run(Tk, Bk, 2)
            assert "pass32_r32_renorm" not in kernels(c.stats())
    odd = sc_periodic(5)  # an odd periodic side needs a third colour
    with ctx([odd], seed=3, variant=0) as c:
        c.run(T, B, 2)
        assert "pass32_r32_renorm" not in kernels(c.stats())
