"""Checkpoint and resume: a new context continues a chain bit for bit.

The random numbers of an attempt are keyed by (site, global MCS counter, instance, purpose),
so the state of a chain between temperature/field steps is its spins, the MCS counter and,
for the adaptive policy, the instance's width. A context that loads these from another
context's checkpoint must then produce the spins and accept/reject decisions of the
uninterrupted chain, in FP64 (and equal the oracle started from the same state) and in FP32
under the automatic, wavefront and adaptive-policy paths; rewinding a context to an earlier
checkpoint must replay the same MCS. The Ising contexts resume the same way.
"""

import numpy as np
import pytest

import oracle
import paper_1803_07030_gb300 as vg
from paper_1803_07030_gb300 import vegas as vb
from lattices import sc_periodic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    vg.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def schedule(R, n_steps):
    T = np.stack([np.linspace(2.2, 0.6, n_steps) * (0.8 + 0.4 * r / max(R - 1, 1)) for r in range(R)])
    return T, np.full_like(T, 0.15)


def sample(policy):
    s = sc_periodic((8, 6, 10), bimodal_seed=4, k_uni=0.3)
    if policy:
        s.with_policy([vg.POLICY_ADAPTIVE], [0.4])
    return s


CASES = [
    ("fp64", dict(precision=64, replicas=4, variant=0), False),
    ("fp32_auto", dict(precision=32, replicas=32, variant=-1), False),
    ("fp32_wave", dict(precision=32, replicas=32, variant=4), False),
    ("fp32_adaptive", dict(precision=32, replicas=4, variant=-1), True),
]


@pytest.mark.parametrize("name,kw,policy", CASES, ids=[c[0] for c in CASES])
def test_resume_in_a_new_context_continues_the_chain(name, kw, policy):
    s = sample(policy)
    R, mcs = kw["replicas"], 5
    T, B = schedule(R, 3)
    opts = dict(kw, seed=19, stream=None)
    with vg.Context([s], **opts) as a:
        a.run(T, B, mcs)
        want = [a.spins(i) for i in range(R)]
        H_want, acc_want = a.history(), a.accept_history()
    with vg.Context([s], **opts) as b:
        b.run(T[:, :2], B[:, :2], mcs)
        state = b.checkpoint()
    assert state["mcs"] == 2 * mcs
    with vg.Context([s], **opts) as c:
        c.restore(state)
        c.run(T[:, 2:], B[:, 2:], mcs)
        assert c.stats()["mcs_done"] == 3 * mcs
        for i in range(R):
            assert np.array_equal(c.spins(i), want[i]), (name, i)
        assert np.array_equal(c.accept_history(), acc_want[:, 2 * mcs:])
        H = c.history()
        if kw["precision"] == 64:
            assert np.array_equal(H, H_want[:, 2 * mcs:])
            ref = oracle.run(s, T[:, 2:], B[:, 2:], mcs, seed=19, spins=np.stack(state["spins"]), t0=2 * mcs,
                             n_threads=R)
            for i in range(R):
                assert np.array_equal(c.spins(i), ref["spins"][i]), i
        else:
            assert np.all(np.abs(H - H_want[:, 2 * mcs:]) <= 2e-6 * s.n_sites)


@pytest.mark.parametrize("variant", [0, 4])
def test_rewinding_a_context_replays_the_same_mcs(variant):
    """Restoring an earlier checkpoint into the same context runs those MCS again: the last
    step run twice gives the same spins both times (for the wavefront sweep this needs its
    completion words of the later MCS cleared)."""
    s = sample(False)
    R, mcs = 32, 4
    T, B = schedule(R, 3)
    with vg.Context([s], precision=32, replicas=R, seed=23, variant=variant, stream=None) as c:
        c.run(T[:, :2], B[:, :2], mcs)
        state = c.checkpoint()
        c.run(T[:, 2:], B[:, 2:], mcs)
        first = [c.spins(i) for i in range(R)]
        c.restore(state)
        c.run(T[:, 2:], B[:, 2:], mcs)
        assert c.stats()["mcs_done"] == 3 * mcs
        for i in range(R):
            assert np.array_equal(c.spins(i), first[i]), i


def test_mcs_counter_limit():
    with vg.Context([sample(False)], precision=32, replicas=4, seed=1, stream=None) as c:
        with pytest.raises(vb.VegasError) as e:
            c.set_mcs_counter(2 ** 32 - 1)
        assert e.value.status == vb.EINVAL
        c.set_mcs_counter(2 ** 32 - 10)
        with pytest.raises(vb.VegasError):  # 3 x 5 more MCS would pass the 32-bit counter
            c.run(np.ones((4, 3)), np.zeros((4, 3)), 5)


def test_ising_resume_in_a_new_context():
    R, L, mcs = 8, 64, 4
    T = np.stack([[2.6 - 0.1 * r, 2.2, 1.9] for r in range(R)])
    h = np.full_like(T, 0.05)
    with vg.IsingContext(2, L, replicas=R, seed=29) as a:
        a.run(T, h, mcs)
        want, H_want = [a.spins(r) for r in range(R)], a.history()
    with vg.IsingContext(2, L, replicas=R, seed=29) as b:
        b.run(T[:, :2], h[:, :2], mcs)
        saved, t = [b.spins(r) for r in range(R)], b.stats()["mcs_done"]
    with vg.IsingContext(2, L, replicas=R, seed=29) as c:
        for r in range(R):
            c.set_spins(r, saved[r])
        c.set_mcs_counter(t)
        c.run(T[:, 2:], h[:, 2:], mcs)
        for r in range(R):
            assert np.array_equal(c.spins(r), want[r]), r
        assert np.array_equal(c.history(), H_want[:, 2 * mcs:])
        ref = oracle.ising_run(2, L, 1.0, T[:, 2:], h[:, 2:], mcs, seed=29, spins=np.stack(saved), t0=t)
        assert np.array_equal(c.history(), ref["history"])
