"""Ising model (spin flip, Sec. II) on the GPU against the oracle, bit for bit.

The multi-spin-coded kernel takes its decisions with integer thresholds, so the spins and
the (E, M) history must equal the oracle's exactly: square and cubic lattices, several
replicas with their own temperature and field, run continuation, the all-up start and
spins set by the caller.
"""

import math

import numpy as np
import pytest

import oracle
import paper_1803_07030_gb300 as vg
from paper_1803_07030_gb300 import vegas as vb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    vg.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _check(ctx, ref):
    H = ctx.history()
    assert np.array_equal(H, ref["history"]), np.argwhere(H != ref["history"])[:3]
    for r in range(ctx.replicas):
        assert np.array_equal(ctx.spins(r), ref["spins"][r]), r


def test_square_lattice_bitwise():
    R, L = 8, 64
    T = np.stack([[1.5 + 0.25 * r, 3.0 - 0.2 * r] for r in range(R)])
    h = np.stack([[0.1 * (r % 3) - 0.1, 0.05] for r in range(R)])
    with vg.IsingContext(2, L, J=1.0, replicas=R, seed=11, inst_base=4) as c:
        c.run(T, h, 6)
        _check(c, oracle.ising_run(2, L, 1.0, T, h, 6, seed=11, inst_base=4))


def test_cubic_lattice_bitwise():
    R, L = 4, 64
    T = np.array([[3.5], [4.5], [5.5], [8.0]])
    h = np.array([[0.0], [0.2], [-0.3], [0.0]])
    with vg.IsingContext(3, L, J=0.8, replicas=R, seed=12) as c:
        c.run(T, h, 2)
        _check(c, oracle.ising_run(3, L, 0.8, T, h, 2, seed=12))


def test_continuation_all_up_and_set_spins():
    R, L = 4, 64
    T = np.array([[1.8, 2.2, 2.6]] * R)
    h = np.zeros_like(T)
    with vg.IsingContext(2, L, replicas=R, seed=13, init_up=True) as c:
        assert np.all(c.spins(2) == 1)
        c.run(T[:, :1], h[:, :1], 5)
        c.run(T[:, 1:], h[:, 1:], 5)
        up = np.ones((R, L * L), dtype=np.int8)
        _check(c, oracle.ising_run(2, L, 1.0, T, h, 5, seed=13, spins=up))
        rng = np.random.default_rng(1)
        S = rng.choice(np.array([-1, 1], dtype=np.int8), size=L * L)
        c.set_spins(1, S)
        assert np.array_equal(c.spins(1), S)


def test_ordered_phase_magnetization():
    L, R, T = 256, 4, 1.8
    with vg.IsingContext(2, L, replicas=R, seed=14, init_up=True) as c:
        c.run(np.full((R, 1), T), np.zeros((R, 1)), 400)
        H = c.history()
    m = np.abs(H[:, 100:, 1]).mean() / L ** 2
    assert abs(m - (1.0 - math.sinh(2.0 / T) ** -4) ** 0.125) < 0.01, m


def test_ising_option_errors():
    for kw in ({"L": 96}, {"L": 32}, {"replicas": 6}, {"inst_base": 2}, {"dims": 4}):
        with pytest.raises(vb.VegasError) as e:
            vg.IsingContext(**kw)
        assert e.value.status == vb.EINVAL
    with vg.IsingContext(2, 64, replicas=4) as c:
        with pytest.raises(vb.VegasError):
            c.run([[0.0]] * 4, [[0.0]] * 4, 1)
        with pytest.raises(vb.VegasError):
            c.set_spins(0, np.zeros(64 * 64, dtype=np.int8))
