"""Pins of the CPU oracle to facts outside itself (no GPU).

Each check below ties one part of the oracle to mathematics or to an independent
implementation, so that a dropped term, a flipped sign, a wrong index or a transposed
operand in the oracle fails at least one of them:

  Philox4x32-10      bit-exact against Triton's own Philox (run in its CPU interpreter)
  sphere sampler     unit norm, moments, uniform z and azimuth (Kolmogorov-Smirnov)
  energy (Eq. 1-3)   hand-computed configurations (pair angle, Neel state, cubic axes)
  dE                 equals E(after) - E(before) on random graphs with every term on
  Zeeman             Langevin law <S.n> = s L(beta B s), L(x) = coth x - 1/x
  exchange           open classical Heisenberg chain: U = -(N-1) J L(beta J) and
                     <M^2> = N + 2 sum_d (N-d) L(beta J)^d, for J > 0 and J < 0
  uniaxial           single spin, beta k > 0: <(S.e)^2> = e^a / (sqrt(pi a) erfi sqrt a) - 1/(2a);
                     beta k < 0 by 1D quadrature
  cubic              single spin, 2D quadrature over the sphere, both signs
  mixed terms        dimer with exchange + field + uniaxial axis, 4D quadrature
  non-bipartite      three-spin ring (3 colours), J = +1 and J = -1, quadrature
  detailed balance   dimer bond-angle histogram against exp(beta J cos theta), chi^2
  update order       random-site selection (Sec. III.B) and the colour sweep agree
  limits             high-T series U/N = -beta sum J^2 / (3N); low-T equipartition
  colouring          identical to networkx's greedy colouring in index order
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import integrate, special, stats

from conftest import binned

import oracle
from lattices import chain_open, dimers, free_spins, random_graph, sc_periodic, triangles


def langevin(x):
    x = np.asarray(x, dtype=np.float64)
    return 1.0 / np.tanh(x) - 1.0 / x


def pooled(series):
    """Mean and standard error over several independent instances' time series."""
    means, ses = zip(*[binned(s) for s in series])
    means, ses = np.array(means), np.array(ses)
    return float(means.mean()), float(np.sqrt((ses ** 2).sum()) / len(ses))


def sphere_grid(n_cos=48, n_phi=64):
    """Quadrature of the uniform measure on the unit sphere (weights sum to 1)."""
    x, w = np.polynomial.legendre.leggauss(n_cos)
    phi = 2.0 * np.pi * (np.arange(n_phi) + 0.5) / n_phi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1.0 - ct * ct)
    v = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    wt = (w[:, None] / 2.0 / n_phi * np.ones_like(ph)).reshape(-1)
    return v, wt


# --------------------------------------------------------------------------- Philox

_TRITON_PROBE = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def _k(out, seed, c0p, c1p, c2p, c3p, n, BLOCK: tl.constexpr):
    off = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
    m = off < n
    a, b, c, d = tl.philox(seed, tl.load(c0p + off, mask=m), tl.load(c1p + off, mask=m),
                           tl.load(c2p + off, mask=m), tl.load(c3p + off, mask=m), 10)
    tl.store(out + off * 4 + 0, a, mask=m)
    tl.store(out + off * 4 + 1, b, mask=m)
    tl.store(out + off * 4 + 2, c, mask=m)
    tl.store(out + off * 4 + 3, d, mask=m)

req = json.loads(sys.stdin.read())
res = []
for seed, ctrs in req:
    c = np.array(ctrs, dtype=np.uint32).reshape(-1, 4)
    n = c.shape[0]
    cols = [torch.from_numpy(np.ascontiguousarray(c[:, i])) for i in range(4)]
    out = torch.from_numpy(np.zeros(n * 4, dtype=np.uint32))
    _k[(triton.cdiv(n, 64),)](out, seed, *cols, n, BLOCK=64)
    res.append(out.numpy().astype(np.int64).tolist())
print(json.dumps(res))
"""


def test_philox_matches_triton_interpreter():
    pytest.importorskip("triton")
    rng = np.random.Generator(np.random.PCG64(7))
    seeds = [1, 0x123456789ABCDEF, int(rng.integers(0, 2 ** 63)), 0xFFFFFFFF00000000]
    req = []
    for sd in seeds:
        ctr = rng.integers(0, 2 ** 32, size=(200, 4), dtype=np.uint64)
        ctr[:5] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 0xFFFFFFFF, 5, 0x20000], [7, 3, 1, 0x10000], [2 ** 32 - 1] * 4]
        req.append([sd, ctr.astype(np.int64).tolist()])
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_PROBE], input=json.dumps(req), capture_output=True,
                       text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr.strip().splitlines()[-1][:200])
    got = json.loads(p.stdout.strip().splitlines()[-1])
    for (sd, ctrs), ref in zip(req, got):
        key = [sd & 0xFFFFFFFF, sd >> 32]
        ref = np.array(ref, dtype=np.uint64).reshape(-1, 4)
        for c, r in zip(ctrs, ref):
            assert np.array_equal(oracle.philox4x32_10(c, key).astype(np.uint64), r), (sd, c)


# --------------------------------------------------------------------------- sphere

def test_sphere_sampler_uniform():
    n = 60000
    v = np.empty((n, 3))
    used = np.empty(n, dtype=np.int64)
    for i in range(n):
        v[i], used[i] = oracle.sphere(11, i, 3, 0, 0x20000)
    norm = np.linalg.norm(v, axis=1)
    assert np.all(np.abs(norm - 1.0) < 4e-16)
    se = 1.0 / np.sqrt(n)
    assert np.all(np.abs(v.mean(axis=0)) < 5 * se / np.sqrt(3))
    assert np.all(np.abs((v ** 2).mean(axis=0) - 1.0 / 3.0) < 5 * se * 0.3)
    assert abs((v[:, 0] * v[:, 1]).mean()) < 5 * se * 0.2
    assert stats.kstest(v[:, 2], stats.uniform(-1, 2).cdf).pvalue > 1e-4
    phi = np.arctan2(v[:, 1], v[:, 0])
    assert stats.kstest(phi, stats.uniform(-np.pi, 2 * np.pi).cdf).pvalue > 1e-4
    # a candidate is kept with probability pi/4 (disk inside the square)
    assert abs((used == 1).mean() - np.pi / 4) < 5 * np.sqrt(0.17 / n)
    # same counter, same point
    a, _ = oracle.sphere(11, 5, 3, 0, 0x20000)
    assert np.array_equal(a, v[5])


def test_uniform_range_and_mean():
    u = np.array([oracle.uniform(3, i, 9, 1, 0x10000) for i in range(40000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / len(u))
    assert stats.kstest(u, "uniform").pvalue > 1e-4


# --------------------------------------------------------------------------- energy, closed forms

def test_energy_pair_angle_and_norms():
    for J in (1.0, -0.7):
        s = dimers(1, J=J)
        for th in (0.0, 0.4, 1.9, np.pi):
            S = np.array([[0, 0, 1.0], [np.sin(th), 0, np.cos(th)]])
            assert oracle.energy(s, S, 0.0) == pytest.approx(-J * np.cos(th), abs=1e-15)
    s = dimers(1, J=1.0)
    s.spin_norm = np.array([2.0, 3.0])
    assert oracle.energy(s, np.array([[0, 0, 2.0], [0, 0, 3.0]]), 0.0) == pytest.approx(-6.0)


def test_energy_lattice_states():
    L = 4
    s = sc_periodic(L, J=1.0, k_uni=0.3, e_axis=(0, 0, 1))
    n = s.n_sites
    up = np.tile([0, 0, 1.0], (n, 1))
    assert oracle.energy(s, up, 0.7) / n == pytest.approx(-3.0 - 0.7 - 0.3, abs=1e-14)
    side = np.tile([1.0, 0, 0], (n, 1))
    assert oracle.energy(s, side, 0.7) / n == pytest.approx(-3.0, abs=1e-14)
    idx = np.arange(n)
    par = ((idx % L) + (idx // L) % L + idx // (L * L)) % 2
    neel = up * np.where(par == 0, 1.0, -1.0)[:, None]
    assert oracle.energy(s, neel, 0.0) / n == pytest.approx(3.0 - 0.3, abs=1e-14)


def test_energy_cubic_axes():
    s = free_spins(3, k_cub=2.0)
    S = np.array([[1, 1, 1] / np.sqrt(3.0), [1.0, 0, 0], [1, 1, 0] / np.sqrt(2.0)])
    e = [oracle.energy(free_spins(1, k_cub=2.0), S[i:i + 1], 0.0) for i in range(3)]
    assert e == pytest.approx([-2.0 / 3.0, 0.0, -0.5], abs=1e-15)
    assert oracle.energy(s, S, 0.0) == pytest.approx(sum(e), abs=1e-15)


def test_delta_e_equals_energy_difference():
    rng = np.random.Generator(np.random.PCG64(5))
    for seed in range(4):
        s = random_graph(30, 0.25, seed)
        n = s.n_sites
        u = rng.normal(size=(n, 3))
        S = u / np.linalg.norm(u, axis=1, keepdims=True) * s.spin_norm[:, None]
        for _ in range(60):
            i = int(rng.integers(n))
            B = float(rng.normal())
            t = rng.normal(size=3)
            t = t / np.linalg.norm(t) * s.spin_norm[i]
            e0 = oracle.energy(s, S, B)
            S2 = S.copy()
            S2[i] = t
            e1 = oracle.energy(s, S2, B)
            assert oracle.delta_e(s, S, i, t, B) == pytest.approx(e1 - e0, abs=1e-12 * (1 + abs(e0)))


def test_renormalise_and_init():
    s = random_graph(20, 0.2, 3)
    S = np.random.Generator(np.random.PCG64(1)).normal(size=(20, 3))
    R = oracle.renormalise(s, S)
    assert np.allclose(np.linalg.norm(R, axis=1), s.spin_norm, rtol=0, atol=4e-16)
    assert np.allclose(R / np.linalg.norm(R, axis=1)[:, None], S / np.linalg.norm(S, axis=1)[:, None], atol=1e-15)
    a = oracle.init_spins(s, 1, 0)
    b = oracle.init_spins(s, 1, 0)
    c = oracle.init_spins(s, 1, 1)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.allclose(np.linalg.norm(a, axis=1), s.spin_norm, atol=1e-15)


# --------------------------------------------------------------------------- colouring

def _nx_greedy(sample):
    nx = pytest.importorskip("networkx")
    G = nx.Graph()
    n = sample.n_sites
    G.add_nodes_from(range(n))
    src = np.repeat(np.arange(n), np.diff(sample.row_ptr))
    G.add_edges_from(zip(src.tolist(), sample.col.tolist()))
    col = nx.greedy_color(G, strategy=lambda g, c: list(range(n)))
    return np.array([col[i] for i in range(n)])


@pytest.mark.parametrize("make", [lambda: sc_periodic(8), lambda: sc_periodic(5), lambda: random_graph(80, 0.1, 2),
                                  lambda: triangles(5), lambda: __import__("lattices").fcc_sphere(3.2)])
def test_greedy_colouring_matches_networkx(make):
    s = make()
    c, nc = oracle.greedy_colour(s)
    assert np.array_equal(c, _nx_greedy(s))
    src = np.repeat(np.arange(s.n_sites), np.diff(s.row_ptr))
    assert np.all(c[src] != c[s.col])
    assert nc == c.max() + 1


def test_even_periodic_sc_is_two_coloured():
    s = sc_periodic(6)
    c, nc = oracle.greedy_colour(s)
    idx = np.arange(s.n_sites)
    assert nc == 2
    assert np.array_equal(c, (idx % 6 + (idx // 6) % 6 + idx // 36) % 2)


# --------------------------------------------------------------------------- chain statistics

def test_langevin_law_zeeman():
    n = 3000
    axis = np.array([1.0, 2.0, 2.0]) / 3.0
    s = free_spins(n, field_axis=axis)
    Bs = np.array([0.5, 2.0, 8.0])
    r = oracle.run(s, np.ones((3, 1)), Bs[:, None], 400, seed=3)
    assert r["err"] == 0
    h = r["history"]
    mn = h[:, :, 1:] @ axis
    # history energy is -B sum S.n exactly (no other term is present)
    assert np.allclose(h[:, :, 0], -Bs[:, None] * mn, rtol=1e-12, atol=1e-9)
    for k, B in enumerate(Bs):
        m, se = binned(mn[k] / n)
        assert abs(m - langevin(B)) < 4 * se + 1e-4, (B, m, se, langevin(B))


def test_langevin_law_spin_norm():
    n, sn, B, T = 3000, 1.5, 0.8, 1.2
    s = free_spins(n, spin_norm=sn)
    r = oracle.run(s, [[T]], [[B]], 400, seed=4)
    m, se = binned(r["history"][0, :, 3] / n)
    assert abs(m - sn * langevin(B * sn / T)) < 4 * se + 1e-4


@pytest.mark.parametrize("J,beta", [(1.0, 2.0), (-1.0, 2.0), (1.0, 0.5)])
def test_open_heisenberg_chain(J, beta):
    N, R = 64, 16
    s = chain_open(N, J=J)
    r = oracle.run(s, np.full((R, 1), 1.0 / beta), np.zeros((R, 1)), 1500, seed=5)
    u = langevin(beta * J)
    U = -(N - 1) * J * u
    m, se = pooled(r["history"][:, :, 0])
    assert abs(m - U) < 4 * se + 1e-9, (m, se, U)
    d = np.arange(1, N)
    M2 = N + 2 * np.sum((N - d) * u ** d)
    m2, se2 = pooled((r["history"][:, :, 1:] ** 2).sum(axis=2))
    assert abs(m2 - M2) < 4 * se2, (m2, se2, M2)


@pytest.mark.parametrize("k", [2.0, -1.5])
def test_single_spin_uniaxial(k):
    n, T = 3000, 1.0
    e = np.array([0.0, 1.0, 1.0]) / np.sqrt(2.0)
    s = free_spins(n, k_uni=k, e_uni=e)
    r = oracle.run(s, [[T]], [[0.0]], 400, seed=6)
    m, se = binned(-r["history"][0, :, 0] / (k * n))  # <(S.e)^2>
    a = k / T
    if a > 0:
        exact = np.exp(a) / (np.sqrt(np.pi * a) * special.erfi(np.sqrt(a))) - 1.0 / (2.0 * a)
    else:
        num = integrate.quad(lambda x: x * x * np.exp(a * x * x), -1, 1)[0]
        exact = num / integrate.quad(lambda x: np.exp(a * x * x), -1, 1)[0]
    assert abs(m - exact) < 4 * se + 1e-5, (m, se, exact)


@pytest.mark.parametrize("kc", [2.5, -2.5])
def test_single_spin_cubic(kc):
    n, T = 3000, 0.8
    s = free_spins(n, k_cub=kc)
    r = oracle.run(s, [[T]], [[0.0]], 400, seed=7)
    m, se = binned(r["history"][0, :, 0] / n)
    v, w = sphere_grid(64, 96)
    x2, y2, z2 = (v ** 2).T
    cub = x2 * y2 + y2 * z2 + x2 * z2
    bw = w * np.exp(kc * cub / T)
    exact = -kc * np.sum(bw * cub) / np.sum(bw)
    assert abs(m - exact) < 4 * se + 1e-5, (m, se, exact)


def test_dimer_with_field_and_anisotropy():
    J, B, k, T = 1.0, 0.7, 0.8, 1.0
    e = np.array([1.0, 0.0, 0.0])
    P = 3000
    s = dimers(P, J=J)
    s.k_uni = np.full(2 * P, k)
    s.e_uni = np.tile(e, (2 * P, 1))
    r = oracle.run(s, [[T]], [[B]], 500, seed=8)
    v, w = sphere_grid(40, 56)
    single = -B * v[:, 2] - k * (v @ e) ** 2
    Epair = -J * (v @ v.T) + single[:, None] + single[None, :]
    W = w[:, None] * w[None, :] * np.exp(-(Epair - Epair.min()) / T)
    Z = W.sum()
    E_exact = (W * Epair).sum() / Z
    Mz_exact = (W * (v[:, 2][:, None] + v[:, 2][None, :])).sum() / Z
    m, se = binned(r["history"][0, :, 0] / P)
    assert abs(m - E_exact) < 4 * se + 1e-5, (m, se, E_exact)
    mz, sez = binned(r["history"][0, :, 3] / P)
    assert abs(mz - Mz_exact) < 4 * sez + 1e-5, (mz, sez, Mz_exact)


@pytest.mark.parametrize("J", [-1.0, 1.0])
def test_three_spin_ring(J):
    T, P = 0.7, 2000
    s = triangles(P, J=J)
    _, nc = oracle.greedy_colour(s)
    assert nc == 3
    r = oracle.run(s, [[T]], [[0.0]], 500, seed=9)
    # S1 = z; S2 in the xz-plane (uniform in cos theta2); S3 anywhere
    x2, w2 = np.polynomial.legendre.leggauss(48)
    v3, w3 = sphere_grid(48, 64)
    S2 = np.stack([np.sqrt(1 - x2 ** 2), np.zeros_like(x2), x2], axis=1)
    c12 = x2[:, None]
    c13 = v3[:, 2][None, :]
    c23 = S2 @ v3.T
    E = -J * (c12 + c13 + c23)
    W = (w2 / 2.0)[:, None] * w3[None, :] * np.exp(-(E - E.min()) / T)
    exact = (W * E).sum() / W.sum()
    m, se = binned(r["history"][0, :, 0] / P)
    assert abs(m - exact) < 4 * se + 1e-5, (m, se, exact)


def test_detailed_balance_bond_angle_histogram():
    P, J, T = 20000, 1.0, 0.5
    s = dimers(P, J=J)
    r = oracle.run(s, [[T]], [[0.0]], 200, seed=10)
    S = r["spins"][0]
    c = np.einsum("ij,ij->i", S[0::2], S[1::2])
    K = J / T
    edges = np.linspace(-1, 1, 21)
    obs, _ = np.histogram(c, bins=edges)
    p = (np.exp(K * edges[1:]) - np.exp(K * edges[:-1])) / (np.exp(K) - np.exp(-K))
    chi2 = float(((obs - P * p) ** 2 / (P * p)).sum())
    assert chi2 < stats.chi2.ppf(1 - 1e-4, 19), chi2


def test_random_site_and_colour_sweep_agree():
    s = sc_periodic(6)
    R = 4
    T = np.full((R, 1), 1.5)
    a = oracle.run(s, T, np.zeros((R, 1)), 2500, seed=12, mode=0)
    b = oracle.run(s, T, np.zeros((R, 1)), 2500, seed=13, mode=1)
    ma, sa = pooled(a["history"][:, :, 0] / s.n_sites)
    mb, sb = pooled(b["history"][:, :, 0] / s.n_sites)
    assert abs(ma - mb) < 4 * np.hypot(sa, sb), (ma, sa, mb, sb)


def test_high_temperature_series_spin_glass():
    s = sc_periodic(6, bimodal_seed=4)
    T = 10.0
    R = 4
    r = oracle.run(s, np.full((R, 1), T), np.zeros((R, 1)), 1500, seed=14)
    m, se = pooled(r["history"][:, :, 0] / s.n_sites)
    lead = -(1.0 / T) * np.sum(s.J ** 2) / 2.0 / 3.0 / s.n_sites
    assert abs(m - lead) < 4 * se + 0.02 * abs(lead), (m, se, lead)


def test_low_temperature_equipartition():
    s = sc_periodic(6)
    n = s.n_sites
    T = 0.1
    up = np.tile([0, 0, 1.0], (4, n, 1))
    r = oracle.run(s, np.full((4, 1), T), np.zeros((4, 1)), 3000, seed=15, spins=up)
    m, se = pooled(r["history"][:, :, 0] / n)
    assert abs(m - (-3.0 + T)) < 0.15 * T + 4 * se, m


def test_chain_continuation_bitwise():
    s = sc_periodic(4, k_uni=0.2)
    T = np.array([[2.0, 1.0, 0.5]])
    B = np.array([[0.1, -0.3, 0.2]])
    full = oracle.run(s, T, B, 7, seed=21)
    a = oracle.run(s, T[:, :1], B[:, :1], 7, seed=21)
    b = oracle.run(s, T[:, 1:], B[:, 1:], 7, seed=21, spins=a["spins"], t0=7)
    assert np.array_equal(full["spins"], b["spins"])
    assert np.array_equal(full["history"], np.concatenate([a["history"], b["history"]], axis=1))
