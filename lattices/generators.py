"""Synthetic atomistic samples: site list, directed neighbour CSR and site parameters.

The layout mirrors the paper's material file (Sec. III.C): per site a spin norm, a field
axis, a type; per link a pair of sites and an exchange constant; plus the anisotropy
constants and axes of the anisotropy file. Links are listed in both directions with equal
exchange, as the C-ABI requires. Every generator is deterministic for a given seed.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np


@dataclass
class Sample:
    """One atomistic sample. Arrays follow the C-ABI field names and dtypes.

    row_ptr int64[n+1], col int32[E], J float64[E] (directed, both directions present);
    optional per-site arrays (None means the library default): type int32[n],
    spin_norm float64[n] (default 1), field_axis float64[n,3] (default +z),
    k_uni float64[n] (default 0), e_uni float64[n,3] (default +z), k_cub float64[n]
    (default 0), colour int32[n] (default: greedy colouring), positions float64[n,3]
    (geometry only, never used by the method). Update policy per site type (Sec. II):
    type_policy int32[n_types] (0 random, 1 spin flip, 2 small step, 3 Gaussian,
    4 Hinzke-Nowak, 5 adaptive) and type_param float64[n_types] (cap half-angle in radians
    for 2 and 4, Gaussian width for 3 and the starting width for 5); None means random for
    every site.
    """

    name: str
    row_ptr: np.ndarray
    col: np.ndarray
    J: np.ndarray
    type: Optional[np.ndarray] = None
    spin_norm: Optional[np.ndarray] = None
    field_axis: Optional[np.ndarray] = None
    k_uni: Optional[np.ndarray] = None
    e_uni: Optional[np.ndarray] = None
    k_cub: Optional[np.ndarray] = None
    colour: Optional[np.ndarray] = None
    positions: Optional[np.ndarray] = None
    type_policy: Optional[np.ndarray] = None
    type_param: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    def with_policy(self, policies, params) -> "Sample":
        """Set the update policy table (one entry per site type) and return self."""
        self.type_policy = np.asarray(np.atleast_1d(policies), dtype=np.int32)
        self.type_param = np.asarray(np.broadcast_to(np.atleast_1d(params), self.type_policy.shape), dtype=np.float64)
        return self

    @property
    def n_sites(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def n_edges(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def param(self, name: str) -> np.ndarray:
        """Per-site parameter with the library default filled in."""
        n = self.n_sites
        v = getattr(self, name)
        if v is not None:
            return v
        if name == "spin_norm":
            return np.ones(n)
        if name in ("field_axis", "e_uni"):
            out = np.zeros((n, 3))
            out[:, 2] = 1.0
            return out
        if name in ("k_uni", "k_cub"):
            return np.zeros(n)
        if name == "type":
            return np.zeros(n, dtype=np.int32)
        raise KeyError(name)


def _csr_from_neighbour_table(nbr: np.ndarray, Jtab: np.ndarray) -> tuple:
    """Build CSR from a [n, z] neighbour table where -1 marks a missing neighbour.

    Within a row the neighbours keep the table's column order.
    """
    n, z = nbr.shape
    present = nbr >= 0
    deg = present.sum(axis=1).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    col = nbr[present].astype(np.int32)
    J = Jtab[present].astype(np.float64)
    return row_ptr, col, J


def sc_periodic(
    L,
    J: float = 1.0,
    k_uni: float = 0.0,
    e_axis: Sequence[float] = (0.0, 0.0, 1.0),
    bimodal_seed: Optional[int] = None,
) -> Sample:
    """Simple cubic lattice with periodic boundaries, site i = x + Lx*(y + Ly*z).

    Row order of every site: +x, -x, +y, -y, +z, -z. Each side must be >= 3 so the six
    neighbours are distinct. With bimodal_seed set, every undirected bond gets J or -J
    with equal probability (an Edwards-Anderson +-J spin glass); the same draw is shared
    by both directions of the bond.
    """
    Lx, Ly, Lz = (L, L, L) if np.isscalar(L) else tuple(L)
    if min(Lx, Ly, Lz) < 3:
        raise ValueError("periodic sc needs every side >= 3")
    n = Lx * Ly * Lz
    idx = np.arange(n, dtype=np.int64)
    x = idx % Lx
    y = (idx // Lx) % Ly
    z = idx // (Lx * Ly)

    def site(xx, yy, zz):
        return xx + Lx * (yy + Ly * zz)

    nbr = np.empty((n, 6), dtype=np.int64)
    nbr[:, 0] = site((x + 1) % Lx, y, z)
    nbr[:, 1] = site((x - 1) % Lx, y, z)
    nbr[:, 2] = site(x, (y + 1) % Ly, z)
    nbr[:, 3] = site(x, (y - 1) % Ly, z)
    nbr[:, 4] = site(x, y, (z + 1) % Lz)
    nbr[:, 5] = site(x, y, (z - 1) % Lz)
    if bimodal_seed is None:
        Jtab = np.full((n, 6), float(J))
    else:
        rng = np.random.Generator(np.random.PCG64(bimodal_seed))
        # one draw per bond in the +x, +y, +z direction of every site
        sgn = np.where(rng.integers(0, 2, size=(n, 3), dtype=np.int8) == 1, 1.0, -1.0) * float(J)
        Jtab = np.empty((n, 6))
        Jtab[:, 0] = sgn[:, 0]
        Jtab[:, 1] = sgn[nbr[:, 1], 0]
        Jtab[:, 2] = sgn[:, 1]
        Jtab[:, 3] = sgn[nbr[:, 3], 1]
        Jtab[:, 4] = sgn[:, 2]
        Jtab[:, 5] = sgn[nbr[:, 5], 2]
    row_ptr = np.arange(0, 6 * n + 1, 6, dtype=np.int64)
    col = nbr.reshape(-1).astype(np.int32)
    Jf = Jtab.reshape(-1)
    s = Sample(name=f"sc{Lx}x{Ly}x{Lz}", row_ptr=row_ptr, col=col, J=Jf)
    s.positions = np.stack([x, y, z], axis=1).astype(np.float64)
    if k_uni != 0.0:
        e = np.asarray(e_axis, dtype=np.float64)
        e = e / np.linalg.norm(e)
        s.k_uni = np.full(n, float(k_uni))
        s.e_uni = np.tile(e, (n, 1))
    s.meta = {"L": (Lx, Ly, Lz), "bimodal_seed": bimodal_seed}
    return s


def chain_open(n: int, J: float = 1.0) -> Sample:
    """Open chain of n spins with n-1 bonds; row order: left neighbour, then right."""
    nbr = np.full((n, 2), -1, dtype=np.int64)
    nbr[1:, 0] = np.arange(n - 1)
    nbr[:-1, 1] = np.arange(1, n)
    row_ptr, col, Jv = _csr_from_neighbour_table(nbr, np.full((n, 2), float(J)))
    return Sample(name=f"chain{n}", row_ptr=row_ptr, col=col, J=Jv)


def free_spins(
    n: int,
    field_axis: Optional[Sequence[float]] = None,
    k_uni: float = 0.0,
    e_uni: Optional[Sequence[float]] = None,
    k_cub: float = 0.0,
    spin_norm: float = 1.0,
) -> Sample:
    """n non-interacting spins (no links) with shared axes and constants."""
    s = Sample(
        name=f"free{n}",
        row_ptr=np.zeros(n + 1, dtype=np.int64),
        col=np.zeros(0, dtype=np.int32),
        J=np.zeros(0),
    )
    if field_axis is not None:
        a = np.asarray(field_axis, dtype=np.float64)
        s.field_axis = np.tile(a / np.linalg.norm(a), (n, 1))
    if k_uni != 0.0:
        e = np.asarray(e_uni if e_uni is not None else (0, 0, 1), dtype=np.float64)
        s.k_uni = np.full(n, float(k_uni))
        s.e_uni = np.tile(e / np.linalg.norm(e), (n, 1))
    if k_cub != 0.0:
        s.k_cub = np.full(n, float(k_cub))
    if spin_norm != 1.0:
        s.spin_norm = np.full(n, float(spin_norm))
    return s


def _clusters(n_groups: int, size: int, J: float) -> tuple:
    """Disconnected complete graphs K_size; row order: increasing neighbour index."""
    n = n_groups * size
    nbr = np.full((n, size - 1), -1, dtype=np.int64)
    for a in range(size):
        others = [b for b in range(size) if b != a]
        for k, b in enumerate(others):
            nbr[a::size, k] = np.arange(n_groups) * size + b
    return _csr_from_neighbour_table(nbr, np.full(nbr.shape, float(J)))


def dimers(n_pairs: int, J: float = 1.0) -> Sample:
    """n_pairs disconnected two-spin systems (sites 2p and 2p+1 linked)."""
    row_ptr, col, Jv = _clusters(n_pairs, 2, J)
    return Sample(name=f"dimers{n_pairs}", row_ptr=row_ptr, col=col, J=Jv)


def triangles(n_tri: int, J: float = -1.0) -> Sample:
    """n_tri disconnected three-spin rings (complete graph K3); J < 0 is frustrated."""
    row_ptr, col, Jv = _clusters(n_tri, 3, J)
    return Sample(name=f"triangles{n_tri}", row_ptr=row_ptr, col=col, J=Jv)


_FCC_OFFSETS = np.array(
    [
        (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
        (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
        (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1),
    ],
    dtype=np.int64,
)


def fcc_sphere(radius: float, a: float = 1.0, centre: Sequence[float] = (0.0, 0.0, 0.0), J: float = 1.0) -> Sample:
    """Sphere cut from an fcc lattice of conventional cube side a (open surface).

    Lattice points are (a/2)*(i, j, k) with i+j+k even; nearest neighbours sit at the 12
    offsets (+-1, +-1, 0) and permutations (distance a/sqrt 2). Sites are kept when
    |r - centre| <= radius and numbered in (i, j, k) lexicographic order; each row lists
    the neighbours present in the fixed offset order. The sample carries the sublattice
    colouring (4 colour classes).
    """
    c = np.asarray(centre, dtype=np.float64)
    h = a / 2.0
    lo = np.floor((c - radius) / h).astype(np.int64) - 1
    hi = np.ceil((c + radius) / h).astype(np.int64) + 1
    shape = tuple((hi - lo + 1).tolist())
    ii, jj, kk = np.meshgrid(
        np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1), np.arange(lo[2], hi[2] + 1), indexing="ij"
    )
    pos = np.stack([ii, jj, kk], axis=-1).astype(np.float64) * h
    d2 = ((pos - c) ** 2).sum(axis=-1)
    keep = (((ii + jj + kk) % 2) == 0) & (d2 <= radius * radius)
    index = np.full(shape, -1, dtype=np.int64)
    coords = np.argwhere(keep)
    n = coords.shape[0]
    index[keep] = np.arange(n)
    nbr = np.full((n, 12), -1, dtype=np.int64)
    for k, off in enumerate(_FCC_OFFSETS):
        q = coords + off
        inside = np.all((q >= 0) & (q < np.asarray(shape)), axis=1)
        qq = q[inside]
        nbr[inside, k] = index[qq[:, 0], qq[:, 1], qq[:, 2]]
    row_ptr, col, Jv = _csr_from_neighbour_table(nbr, np.full((n, 12), float(J)))
    s = Sample(name=f"fcc_r{radius:g}", row_ptr=row_ptr, col=col, J=Jv)
    ijk = coords + lo
    s.positions = ijk.astype(np.float64) * h
    # the four simple-cubic sublattices of the fcc lattice: every nearest-neighbour offset
    # changes the parity of exactly two of i, j, k, so (i mod 2) + 2 (j mod 2) is a proper
    # colouring with 4 classes (the greedy colouring in site order needs 7 on these spheres)
    s.colour = ((ijk[:, 0] & 1) + 2 * (ijk[:, 1] & 1)).astype(np.int32)
    s.meta = {"radius": radius, "a": a, "centre": c.tolist()}
    return s


def core_shell_particle(
    seed: int,
    radius: float = 12.0,
    core_radius: float = 9.0,
    a: float = 1.0,
    J_core: float = 1.0,
    J_shell: float = 0.5,
    J_interface: float = -0.3,
    k_surface: float = 0.5,
) -> Sample:
    """Core/shell sphere cut from fcc (type 0 core: |r-c| <= core_radius; type 1 shell).

    The centre is the lattice origin plus a seeded uniform offset in [0, a)^3. Bond
    exchange follows the endpoint types (core-core, shell-shell, core-shell). Surface
    sites (fewer than 12 neighbours in the cut) carry uniaxial anisotropy k_surface along
    the radial unit vector.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    centre = rng.uniform(0.0, 1.0, size=3) * a
    s = fcc_sphere(radius, a=a, centre=centre)
    n = s.n_sites
    r = s.positions - centre
    dist = np.sqrt((r * r).sum(axis=1))
    typ = np.where(dist <= core_radius, 0, 1).astype(np.int32)
    src = np.repeat(np.arange(n), np.diff(s.row_ptr))
    t0, t1 = typ[src], typ[s.col]
    J = np.where((t0 == 0) & (t1 == 0), J_core, np.where((t0 == 1) & (t1 == 1), J_shell, J_interface))
    s.J = J.astype(np.float64)
    s.type = typ
    deg = np.diff(s.row_ptr)
    surf = deg < 12
    s.k_uni = np.where(surf, k_surface, 0.0)
    e = np.zeros((n, 3))
    e[:, 2] = 1.0
    safe = dist > 0
    e[surf & safe] = r[surf & safe] / dist[surf & safe, None]
    s.e_uni = e
    s.name = f"coreshell_r{radius:g}"
    s.meta.update({"seed": seed, "core_radius": core_radius, "n_surface": int(surf.sum())})
    return s


def nanoparticle_batch(
    n_particles: int, seed: int, r_min: float = 3.0, r_max: float = 15.0, a: float = 4.0 ** (1.0 / 3.0)
) -> list:
    """Independent fcc spheres with radii uniform in [r_min, r_max] and seeded centres.

    The default cube side 4^(1/3) gives one site per unit volume, so a radius-r particle
    holds about (4/3) pi r^3 sites (about 113 at r=3 and 14k at r=15).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    radii = rng.uniform(r_min, r_max, size=n_particles)
    offs = rng.uniform(0.0, 1.0, size=(n_particles, 3)) * a
    out = []
    for p in range(n_particles):
        s = fcc_sphere(float(radii[p]), a=a, centre=offs[p])
        s.name = f"np{p}_r{radii[p]:.2f}"
        out.append(s)
    return out


def random_graph(n: int, p: float, seed: int, all_terms: bool = True) -> Sample:
    """Erdos-Renyi graph with Gaussian exchange and (optionally) random site terms.

    Used for exact energy-difference checks: random spin norms in [0.5, 1.5], random
    field and anisotropy axes, uniaxial and cubic constants of either sign.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    upper = np.triu(rng.uniform(size=(n, n)) < p, k=1)
    Jm = np.where(upper, rng.normal(size=(n, n)), 0.0)
    Jm = Jm + Jm.T
    adj = upper | upper.T
    rows, cols = np.nonzero(adj)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    s = Sample(name=f"er{n}", row_ptr=row_ptr, col=cols.astype(np.int32), J=Jm[rows, cols].astype(np.float64))
    if all_terms:
        def unit(m):
            v = rng.normal(size=(m, 3))
            return v / np.linalg.norm(v, axis=1, keepdims=True)

        s.spin_norm = rng.uniform(0.5, 1.5, size=n)
        s.field_axis = unit(n)
        s.k_uni = rng.normal(size=n)
        s.e_uni = unit(n)
        s.k_cub = rng.normal(size=n)
        s.type = rng.integers(0, 3, size=n).astype(np.int32)
    return s
