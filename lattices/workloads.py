"""The five workloads the sweep is measured and tested on, as plain input specs.

Each workload is a list of samples, a replica count per sample, and a schedule of
temperatures and fields per instance (instances are numbered sample-major:
inst = sample * replicas + replica). k_B = 1 throughout (Sec. III.C).

  sc8_fp64       8^3 periodic sc ferromagnet, J=1, 30 temperatures 3.0 -> 0.1, 1000 MCS, FP64
  sc64_hyst      64^3 periodic sc, J=1, K=0.05 along z, T=0.5, B_z 2 -> -2 -> 2 in 0.05 steps
                 (161 steps), 500 MCS per step, FP32
  coreshell_fc   fcc core/shell sphere r=12 (~29k sites), field-cooled in B_z=0.5 from T=3.0
                 to 0.05 in 60 steps, 2000 MCS each, FP32
  np256          256 fcc nanoparticles, radii U[3,15] (one site per unit volume), each at one
                 of 64 temperatures 0.05..3.0, B=0, 5000 MCS, FP32
  sg256x32       32 temperature replicas of a 256^3 periodic sc +-J spin glass, T geometric
                 0.1 -> 2.0, B=0, 200 MCS, FP32

`scale` shrinks a workload (lattice side, particle count, MCS) for tests that must run
the CPU oracle in seconds; the structure (coordination, colour count, parameter mix) is
kept.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import generators as g


@dataclass
class Workload:
    name: str
    samples: list
    replicas: int
    T: np.ndarray  # [n_inst, n_steps]
    B: np.ndarray  # [n_inst, n_steps]
    mcs: int
    precision: int  # 64 or 32
    seed: int

    @property
    def n_inst(self) -> int:
        return len(self.samples) * self.replicas

    @property
    def n_steps(self) -> int:
        return int(self.T.shape[1])

    @property
    def n_sites_total(self) -> int:
        return sum(s.n_sites for s in self.samples) * self.replicas

    def attempts(self) -> int:
        """Metropolis attempts of the whole schedule (one per site per MCS)."""
        return self.n_sites_total * self.n_steps * self.mcs


def hysteresis_fields(b_max: float = 2.0, db: float = 0.05) -> np.ndarray:
    """+b_max -> -b_max -> +b_max in steps of db; -b_max is not repeated."""
    k = int(round(b_max / db))
    down = b_max - db * np.arange(2 * k + 1)
    up = -b_max + db * np.arange(1, 2 * k + 1)
    return np.concatenate([down, up])


def workload(name: str, scale: float = 1.0, mcs: int | None = None, seed: int = 1) -> Workload:
    if name == "sc8_fp64":
        s = g.sc_periodic(8)
        T = np.linspace(3.0, 0.1, 30)[None, :]
        return Workload(name, [s], 1, T, np.zeros_like(T), mcs or 1000, 64, seed)
    if name == "sc64_hyst":
        L = max(4, int(round(64 * scale)))
        L += L % 2
        s = g.sc_periodic(L, J=1.0, k_uni=0.05, e_axis=(0, 0, 1))
        B = hysteresis_fields()[None, :]
        T = np.full_like(B, 0.5)
        return Workload(name, [s], 1, T, B, mcs or 500, 32, seed)
    if name == "coreshell_fc":
        s = g.core_shell_particle(seed=seed, radius=12.0 * scale, core_radius=9.0 * scale)
        T = np.linspace(3.0, 0.05, 60)[None, :]
        return Workload(name, [s], 1, T, np.full_like(T, 0.5), mcs or 2000, 32, seed)
    if name == "np256":
        n = max(4, int(round(256 * scale)))
        samples = g.nanoparticle_batch(n, seed=seed, r_max=3.0 + 12.0 * min(1.0, scale ** 0.5))
        temps = 0.05 + (np.arange(n) % 64) * (2.95 / 63.0)
        T = temps[:, None]
        return Workload(name, samples, 1, T, np.zeros_like(T), mcs or 5000, 32, seed)
    if name == "sg256x32":
        L = max(4, int(round(256 * scale)))
        L += L % 2
        s = g.sc_periodic(L, J=1.0, bimodal_seed=seed)
        R = 32
        T = (0.1 * 20.0 ** (np.arange(R) / (R - 1.0)))[:, None]
        return Workload(name, [s], R, T, np.zeros_like(T), mcs or 200, 32, seed)
    raise KeyError(name)
