"""Writes the oracle's regression fixtures in this folder (run from the repository root:
`python tests/golden/make_golden.py`). It calls only the oracle and the seeded input
generators.

The paper prints no worked example with values for the sweep, so none of these files is a
pin of the oracle to the paper: they record what the oracle computes today, bit for bit (hex
floats), so that any later change to its arithmetic shows up in tests/test_golden.py and has
to be made on purpose, together with these files.

  oracle_sc4_chain.txt    Eq. 1-4, Sec. III.B: a 4^3 periodic +-J lattice with uniaxial
                          anisotropy and a field, 2 replicas, 2 steps x 10 MCS, seed 5: the
                          (E, Mx, My, Mz) history and the accepted counts of every MCS, and
                          the final spins' sums
  oracle_ising_chain.txt  Sec. II (Ising, spin flip): 8 x 8 periodic square lattice, 4
                          replicas, 12 MCS, seed 7: the (E, M) history
  oracle_thermal.txt      Sec. II, IV.A-B (thermal averages, cumulants, tau): the 16 fields
                          of a fixed synthetic history
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import analysis  # noqa: E402
from lattices import sc_periodic  # noqa: E402


def sc4_chain():
    s = sc_periodic(4, bimodal_seed=3, k_uni=0.2)
    T = np.array([[1.5, 0.9], [0.8, 0.6]])
    B = np.array([[0.1, 0.2], [-0.1, 0.0]])
    r = oracle.run(s, T, B, 10, seed=5)
    rows = [("history", r["history"].reshape(-1)), ("accepted", r["accepted"].reshape(-1).astype(np.float64)),
            ("spin_sums", r["spins"].sum(axis=1).reshape(-1))]
    return rows


def ising_chain():
    T = np.array([[2.0], [2.3], [2.6], [3.0]])
    h = np.array([[0.0], [0.1], [-0.1], [0.05]])
    r = oracle.ising_run(2, 8, 1.0, T, h, 12, seed=7)
    return [("history", r["history"].reshape(-1))]


def thermal():
    t = np.arange(2000, dtype=np.float64)
    E = -400.0 + 10.0 * np.sin(0.05 * t) + 3.0 * np.cos(0.31 * t)
    M = np.stack([30.0 + 2.0 * np.sin(0.02 * t), 5.0 * np.cos(0.07 * t), 1.0 + 0.5 * np.sin(0.11 * t)], axis=1)
    series = np.concatenate([E[:, None], M], axis=1)
    d = analysis.thermal_averages(series, cut=200, n_bins=20, T=1.3, N=512.0)
    return [("fields", np.array([float(d[k]) for k in sorted(d)])), ("names", None, sorted(d))]


def write(name, rows, header):
    with open(os.path.join(HERE, name), "w") as f:
        f.write("# " + header + "\n# written by tests/golden/make_golden.py from the oracle; hex floats\n")
        for row in rows:
            if row[1] is None:
                f.write(row[0] + " " + " ".join(row[2]) + "\n")
            else:
                f.write(row[0] + " " + " ".join(float(v).hex() for v in row[1]) + "\n")


def main():
    write("oracle_sc4_chain.txt", sc4_chain(), "Eq. 1-4, Sec. III.B: 4^3 +-J lattice, k = 0.2, 2 replicas, 2 x 10 MCS")
    write("oracle_ising_chain.txt", ising_chain(), "Sec. II Ising with spin flips: 8 x 8 square, 4 replicas, 12 MCS")
    write("oracle_thermal.txt", thermal(), "Sec. II, IV.A-B: thermal averages of a fixed synthetic history")


if __name__ == "__main__":
    main()
