"""The oracle's pins must catch plausible mistakes (no GPU).

Each case compiles a copy of vegas_oracle.c with one deliberate error (a flipped sign, a
dropped factor, a wrong index, a transposed operand, a wrong constant) and checks that at
least one of the named pins in test_oracle_pins.py fails against that copy. Mistakes are
planted only in the CPU oracle.
"""

import os
import tempfile

import pytest

import oracle
from oracle import oracle as ora
import test_oracle_pins as pins

SRC = open(os.path.join(os.path.dirname(ora.__file__), "vegas_oracle.c")).read()

MUTANTS = [
    ("zeeman sign in dE", "hx = hx + B * n[0];", "hx = hx - B * n[0];",
     [pins.test_langevin_law_zeeman, pins.test_delta_e_equals_energy_difference]),
    ("bond counted twice", "return -0.5 * ex", "return -1.0 * ex",
     [pins.test_energy_pair_angle_and_norms]),
    ("anisotropy sign in dE", "const double dEan = -(k * (pn * pn - po * po));",
     "const double dEan = (k * (pn * pn - po * po));",
     [lambda: pins.test_single_spin_uniaxial(2.0)]),
    ("cubic form term", "return (xx * yy + yy * zz) + xx * zz;", "return (xx * yy + yy * zz) + xx * xx;",
     [pins.test_energy_cubic_axes]),
    ("neighbour index in field", "const double *Sj = S + 3 * (int64_t)s->col[e];\n        const double J = s->J[e];",
     "const double *Sj = S + 3 * (int64_t)i;\n        const double J = s->J[e];",
     [lambda: pins.test_open_heisenberg_chain(1.0, 2.0)]),
    ("temperature dropped from acceptance", "acc = r < exp(-(beta * dE));", "acc = r < exp(-(dE));",
     [lambda: pins.test_open_heisenberg_chain(1.0, 0.5)]),
    ("sphere z component", "out[2] = 1.0 - 2.0 * s;", "out[2] = 1.0 - s;",
     [pins.test_sphere_sampler_uniform]),
    ("philox multiplier", "0xD2511F53u * c[0]", "0xD2511F55u * c[0]",
     [pins.test_philox_matches_triton_interpreter]),
    ("philox output words transposed", "c[1] = lo1;\n    c[2] = n2;\n    c[3] = lo0;",
     "c[1] = lo0;\n    c[2] = n2;\n    c[3] = lo1;", [pins.test_philox_matches_triton_interpreter]),
    ("spin norm ignored in trial", "const double Sp[3] = {sn * u[0], sn * u[1], sn * u[2]};",
     "const double Sp[3] = {u[0], u[1], u[2]};", [pins.test_langevin_law_spin_norm]),
    ("colouring not greedy", "while (c < cap && mark[c] == i) ++c;", "while (c < cap && mark[c] == i) c += 2;",
     [lambda: pins.test_greedy_colouring_matches_networkx(lambda: pins.sc_periodic(5))]),
    ("exchange sign", "ex += s->J[e] *", "ex -= s->J[e] *", [lambda: pins.test_three_spin_ring(-1.0)]),
]


def _fails(check) -> bool:
    try:
        check()
    except AssertionError:
        return True
    except pytest.skip.Exception:
        pytest.skip("a pin needed for this mutant is skipped here")
    return False


@pytest.mark.parametrize("name,old,new,checks", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new, checks):
    assert SRC.count(old) >= 1, f"mutation site for '{name}' not found"
    text = SRC.replace(old, new)
    with tempfile.TemporaryDirectory() as d:
        path = oracle.oracle.compile_source(text, os.path.join(d, "mutant.so"))
        with ora.use_library(path):
            assert any(_fails(c) for c in checks), f"no pin caught: {name}"
