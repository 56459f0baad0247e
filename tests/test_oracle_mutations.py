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
import test_oracle_policies as pol
import test_oracle_outputs as outs
import test_oracle_ising as ising

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
    ("spin norm ignored in trial", "        Sp[0] = sn * u[0];\n        Sp[1] = sn * u[1];\n        Sp[2] = sn * u[2];",
     "        Sp[0] = u[0];\n        Sp[1] = u[1];\n        Sp[2] = u[2];", [pins.test_langevin_law_spin_norm]),
    ("colouring not greedy", "while (c < cap && mark[c] == i) ++c;", "while (c < cap && mark[c] == i) c += 2;",
     [lambda: pins.test_greedy_colouring_matches_networkx(lambda: pins.sc_periodic(5))]),
    ("exchange sign", "ex += s->J[e] *", "ex -= s->J[e] *", [lambda: pins.test_three_spin_ring(-1.0)]),
    ("cap height not scaled by s", "const double z = 1.0 - sh;", "const double z = 1.0 - h;",
     [lambda: pol.test_small_step_uniform_in_cap(1.0)]),
    ("cap radius factor", "const double r = sqrt(h * (2.0 - sh));", "const double r = sqrt(h * (1.0 - sh));",
     [lambda: pol.test_small_step_uniform_in_cap(1.0)]),
    ("polar method factor", "sqrt((-2.0 * vo_log(s)) / s)", "sqrt((-1.0 * vo_log(s)) / s)",
     [pol.test_gaussian_offsets_are_standard_normals]),
    ("log series term dropped", "k >= 1; k -= 2", "k >= 3; k -= 2", [pol.test_log_series_matches_libm]),
    ("Gaussian third normal reused", "sigma * g1[0]}", "sigma * g0[0]}", [pol.test_gaussian_wide_is_uniform]),
    ("Hinzke-Nowak thirds", "vo_uniform(jb->seed, c0, t, inst, 0x0C000u) * 3.0", "vo_uniform(jb->seed, c0, t, inst, 0x0C000u) * 2.5",
     [pol.test_hinzke_nowak_mixture]),
    ("adaptive law inverted", "jb->sigma * (0.5 / f)", "jb->sigma * (f / 0.5)",
     [pol.test_adaptive_acceptance_and_control_law]),
    ("adaptation never frozen", "m < jb->mcs / 5", "m < jb->mcs", [pol.test_adaptive_acceptance_and_control_law]),
    ("flip keeps the spin", "out[0] = -Si[0] / sn;", "out[0] = Si[0] / sn;", [pol.test_spin_flip_trial_is_minus_s]),
    ("type magnetization in one slot", "th[3 * ty + q] += jb->S[3 * (int64_t)i + q];",
     "th[q] += jb->S[3 * (int64_t)i + q];", [outs.test_type_magnetizations_add_up_and_match_the_final_states]),
    ("type magnetization components transposed", "th[3 * ty + q] += jb->S[3 * (int64_t)i + q];",
     "th[3 * ty + q] += jb->S[3 * (int64_t)i + 2 - q];", [outs.test_two_phases_follow_their_own_field_axes]),
    ("snapshot before the renormalisation",
     "        vo_renormalise(s, jb->S);\n        if (jb->snaps) memcpy(",
     "        if (jb->snaps) memcpy(jb->snaps + (int64_t)st * n * 3, jb->S, sizeof(double) * 3 * (size_t)n);\n"
     "        vo_renormalise(s, jb->S);\n        if (0) memcpy(",
     [outs.test_snapshots_are_the_final_states_per_step]),
    ("qIsing proposal skips no value", "        if (k >= idx) k += 1;\n", "",
     [lambda: pol.test_qising_free_spins_boltzmann(1.0, 0.6, 0.8)]),
    ("qIsing sites renormalised", "        if (is_qising(s, i)) continue;  /* discrete values keep their length */", "",
     [pol.test_qising_values_stay_discrete_and_start_uniform, lambda: pol.test_qising_free_spins_boltzmann(1.5, 0.4, -0.3)]),
    ("qIsing start misses the top value", "0x20000u) * (double)nv);", "0x20000u) * (double)(nv - 1));",
     [pol.test_qising_values_stay_discrete_and_start_uniform]),
    ("Ising field sign", "const double dE = 2.0 * si * (J * (double)sum + hh);",
     "const double dE = 2.0 * si * (J * (double)sum - hh);", [ising.test_paramagnet_tanh_law]),
    ("Ising bonds counted twice", "for (int d = 0; d < dims; ++d) bsum += (int64_t)s[i] * s[nb[2 * d + 1]];",
     "for (int d = 0; d < 2 * dims; ++d) bsum += (int64_t)s[i] * s[nb[d]];",
     [ising.test_four_by_four_exact_averages]),
    ("Ising acceptance without beta", "acc = (double)w[inst & 3u] * 0x1p-32 < exp(-(beta * dE));",
     "acc = (double)w[inst & 3u] * 0x1p-32 < exp(-(dE));", [ising.test_paramagnet_tanh_law]),
    ("Ising neighbour along the wrong axis", "q[d] = (q[d] + sgn + L) % L;", "q[0] = (q[0] + sgn + L) % L;",
     [ising.test_four_by_four_exact_averages, ising.test_onsager_energy_and_spontaneous_magnetization]),
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


# --------------------------------------------------------------------------- analysis (numpy)

import types  # noqa: E402

import test_oracle_analysis as ana  # noqa: E402
from oracle import analysis as _analysis  # noqa: E402

ASRC = open(_analysis.__file__).read()

ANALYSIS_MUTANTS = [
    ("specific heat without T^2", "c = np.var(E) / (N * T * T)", "c = np.var(E) / (N * T)",
     [ana.test_thermal_averages_of_gaussian_series]),
    ("Binder factor", "u4 = 1.0 - np.mean(M2 * M2) / (3.0 * np.mean(M2) ** 2)",
     "u4 = 1.0 - np.mean(M2 * M2) / (2.0 * np.mean(M2) ** 2)", [ana.test_thermal_averages_of_gaussian_series]),
    ("cumulant sign", 'out["v1"] = E.mean() - np.mean(A * E) / A.mean()',
     'out["v1"] = np.mean(A * E) / A.mean() - E.mean()', [ana.test_cumulants_v1_v2_of_independent_ising_spins]),
    ("autocorrelation doubled", "        tau += rho", "        tau += 2.0 * rho", [ana.test_tau_of_ar1_series]),
    ("jackknife factor", "np.sqrt((n_bins - 1) / n_bins *", "np.sqrt(1.0 / n_bins *",
     [ana.test_thermal_averages_of_gaussian_series]),
    ("reweighting sign", "g_new = np.logaddexp.reduce(-np.outer(bk, Ei) - D[None, :], axis=1)",
     "g_new = np.logaddexp.reduce(np.outer(bk, Ei) - D[None, :], axis=1)",
     [ana.test_multiple_histogram_interpolation_and_free_energies]),
    ("reweighting weight of the target", "        lw = -b * Ei - D", "        lw = -b * Ei + D",
     [ana.test_single_histogram_reweighting_of_free_spins]),
]


@pytest.mark.parametrize("name,old,new,checks", ANALYSIS_MUTANTS, ids=[m[0] for m in ANALYSIS_MUTANTS])
def test_analysis_pins_catch_mutant(name, old, new, checks):
    assert ASRC.count(old) == 1, name
    mod = types.ModuleType("analysis_mutant")
    exec(compile(ASRC.replace(old, new), "analysis_mutant.py", "exec"), mod.__dict__)
    saved = ana.analysis
    ana.analysis = mod
    try:
        assert any(_fails(c) for c in checks), f"no pin caught: {name}"
    finally:
        ana.analysis = saved
