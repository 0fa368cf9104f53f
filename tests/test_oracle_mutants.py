"""Pin strength: plausible mistakes planted in a copy of the oracle (on the
CPU) must each make at least one pin fail.

Each mutant rebuilds the oracle with one textual change, swaps it in, runs
the pins listed for it, and expects a failure.  The mutants follow the
paper's steps: the transfer probability of Eq. 1, the mean occupancy of
Eq. 2-3, the conditional binomials of the multinomial split (Sec. II.B), the
per-molecule thresholds, the discarded SSA event past tau (Algorithm 1,
Step 2), the occupancy integral, the reverse face of the synchronous apply,
the second-order propensity constant.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

from tests import test_oracle_laws as L

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE = os.path.join(os.path.dirname(HERE), "oracle")

MUTANTS = {
    "transfer_probability_1_minus_exp": (
        "    double z = tau_k * (D * Gt);\n    return z > 1.0 ? 1.0 : z;",
        "    double z = tau_k * (D * Gt);\n    return 1.0 - own_exp(-(z > 1.0 ? 1.0 : z));",
        [lambda o: L.test_exact_law_of_pure_diffusion(o, 300)]),
    "no_mean_correction": (
        "    } else if (P.rule == kRuleMean && touched) {\n        Stream rs(",
        "    } else if (false) {\n        Stream rs(",
        [L.test_mean_corrected_transfer]),
    "rounding_to_nearest": (
        "Nstar = (int64_t)fl + (rs.u01() < frac ? 1 : 0);",
        "Nstar = (int64_t)fl + (frac >= 0.5 ? 1 : 0);",
        [lambda o: L.test_mean_rule_exact_law(o, 0, 2.0, 1.0, 40000)]),
    "no_cap_at_molecules_present": (
        "            if (moved == Nt) break;",
        "            if (false) break;",
        [L.test_transfer_is_capped_by_the_molecules_present]),
    "dimer_counts_ordered_pairs": (
        "else if (nu == 2) h = h * (N[s] * (N[s] - 1) / 2);",
        "else if (nu == 2) h = h * (N[s] * N[s] / 2);",
        [L.test_production_and_dimer_decay_matches_master_equation]),
    "outlier_rank_off_by_one": (
        "    const double dsel = dt[P.outliers];",
        "    const double dsel = dt[P.outliers > 0 ? P.outliers - 1 : 0];",
        [lambda o: L.test_outlier_option_takes_tau_from_the_next_tet(o, 1)]),
    "mid_rule_takes_end_count": (
        "        Nstar = Nmid;",
        "        Nstar = Nt;",
        [lambda o: L.test_comparison_rules_exact_laws(o, 2)]),
    "mid_snapshot_at_end": (
        "if (!past_half && tn >= half) {",
        "if (!past_half && tn >= tau_k) {",
        [lambda o: L.test_comparison_rules_exact_laws(o, 2)]),
    "end_rule_rounds_occupancy": (
        "    } else if (P.rule == kRuleMean && touched) {\n        Stream rs(",
        "    } else if (touched) {\n        Stream rs(",
        [lambda o: L.test_comparison_rules_exact_laws(o, 1)]),
    "split_without_renormalisation": (
        "int64_t nf = binomial(m, g[f] / suf[f], st);",
        "int64_t nf = binomial(m, g[f] / suf[0], st);",
        [lambda o: L.test_exact_law_of_pure_diffusion(o, 6000)]),
    "thresholds_not_cumulative": (
        "C[f] = threshold_of(zeta * (cum / Gt));",
        "C[f] = threshold_of(zeta * (g[f] / Gt));",
        [lambda o: L.test_exact_law_of_pure_diffusion(o, 6)]),
    "event_past_tau_kept": (
        "if (tn >= tau_k) break;",
        "if (tn >= 2.0 * tau_k) break;",
        [L.test_first_order_decay_is_exactly_binomial, lambda o: L.test_reversible_binding_matches_master_equation(o, True)]),
    "occupancy_sign": (
        "occ[s] = occ[s] + (double)N[s] * (tn - tlast[s]);",
        "occ[s] = occ[s] + (double)N[s] * (tlast[s] - tn);",
        [L.test_mean_corrected_transfer]),
    "wrong_reverse_face": (
        "if (u >= 0) v += out[((size_t)u * S + s) * 4 + rev[4 * t + f]];",
        "if (u >= 0) v += out[((size_t)u * S + s) * 4 + f];",
        [L.test_conservation_and_sign, lambda o: L.test_exact_law_of_pure_diffusion(o, 6)]),
    "second_order_constant": (
        "else c[r] = kr / avv;",
        "else c[r] = kr * avv / 1e12;",
        [lambda o: L.test_reversible_binding_matches_master_equation(o, False)]),
}


def _build_mutant(tmp, old, new):
    src = open(os.path.join(ORACLE, "rdsplit_oracle.cpp")).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    path = os.path.join(tmp, "rdsplit_oracle.cpp")
    open(path, "w").write(src.replace(old, new))
    shutil.copy(os.path.join(ORACLE, "issa.cpp"), os.path.join(tmp, "issa.cpp"))
    lib = os.path.join(tmp, "libmutant.so")
    subprocess.run([os.environ.get("CXX", "g++"), "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
                    "-fPIC", "-shared", "-o", lib, path, os.path.join(tmp, "issa.cpp")], check=True)
    return lib


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(oracle, tmp_path, name):
    old, new, pins = MUTANTS[name]
    lib_path = _build_mutant(str(tmp_path), old, new)
    saved = oracle._lib
    try:
        oracle._lib = None
        real_cdll = ctypes.CDLL
        import oracle.build as ob
        orig = ob.build
        ob.build = lambda force=False: lib_path
        try:
            oracle.lib()
        finally:
            ob.build = orig
        caught = 0
        for pin in pins:
            try:
                pin(oracle)
            except (AssertionError, oracle.OracleError):
                caught += 1
        assert caught > 0, f"mutant {name} passed every pin"
    finally:
        oracle._lib = saved
