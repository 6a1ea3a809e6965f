"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a wrong index,
a wrong total ...) in a temporary copy of ``oracle/uf_oracle.c``, builds it
with gcc on the CPU and runs the pins of ``test_oracle_pins`` against it: at
least one pin must fail.  The committed oracle is never modified.
"""
import os

import pytest

import oracle
from tests import test_oracle_pins as pins
from tests import test_oracle_variants as variants

MUTANTS = {
    "xor_as_or": ("num += l * (double)(xa ^ xb);", "num += l * (double)(xa | xb);"),
    "or_as_and": ("den += l * (double)(xa | xb);", "den += l * (double)(xa & xb);"),
    "unnormalized_drops_length": ("num += l * fabs(pA - pB);\n            break;",
                                  "num += fabs(pA - pB);\n            break;"),
    "normalized_den_sign": ("den += l * (pA + pB);", "den += l * (pA - pB);"),
    "generalized_drops_div_s": ("num += l * sa * fabs(pA - pB) / s;", "num += l * sa * fabs(pA - pB);"),
    "generalized_alpha_flipped": ("pow(s, J->alpha)", "pow(s, 1.0 - J->alpha)"),
    "generalized_zero_s_kept": ("if (s > 0.0) {\n                const double sa",
                                "if (s >= 0.0) {\n                const double sa"),
    "root_branch_included": ("for (int64_t v = 0; v + 1 < J->n_nodes; v++) {\n        const double l",
                             "for (int64_t v = 0; v < J->n_nodes; v++) {\n        const double l"),
    "wrong_total": ("pB = CB[v] / TB;", "pB = CB[v] / TA;"),
    "sum_overwrites": ("C[J->parent[v]] += C[v];", "C[J->parent[v]] = C[v];"),
    "feature_as_node": ("C[J->tip_node[J->indices[q]]] = J->data[q];", "C[J->indices[q]] = J->data[q];"),
    "total_counts_nnz": ("t += J->data[q];\n    return t;", "t += 1.0;\n    return t;"),
    "zero_den_gives_one": ("d = (den == 0.0) ? 0.0 : num / den;", "d = (den == 0.0) ? 1.0 : num / den;"),
    "counts_not_proportions": ("num += l * fabs(pA - pB);\n            den", "num += l * fabs(CA[v] - CB[v]);\n            den"),
    "tips_numbered_from_one": ("for (int64_t i = 0; i < n_nodes; i++)\n        if (!has_child[i])",
                               "for (int64_t i = 1; i < n_nodes; i++)\n        if (!has_child[i])"),
    # further family members
    "unweighted_unnormalized_divides": ("return method == UO_WEIGHTED_UNNORMALIZED || method == UO_UNWEIGHTED_UNNORMALIZED ||",
                                        "return method == UO_WEIGHTED_UNNORMALIZED ||"),
    "vaw_drops_sqrt": ("const double w = 1.0 / sqrt(mv * rest);", "const double w = 1.0 / (mv * rest);"),
    "vaw_rest_is_total": ("rest = (TA + TB) - mv;\n            if", "rest = (TA + TB);\n            if"),
    "vaw_weight_from_proportions": ("const double mv = CA[v] + CB[v], rest",
                                    "const double mv = pA + pB, rest"),
    "vaw_full_branch_kept": ("if (mv > 0.0 && rest > 0.0) {\n                const double w",
                             "if (mv > 0.0 && rest >= 0.0 && rest + mv > 0.0) {\n                const double w"),
    "vaw_den_drops_weight": ("den += l * w * (pA + pB);", "den += l * (pA + pB);"),
}

CHECKS = [pins.check_two_tip, pins.check_three_tip, pins.check_star_textbook,
          pins.check_path_enumeration, pins.check_hand_small, pins.check_invariants,
          pins.check_structural, pins.check_zero_lengths, pins.check_earth_movers,
          variants.check_variant_two_tip, variants.check_variant_three_tip, variants.check_variant_star,
          variants.check_hand_variants, variants.check_variant_paths, variants.check_variant_invariants]


def _run_checks(lib):
    failed = []
    for check in CHECKS:
        try:
            check(lib=lib)
        except (AssertionError, oracle.OracleError, ValueError, ZeroDivisionError) as e:
            failed.append((check.__name__, type(e).__name__))
    return failed


def test_unmutated_copy_passes(tmp_path):
    src = open(oracle.SRC).read()
    path = tmp_path / "uf_oracle.c"
    path.write_text(src)
    lib = oracle.load(oracle.build(str(path), str(tmp_path / "lib.so"), force=True))
    assert _run_checks(lib) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    before, after = MUTANTS[name]
    src = open(oracle.SRC).read()
    assert before in src, f"mutation site for {name} not found"
    path = tmp_path / "uf_oracle.c"
    path.write_text(src.replace(before, after, 1))
    lib = oracle.load(oracle.build(str(path), str(tmp_path / "lib.so"), force=True))
    failed = _run_checks(lib)
    assert failed, f"no pin caught mutant {name}"
