"""Plant plausible mistakes in a copy of the oracle and check that a pin catches each.

Every mutant is a one-line edit of oracle/oracle.c (a dropped term, a wrong sign
or index, a transposed operand, a strict instead of inclusive comparison, a
missing tie-break ...). Mutants are chosen so that every index they compute stays
inside its buffer. It is compiled to a temporary library with the same
flags as the real oracle and the full pin suite runs against it: at least one
pin must fail. Runs on the CPU only.
"""

import os

import pytest

import oracle
from oracle_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "square_dropped": ("s = s + t * t;", "s = s + t;"),
    "sum_dropped": ("s = s + t * t;", "s = t * t;"),
    "sign_flipped": ("(double)q[k] - (double)x[k]", "(double)q[k] + (double)x[k]"),
    "index_slip": ("(double)q[k] - (double)x[k]", "(double)q[k] - (double)x[0]"),
    "first_term_dropped": ("for (int32_t k = 0; k < d; ++k)", "for (int32_t k = 1; k < d; ++k)"),
    "strict_threshold": ("if (s <= e2)", "if (s < e2)"),
    "eps_not_squared": ("const double e2 = eps * eps;", "const double e2 = eps;"),
    "diagonal_in_upper": ("int64_t j0 = (mode == 1) ? i + 1 : 0;", "int64_t j0 = (mode == 1) ? i : 0;"),
    "second_operand_is_R": ("const float *T = (mode == 0) ? S : R;", "const float *T = R;"),
    "pair_transposed": ("out_s[cnt] = j;", "out_s[cnt] = i;"),
    "tie_break_reversed": ("return (x->j < y->j) ? -1 : (x->j > y->j);",
                           "return (x->j > y->j) ? -1 : (x->j < y->j);"),
    "topk_descending": ("if (x->d2 < y->d2) return -1;\n    if (x->d2 > y->d2) return 1;",
                        "if (x->d2 < y->d2) return 1;\n    if (x->d2 > y->d2) return -1;"),
    "topk_keep_k": ("int64_t keep = (k < nS) ? k : nS;", "int64_t keep = k;"),
    "cosine_threshold_halved": ("const double e2 = 2.0 - 2.0 * c;", "const double e2 = 2.0 - c;"),
    "norm_not_rooted": ("const float nr = (float)sqrt(s);", "const float nr = (float)s;"),
    "norm_multiplies": ("o[k] = x[k] / nr;", "o[k] = x[k] * nr;"),
    "l1_abs_dropped": ("s = s + fabs(t);", "s = s + t;"),
    "chi2_no_division": ("if (u > 0.0) s = s + (t * t) / u;", "if (u > 0.0) s = s + (t * t);"),
    "chi2_divides_by_q": ("double u = (double)q[k] + (double)x[k];", "double u = (double)q[k];"),
    "hist_join_strict": ("if (s <= eps)", "if (s < eps)"),
    "hist_channels_swapped": ("r = (px[0] * br) >> 8, g = (px[1] * bg) >> 8, b = (px[2] * bb) >> 8;",
                              "r = (px[2] * br) >> 8, g = (px[1] * bg) >> 8, b = (px[0] * bb) >> 8;"),
    "hist_row_stride": ("((f * H + y) * (int64_t)W + x) * 3", "((f * H + y) * (int64_t)H + x) * 3"),
    "hist_area_width_only": ("const float area = (float)((int64_t)(x1 - x0) * (y1 - y0));",
                             "const float area = (float)((int64_t)(x1 - x0));"),
    "hist_joint_index_transposed": ("cnt[(r * bg + g) * bb + b] += 1;", "cnt[(g * br + r) * bb + b] += 1;"),
    "hist_topk_metric_swapped": ("c[j].d2 = (metric == 1) ? oracle_l1dist(q, x, d) : oracle_chi2dist(q, x, d);",
                                 "c[j].d2 = (metric == 2) ? oracle_l1dist(q, x, d) : oracle_chi2dist(q, x, d);"),
    "dot_sign_flipped": ("s = s + (double)q[k] * (double)x[k];", "s = s - (double)q[k] * (double)x[k];"),
    "ip_threshold_strict": (">= t) {", "> t) {"),
    "components_max_label": ("const int64_t lo = (la < lb) ? la : lb;", "const int64_t lo = (la > lb) ? la : lb;"),
    "components_one_pass": ("while (changed) {", "if (changed) {"),
    "components_count_inverted": ("c += (label[i] == i);", "c += (label[i] != i);"),
    "dist_block_transposed": ("out[(i - r0) * nS + j] = oracle_sqdist(",
                              "out[(i - r0) + j * (r1 - r0)] = oracle_sqdist("),
    "dist_block_row_offset_dropped": ("oracle_sqdist(R + i * (int64_t)d, S + j * (int64_t)d, d);",
                                      "oracle_sqdist(R + (i - r0) * (int64_t)d, S + j * (int64_t)d, d);"),
    "hist_block_metric_swapped": ("out[(i - r0) * nS + j] = (metric == 1) ?",
                                  "out[(i - r0) * nS + j] = (metric == 2) ?"),
    "hist_block_transposed": ("out[(i - r0) * nS + j] = (metric == 1) ?",
                              "out[(i - r0) + j * (r1 - r0)] = (metric == 1) ?"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutated = src.replace(old, new, 1)
    path = tmp_path / f"oracle_{name}.c"
    path.write_text(mutated)
    lib = oracle.load(oracle.build(str(path), str(tmp_path / f"lib_{name}.so")))
    orc = oracle.Oracle(lib)
    failed = []
    for pin in ALL_PINS:
        try:
            pin(orc)
        except AssertionError:
            failed.append(pin.__name__)
        except (IndexError, ValueError, MemoryError, OverflowError, StopIteration):
            failed.append(pin.__name__)
    assert failed, f"mutant {name} passed every pin"
