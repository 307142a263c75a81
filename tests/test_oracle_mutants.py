"""Plant plausible mistakes in a copy of the oracle's C source and check that the
pins catch every one: a pin set that a dropped term, a flipped sign or a wrong
index slips through is too weak to trust the oracle with."""
import os

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "pgg_oracle.c")

MUTANTS = {
    "cooperator_cost_dropped": ("pi += s ? (share - c) : share;", "pi += share;"),
    "payoff_total_sign": ("return (r * (double)S) / 5.0 - 5.0 * (double)s;",
                          "return (r * (double)S) / 5.0 + 5.0 * (double)s;"),
    "group_size_4": ("return (r * (double)S) / 5.0 - 5.0 * (double)s;",
                     "return (r * (double)S) / 4.0 - 5.0 * (double)s;"),
    "fermi_sign": ("exp((pi_x - pi_y) / K)", "exp((pi_y - pi_x) / K)"),
    "fermi_K_multiplied": ("exp((pi_x - pi_y) / K)", "exp((pi_x - pi_y) * K)"),
    "group_without_centre": ("int n = strategy_at(lat, L, ci, cj);", "int n = 0;"),
    "neighbour_table_typo": ("static const int NB_DI[4] = {0, 0, 1, -1};",
                             "static const int NB_DI[4] = {0, 0, 1, 1};"),
    "comparator_flipped": ("if (u < t) {", "if (u > t) {"),
    "init_inverted": ("lat[x] = ((uint64_t)w[x & 3] < thr) ? 1 : 0;",
                      "lat[x] = ((uint64_t)w[x & 3] < thr) ? 0 : 1;"),
    "count_everything": ("c += lat[x] ? 1 : 0;", "c += 1;"),
    "row_offset_ignored": ("int i = 4 * a + oi, j = 4 * b + oj;",
                           "int i = 4 * a, j = 4 * b + oj;"),
    "philox_key_bump": ("k1 += PHILOX_W1;", "k1 += PHILOX_W0;"),
    "philox_word_swap": ("uint32_t n1 = lo1;", "uint32_t n1 = lo0;"),
    "total_misses_one_group": ("for (int d = 0; d < 4; ++d)\n        S += oracle_group_cooperators",
                               "for (int d = 0; d < 3; ++d)\n        S += oracle_group_cooperators"),
    # the random-stream layout
    "dir_field_width": ("return (int)((word >> (2 * (b & 15))) & 3u);", "return (int)((word >> (2 * (b & 7))) & 3u);"),
    "dir_word_index": ("uint32_t word = w[(b >> 4) & 3];", "uint32_t word = w[(b >> 3) & 3];"),
    "u_word_index": ("    return w[b & 3];", "    return w[(b + 1) & 3];"),
    "offset_nibble": ("return (int)((word >> (4 * (k & 7))) & 15u);", "return (int)((word >> (4 * (k & 3))) & 15u);"),
    "u_counter_row": ("philox_seeded(seed, b >> 2, a, (uint32_t)k,", "philox_seeded(seed, b >> 2, a + 1, (uint32_t)k,"),
    # the pairwise game (Section VI)
    "pair_sucker_temptation_swapped": ("return s_other ? pay[0] : pay[1];", "return s_other ? pay[0] : pay[2];"),
    "pair_total_complement_5": ("(double)(4 - n) * b;", "(double)(5 - n) * b;"),
    "pair_count_includes_self": ("int n = 0;\n    for (int d = 0; d < 4; ++d)\n        n += strategy_at",
                                 "int n = strategy_at(lat, L, i, j);\n    for (int d = 0; d < 4; ++d)\n        n += strategy_at"),
    "pair_defector_row_ignored": ("double a = s ? pay[0] : pay[2];", "double a = pay[0];"),
    "pair_threshold_args_swapped": ("return oracle_fermi_threshold(px, py, K);",
                                    "return oracle_fermi_threshold(py, px, K);"),
    "pair_ny_counted_at_x": ("int ny = oracle_pair_neighbour_cooperators(lat, L, yi, yj);",
                             "int ny = oracle_pair_neighbour_cooperators(lat, L, i, j);"),
    "pair_games_skip_one": ("for (int d = 0; d < 4; ++d)\n        pi += pair_matrix",
                            "for (int d = 0; d < 3; ++d)\n        pi += pair_matrix"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    so = oracle.compile_source(str(mutated), str(tmp_path / "libmutant.so"))
    o = oracle.Oracle(oracle.load(so))
    failures = []
    for pin in P.FAST_PINS:
        try:
            pin(o)
        except AssertionError:
            failures.append(pin.__name__)
    assert failures, f"no pin caught mutant {name}"
