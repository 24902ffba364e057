"""The oracle's pins must catch plausible mistakes.

Each case copies ``oracle/argcsr_oracle.c``, plants one mistake by a textual
substitution (a dropped term, a wrong comparison, a transposed index, a
wrong prefix kind ...), builds the copy into a temporary library and re-runs
the pins of ``test_oracle_pins`` against it: at least one pin must fail.
The mistakes live only in those temporary copies, on the CPU.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "argcsr_oracle.c")

MUTANTS = {
    "group_close_on_equal": ("if (count > limit)", "if (count >= limit)"),
    "group_row_cap_off_by_one": ("if (rows == G)", "if (rows == G + 1)"),
    "greedy_double_step": ("t[best] += 1;", "t[best] += 2;"),
    "greedy_fill_floor": ("int64_t f = ceil_div(len[i], t[i]);\n            if (f > bestFill)",
                          "int64_t f = len[i] / t[i];\n            if (f > bestFill)"),
    "threads_floor": ("int64_t threads = chunk == 0 ? 1 : ceil_div(len[i], chunk);",
                      "int64_t threads = chunk == 0 ? 1 : len[i] / chunk;"),
    "threads_keep_greedy": ("if (threads < 1) threads = 1;                        /* A2, A4 */",
                            "if (threads < 1) threads = 1; if (i == size[g] - 1) threads += G - prefix - threads;"),
    "prefix_exclusive": ("prefix += threads;                                   /* A5 */\n"
                         "            if (threadsMapping) threadsMapping[firstRow[g] + i] = (int32_t)prefix;",
                         "if (threadsMapping) threadsMapping[firstRow[g] + i] = (int32_t)prefix;\n"
                         "            prefix += threads;"),
    "offset_by_rows": ("offset += chunk * G;", "offset += chunk * size[g];"),
    "fill_row_major": ("const int64_t slot = offset + (j / V) * G * V + c * V + (j % V);\n"
                       "                    if (slot < 0",
                       "const int64_t slot = offset + c * chunk + j;\n"
                       "                    if (slot < 0"),
    "fill_off_by_one": ("if (e >= len) break;", "if (e > len) break;"),
    "fill_pad_zero_column": ("out_columns[s] = -1;", "out_columns[s] = 0;"),
    "vector_no_roundup": ("if (chunk > 0) chunk = ceil_div(chunk, V) * V;", ";"),
    "spmv_wrong_gather": ("sum += values[k] * x[columns[k]];\n        y[i] = sum;",
                          "sum += values[k] * x[columns[k] / 2];\n        y[i] = sum;"),
    "spmv_drop_first": ("for (int32_t k = rowPointers[i]; k < rowPointers[i + 1]; k++)\n            sum += values[k]",
                        "for (int32_t k = rowPointers[i] + 1; k < rowPointers[i + 1]; k++)\n            sum += values[k]"),
    "argspmv_begin_index": ("const int32_t begin = i == 0 ? 0 : threadsMapping[r - 1];\n            const int32_t end",
                            "const int32_t begin = i == 0 ? 0 : threadsMapping[r - 1] + 1;\n            const int32_t end"),
    "abs_sum_signed": ("sum += p < 0 ? -p : p;", "sum += p;"),
    "one_per_row_ignored": ("one_thread_per_row ? size[g] : G", "G"),
    "one_per_row_spare_thread": ("one_thread_per_row ? size[g] : G", "one_thread_per_row ? size[g] + 1 : G"),
}

# pins that take no arguments, plus parametrised ones with a few arguments
PINS = [
    (pins.test_fig3_adaptive_mapping, ()),
    (pins.test_fig3_one_thread_per_row, ()),
    (pins.test_fig3_without_adaptive_step, ()),
    (pins.test_one_thread_per_row_is_sliced_ellpack_of_the_groups, (32, 2, 1)),
    (pins.test_fig3_full_conversion_roundtrip, ()),
    (pins.test_greedy_matches_exhaustive_search, ()),
    (pins.test_greedy_matches_min_feasible_chunk, (32,)),
    (pins.test_grouping_predicate_random, ()),
    (pins.test_encoding_invariants_laplacian_config, ()),
    (pins.test_encoding_invariants_random, (3, 1)),
    (pins.test_encoding_invariants_random, (5, 2)),
    (pins.test_encoding_invariants_random, (7, 4)),
    (pins.test_sliced_ellpack_special_case, (32,)),
    (pins.test_identity_and_diagonal_exact, ()),
    (pins.test_laplacian_row_sums, ((64, 64),)),
    (pins.test_dense_brute_force, (4,)),
    (pins.test_dense_brute_force, (9,)),
    (pins.test_empty_matrix, ()),
]


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutant {name}: pattern not found exactly once"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", str(lib), str(path)])
    return str(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    caught = []
    with oracle.using_library(lib):
        for fn, args in PINS:
            try:
                fn(*args)
            except (AssertionError, oracle.OracleError, IndexError, ValueError):
                caught.append(fn.__name__)
    assert caught, f"no pin fails for mutant {name}"


def test_unmutated_copy_passes_every_pin(tmp_path):
    lib = _build_mutant(tmp_path, "identity", "#define ORACLE_MAX_G 1024", "#define ORACLE_MAX_G 1024")
    with oracle.using_library(lib):
        for fn, args in PINS:
            fn(*args)
