"""Plant plausible mistakes in copies of the oracle and check the pins
catch every one.

Each mutant is one textual change to ``oracle/sivf_oracle.c`` (a dropped
coordinate, a wrong sign, ties sent to the wrong index, a top-k off by one,
first- instead of last-occurrence-wins, an overwrite that forgets the old
copy, a slab never returned, rounding by truncation, ties away from even,
compaction slots, the last slab's fill, budget or threshold off by one, a
row stride in the distance helper, and in the reduced-precision approximate
distance: a scale not undone, a residual from the wrong centroid, the
query norm taken from rounded values, the query scale off by two).
The mutant is compiled into a temporary library, swapped in for the real
oracle, and the pin tests of ``test_oracle_pins.py`` are run against it: at
least one must fail.  The real oracle source is never modified.
"""
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

MUTANTS = {
    "drop_last_coordinate": ("double acc = 0.0;\n    for (int j = 0; j < d; ++j) {",
                             "double acc = 0.0;\n    for (int j = 0; j < d - 1; ++j) {"),
    "wrong_sign": ("double t = (double)a[j] - (double)b[j];",
                   "double t = (double)a[j] + (double)b[j];"),
    "ties_to_highest_centroid": ("if (dc < bd) {", "if (dc <= bd) {"),
    "topk_ties_to_higher_id": ("if (x->key < y->key) return -1;\n    if (x->key > y->key) return 1;",
                               "if (x->key > y->key) return -1;\n    if (x->key < y->key) return 1;"),
    "topk_off_by_one": ("if (j < m) {", "if (j + 1 < m) {"),
    "first_occurrence_wins": ("for (int64_t i = 0; i < n; ++i) last[ids[i]] = i;",
                              "for (int64_t i = n - 1; i >= 0; --i) last[ids[i]] = i;"),
    "overwrite_keeps_old_copy": ("if (win[i] && o->where[ids[i]] >= 0) erase(o, ids[i]);",
                                 ";"),
    "slab_never_returned": ("o->free_slabs += 1;", ";"),
    "compact_slots_reversed": ("L->slot[j] = (int32_t)(j % o->C);",
                               "L->slot[j] = (int32_t)(o->C - 1 - j % o->C);"),
    "compact_last_slab_full": ("R->fill = (int32_t)(f < o->C ? f : o->C);",
                               "R->fill = (int32_t)o->C;"),
    "compact_budget_exclusive": ("if (moved + L->n > max_moves) break;",
                                 "if (moved + L->n >= max_moves) break;"),
    "compact_min_free_off_by_one": ("if (L->nrec - keep < min_free) continue;",
                                    "if (L->nrec - keep <= min_free) continue;"),
    "bf16_truncates": ("if (lower > 0x8000u || (lower == 0x8000u && (upper & 1u))) upper += 1;",
                       ";"),
    "e4m3_ties_up": ("if (dd < bd || (dd == bd && (c & 1) == 0 && (best & 1) == 1)) {",
                     "if (dd <= bd) {"),
    "dists_row_stride": ("out[i] = sqdist(q, x + (size_t)i * d, d);",
                         "out[i] = sqdist(q, x + (size_t)i, d);"),
    "approx_scale_not_undone": ("s = 1.0 / ((double)inv_l[i] * (double)tq);",
                                "s = (double)inv_l[i] * (double)tq;"),
    "approx_residual_wrong_centroid": ("const float y = xi[j] - c[j];",
                                       "const float y = xi[j] - cent[j];"),
    "approx_bf16_norm_of_rounded_query": ("qn += (double)q[j] * (double)q[j];",
                                          "qn += (double)bf16_round(q[j]) * (double)bf16_round(q[j]);"),
    "approx_query_scale_from_max": ("448.0f / (2.0f * mx)", "448.0f / mx"),
}

PINS = [
    (pins.test_assign_matches_exact_rational_argmin, dict(d=2, denom=1)),
    (pins.test_assign_general_floats_exact_rational, {}),
    (pins.test_probe_matches_exact_rational_order, dict(P=3)),
    (pins.test_full_probe_equals_brute_force, dict(integer=True)),
    (pins.test_partial_probe_equals_brute_force_over_probed_lists, {}),
    (pins.test_pad_when_fewer_than_k, {}),
    (pins.test_ties_in_topk_go_to_lower_id, {}),
    (pins.test_golden_tiny_1d, {}),
    (pins.test_random_ops_match_set_model_and_invariants, {}),
    (pins.test_duplicate_in_batch_last_wins, {}),
    (pins.test_overwrite_is_delete_then_insert, {}),
    (pins.test_remove_idempotent_and_absent_ids, {}),
    (pins.test_delete_all_returns_every_slab, {}),
    (pins.test_sliding_window_frees_oldest_slab, {}),
    (pins.test_bf16_matches_torch_rne, {}),
    (pins.test_e4m3_matches_torch_in_range_and_saturates, {}),
    (pins.test_compact_worked_example, {}),
    (pins.test_compact_min_free_and_budget_rules, {}),
    (pins.test_compact_keeps_search_and_members, {}),
    (pins.test_dists_equal_exact_rational_sums, dict(n=17, d=8, denom=4)),
    (pins.test_dists_hand_value, {}),
    (pins.test_approx_bf16_exact_inputs_equal_the_distance, {}),
    (pins.test_approx_bf16_hand_value, {}),
    (pins.test_approx_fp8_exact_codes_equal_the_distance, dict(t_l=4.0, qmax=112.0)),
    (pins.test_approx_fp8_rounding_against_torch_codes, {}),
]


def _compile(src: str, tmp_path) -> str:
    c = tmp_path / "mutant.c"
    so = tmp_path / "mutant.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared",
                    "-ffp-contract=off", "-o", str(so), str(c), "-lm"],
                   check=True)
    return str(so)


def test_unmutated_copy_passes_all_pins(tmp_path, monkeypatch):
    src = open(oracle._SRC).read()
    monkeypatch.setattr(oracle, "_lib", oracle.load_lib(_compile(src, tmp_path)))
    for fn, kw in PINS:
        fn(**kw)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site of {name} not unique"
    lib = oracle.load_lib(_compile(src.replace(old, new), tmp_path))
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = []
    for fn, kw in PINS:
        try:
            fn(**kw)
        except Exception as e:  # AssertionError or an oracle error
            caught.append((fn.__name__, type(e).__name__))
    assert caught, f"mutant {name} passed every pin"
