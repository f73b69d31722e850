"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle source (a dropped term,
a flipped sign, a wrong index, a reversed tie-break ...), compiles it on the
CPU, and runs the pin tests against it: at least one pin must fail.
Mutations that cannot change any result are left out: every batch edge is
stored in both directions, so e.g. marking the target instead of the source
of an arc, or charging the other endpoint's community, is equivalent.
"""
import functools
import os
import types

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "dfl_oracle.cpp")

MUTANTS = {
    "stay_drops_own_weight": ("i128(Sigma_d - Ki)", "i128(Sigma_d)"),
    "score_sign": ("i128(m2) * i128(Hc) - i128(Ki) * i128(Sigma_c)",
                   "i128(m2) * i128(Hc) + i128(Ki) * i128(Sigma_c)"),
    "tie_break_largest": ("(s == best_score && c < best)", "(s == best_score && c > best)"),
    "move_on_equal_gain": ("if (!(best_score > stay)) continue;", "if (best_score < stay) continue;"),
    "self_loop_in_local_move": ("scan_communities(H, Gp, Cold, i, false);",
                                "scan_communities(H, Gp, Cold, i, true);"),
    "aggregate_without_self": ("scan_communities(H, Gp, Cp, i, true);",
                               "scan_communities(H, Gp, Cp, i, false);"),
    "weights_index_by_vertex": ("o.Sigma[o.C[a]] -= int64_t(weff);",
                                "o.Sigma[a] -= int64_t(weff);"),
    "insert_weights_drop_k": ("o.K[a] += int64_t(w);", "o.K[a] += int64_t(w) - 1;"),
    "df_deletion_rule_flipped": ("if (o.C[e.i] == o.C[e.j]) F[e.i] = 1;",
                                 "if (o.C[e.i] != o.C[e.j]) F[e.i] = 1;"),
    "df_insertion_rule_flipped": ("if (o.C[e.i] != o.C[e.j]) F[e.i] = 1;",
                                  "if (o.C[e.i] == o.C[e.j]) F[e.i] = 1;"),
    "modularity_sigma_not_squared": ("s2 += i128(Sig[c]) * i128(Sig[c]);", "s2 += i128(Sig[c]);"),
    "no_singleton_guard": ("sizeold[d] == 1 && sizeold[best] == 1 && best > d",
                           "sizeold[d] == 1 && sizeold[best] == 1 && best > d && false"),
    "frontier_keeps_mover": ("if (a.j != mv.i && R[a.j]) Fnext[a.j] = 1;",
                             "if (R[a.j]) Fnext[a.j] = 1;"),
    "tolerance_off_by_two": ("u128 den = u128(2) * u128(o.tau_den);", "u128 den = u128(o.tau_den);"),
    "ds_scores_with_stale_k": ("i128 s = score_of(o.m2, kv.second, o.K[i], o.Sigma[kv.first]);",
                               "i128 s = score_of(o.m2, kv.second, o.K[kv.first], o.Sigma[kv.first]);"),
    "self_loop_counts_twice_in_k": ("for (const Arc& a : G[i]) K[i] += int64_t(a.w);",
                                    "for (const Arc& a : G[i]) K[i] += int64_t(a.w) * (a.j == i ? 2 : 1);"),
    "ds_no_neighbour_expansion": ("for (const Arc& a : o.G[i]) dV[a.j] = 1;",
                                  "for (const Arc& a : o.G[i]) (void)a;"),
    "ds_no_community_expansion": ("if (dC[o.C[i]]) dV[i] = 1;", "if (false && dC[o.C[i]]) dV[i] = 1;"),
    "aggregation_test_flipped": ("if (double(ncomm) / double(nv) > o.opt.tau_agg) break;",
                                 "if (double(ncomm) / double(nv) < o.opt.tau_agg) break;"),
    "no_tolerance_drop": ("den *= u128(o.tolerance_drop);", "den *= u128(1);"),
    "frontier_dropped_between_iterations": ("F.swap(Fnext);", "F.assign(nv, 0);"),
    "trace_counts_movers_as_processed": ("o.trace.push_back({processed, moved, dq_sum});",
                                         "o.trace.push_back({moved, moved, dq_sum});"),
    "sizes_not_carried": ("sizep[mv.d] -= 1;", "sizep[mv.d] -= 0;"),
    "final_lookup_skips_last_pass": ("for (uint32_t i = 0; i < n; ++i) Ct[i] = Cp[Ctop[i]];",
                                     "for (uint32_t i = 0; i < n; ++i) Ct[i] = Ctop[i];"),
    "later_pass_frontier_empty": ("F.assign(ncomm, 1);", "F.assign(ncomm, 0);"),
    "sigma_not_reset_after_aggregation": ("Sp = Kp;", "Sp.resize(ncomm);"),
}

PIN_TESTS = [
    (pins.test_modularity_equals_newman_all_pairs, {"seed": 1}),
    (pins.test_modularity_special_cases, {}),
    (pins.test_delta_modularity_matches_q_difference, {"seed": 2, "loops": True}),
    (pins.test_move_iteration_matches_brute_force, {"seed": 0, "k": 1, "kind": "weighted"}),
    (pins.test_move_iteration_matches_brute_force, {"seed": 1, "k": 4, "kind": "unit"}),
    (pins.test_move_iteration_matches_brute_force, {"seed": 3, "k": 4, "kind": "loops"}),
    (pins.test_move_iteration_matches_brute_force, {"seed": 4, "k": 1, "kind": "loops"}),
    (pins.test_tie_break_smallest_community, {}),
    (pins.test_singleton_swap_guard, {}),
    (pins.test_incremental_weights_equal_recomputation, {"mode": 2}),
    (pins.test_aggregation_preserves_weight_and_modularity, {"seed": 0, "loops": True}),
    (pins.test_dynamic_frontier_marking_rules, {}),
    (pins.test_delta_screening_best_community, {}),
    (pins.test_delta_screening_choice_is_best_delta_modularity, {"intra": 1}),
    (pins.test_delta_screening_choice_is_best_delta_modularity, {"intra": 6}),
    (pins.test_figure3_initial_frontier, {}),
    (pins.test_iteration_tolerance_is_exact, {}),
    (pins.test_static_equals_nd_from_singletons, {}),
    (pins.test_aggregation_tolerance_rule, {}),
    (pins.test_tolerance_drops_per_pass, {}),
    (pins.test_first_pass_replays_as_single_iterations,
     {"mode": "static", "n": 1500, "blocks": 15, "mu": 0.3, "size": 0, "several": True}),
    (pins.test_first_pass_replays_as_single_iterations,
     {"mode": 2, "n": 1500, "blocks": 15, "mu": 0.3, "size": 1500, "several": True}),
    (pins.test_later_passes_are_louvain_on_the_aggregated_graph, {"case": "static"}),
]


def variant(lib_path):
    ns = types.SimpleNamespace()
    ns.Oracle = functools.partial(oracle.Oracle, library=lib_path)
    ns.OracleError = oracle.OracleError
    return ns


def pins_failing(mod):
    failed = []
    for fn, kw in PIN_TESTS:
        try:
            fn(mod, **kw)
        except pytest.skip.Exception:
            pass
        except Exception:
            failed.append(fn.__name__)
    return failed


def test_unmutated_oracle_passes_the_selected_pins():
    assert pins_failing(variant(None)) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old}"
    path = tmp_path / f"{name}.cpp"
    path.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(path), str(tmp_path / f"lib{name}.so"))
    assert pins_failing(variant(lib)), f"no pin caught mutant {name}"
