"""Each plausible mistake planted in a copy of the oracle must fail the pins.

The mutants are compiled from text edits of bbtc_oracle.c into a temporary
directory; the oracle in the repository is never modified.
"""
import os
import subprocess
import sys

import pytest

import oracle
from tests import pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "bbtc_oracle.c")

MUTANTS = {
    # Alg. 1 exactly as printed (first comparison A[b] = B[b])
    "alg1_printed_typo": ("if (A[a] == B[b]) { ++c; ++a; ++b; }",
                          "if (A[b] == B[b]) { ++c; ++a; ++b; }"),
    "self_loops_kept": ("if (v == u) continue;", ""),
    "duplicates_kept": ("if (i == 0 || keys_out[i] != keys_out[i - 1])", "if (1)"),
    "degree_order_reversed": ("g_sort_deg[a] < g_sort_deg[b] ? -1 : 1",
                              "g_sort_deg[a] > g_sort_deg[b] ? -1 : 1"),
    "orientation_reversed": ("ok[e] = ra < rb ? (ra << 32) | rb : (rb << 32) | ra;",
                             "ok[e] = ra > rb ? (ra << 32) | rb : (rb << 32) | ra;"),
    "cuts_off_by_one": ("while (r < n && rp[r] < target) ++r;",
                        "while (r < n && rp[r] <= target) ++r;"),
    "alg5_wrong_partial_list": ("    partial_list(rp, ci, u, k, cuts, &ik_lo, &ik_hi);\n    for (int64_t e = ij_lo;",
                                "    partial_list(rp, ci, u, j, cuts, &ik_lo, &ik_hi);\n    for (int64_t e = ij_lo;"),
    "alg6_h_starts_at_zero": ("for (int64_t x = 0; x < vk; ++x) H[x] = -1;",
                              "for (int64_t x = 0; x < vk; ++x) H[x] = 0;"),
    "alg6_probe_wrong_block": ("if (H[ci[f] - cuts[k]] == u) ++tau;",
                               "if (H[ci[f] - cuts[k]] == u && ci[f] != cuts[k]) ++tau;"),
    "per_vertex_wrong_corner": ("cnt_out[perm[u]] += 1; cnt_out[perm[v]] += 1;",
                                "cnt_out[perm[u]] += 1; cnt_out[perm[u]] += 1;"),
    "edge_support_drops_vw": ("sup_out[e] += 1; sup_out[a] += 1; sup_out[b] += 1;",
                              "sup_out[e] += 1; sup_out[a] += 1; sup_out[a] += 1;"),
    "edge_support_wrong_edge": ("sup_out[e] += 1; sup_out[a] += 1; sup_out[b] += 1;",
                                "sup_out[e] += 1; sup_out[a] += 1; sup_out[b - 1 >= rp[v] ? b - 1 : b] += 1;"),
    "exec_time_min_not_max": ("(dik > djk ? dik : djk)", "(dik < djk ? dik : djk)"),
    "task_order_ascending": ("g_sort_est[a] > g_sort_est[b] ? -1 : 1",
                             "g_sort_est[a] < g_sort_est[b] ? -1 : 1"),
    "task_count_formula": ("return (int64_t)p * (p + 1) * (p + 2) / 6;",
                           "return (int64_t)p * (p + 1) * (p + 1) / 6;"),
    "pbd_weight_out_degree_only": ("    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) w[ci[e]] += 1;\n", ""),
    "pbd_load_sign": ("return S[r1 * W + c1] - S[r0 * W + c1] - S[r1 * W + c0] + S[r0 * W + c0];",
                      "return S[r1 * W + c1] - S[r0 * W + c1] - S[r1 * W + c0] - S[r0 * W + c0];"),
    "pbd_ignores_column_blocks": ("for (int32_t k = 0; ok && k < i; ++k)",
                                  "for (int32_t k = 0; ok && k < 0; ++k)"),
    "pbd_probe_not_greedy": ("      best = t;\n    }", "      best = t;\n      break;\n    }"),
    "pbd_bisection_keeps_lo": ("if (orc_pbd_probe(G, S, p, mid, x)) hi = mid; else lo = mid;",
                               "if (orc_pbd_probe(G, S, p, mid, x)) lo = mid; else hi = mid;"),
    # |G_ij| stored at (j, i): the largest block is unchanged, the matrix is not
    "block_nnz_transposed": ("nnz[(int64_t)i * p + part_of(ci[e], p, cuts)] += 1;",
                             "nnz[(int64_t)part_of(ci[e], p, cuts) * p + i] += 1;"),
    # a position after an empty part is given to that empty part
    "part_of_stops_at_empty_part": ("while (i + 1 < p && cuts[i + 1] <= r) ++i;",
                                    "while (i + 1 < p && cuts[i + 1] <= r && cuts[i + 1] > cuts[i]) ++i;"),
    "wmerge_counts_v_twice": ("mg += du + dv;", "mg += dv + dv;"),
    "classify_drops_w_part": ("per_task[idx[((int64_t)bu * p + bv) * p + part_of(ci[a], p, cuts)]] += 1;",
                              "per_task[idx[((int64_t)bu * p + bv) * p + bv]] += 1;"),
}


def _build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    return oracle.compile_source(str(path), str(tmp_path / f"lib{name}.so"))


def test_unmodified_oracle_passes():
    assert pins.pin_battery() == []


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RUN = """
import sys
sys.path.insert(0, {root!r})
import oracle
from tests import pins
with oracle.using_library({lib!r}):
    fails = pins.pin_battery()
print("FAILS", len(fails))
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    # A mutant may also corrupt memory (e.g. a wrong task count sizes arrays
    # too small), so each runs in its own process; a crash counts as caught.
    lib = _build_mutant(tmp_path, name)
    proc = subprocess.run([sys.executable, "-c", _RUN.format(root=ROOT, lib=lib)],
                          capture_output=True, text=True, timeout=600)
    caught = proc.returncode != 0 or "FAILS 0" not in proc.stdout
    assert caught, f"mutant {name} passed every pin"
