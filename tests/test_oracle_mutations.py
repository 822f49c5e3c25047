"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a temporary copy of oracle/csaw_ref.c (CPU
only), builds it, and runs the pin suite against that build: the suite must
fail.  The real oracle file is never modified.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "csaw_ref.c")

MUTATIONS = {
    # interval convention: lower instead of upper bound (Eq. 1 intervals)
    "lower_bound": ("if (S[mid] > x) hi = mid;", "if (S[mid] >= x) hi = mid;"),
    # draw layout
    "swap_r64_words": ("return ((uint64_t)out[1] << 32) | (uint64_t)out[0];",
                       "return ((uint64_t)out[0] << 32) | (uint64_t)out[1];"),
    "counter_order": ("uint32_t ctr[4] = { attempt, vertex, layer, instance };",
                      "uint32_t ctr[4] = { vertex, attempt, layer, instance };"),
    "philox_constant": ("k1 += 0xBB67AE85u;", "k1 += 0xBB67AE84u;"),
    # node2vec multipliers on the wrong case
    "n2v_prev_mult": ("else if (u == prev) val = (uint64_t)w * mult[0];",
                      "else if (u == prev) val = (uint64_t)w * mult[1];"),
    "n2v_adjacent_mult": ("else if (is_neighbour(g, prev, u)) val = (uint64_t)w * mult[1];",
                          "else if (is_neighbour(g, prev, u)) val = (uint64_t)w * mult[2];"),
    "walk_prev_not_updated": ("prev = cur;\n            cur = col[off[cur] + j];",
                              "cur = col[off[cur] + j];"),
    # neighbour degree taken from the wrong endpoint
    "degree_of_source": ("case REF_BIAS_NEIGHBOR_DEGREE: val = g->off[u + 1] - g->off[u]; break;",
                         "case REF_BIAS_NEIGHBOR_DEGREE: val = g->off[v + 1] - g->off[v]; break;"),
    # selection without replacement
    "no_take_all": ("if (k == REF_FANOUT_ALL || npos <= k) {", "if (k == REF_FANOUT_ALL) {"),
    "duplicates_kept": ("if (!chosen[i]) { chosen[i] = 1; out_idx[have++] = i; }",
                        "{ chosen[i] = 1; out_idx[have++] = i; }"),
    "updated_sampling_total": ("uint32_t i = upper_bound_u64(S2, d, ref_scale(r, run2));",
                               "uint32_t i = upper_bound_u64(S2, d, ref_scale(r, T) % run2);"),
    # Update: visited filter dropped
    "no_visited_filter": ("if (!in_sorted(visited, nvis, cand[j])) cand[nn++] = cand[j];",
                          "cand[nn++] = cand[j];"),
    # multi-dimensional random walk: VertexBias not the degree, Update
    # dropped, neighbour draw keyed by the slot instead of the vertex
    "mdrw_vertex_bias_uniform": ("run += v < V ? off[v + 1] - off[v] : 0;", "run += v < V ? 1 : 0;"),
    "mdrw_no_update": ("            pool[slot] = u;\n", ""),
    "mdrw_neighbour_key": ("uint64_t y = ref_scale(ref_draw(seed, 0, v, s, inst), d);",
                           "uint64_t y = ref_scale(ref_draw(seed, 0, slot, s, inst), d);"),
    # walks with restart / jump: restart to the wrong vertex, dead ends that
    # stop, a jump range one short
    "restart_to_current": ("if (tele == REF_TELE_RESTART) return start;", "if (tele == REF_TELE_RESTART) return cur;"),
    "teleport_dead_end_stops": ("if (tele == REF_TELE_NONE) break;", "break;"),
    "jump_range": ("return (uint32_t)ref_scale(ref_draw(seed, 2, cur, s, inst), V);",
                   "return (uint32_t)ref_scale(ref_draw(seed, 2, cur, s, inst), V - 1);"),
    # layer sampling: pool entries mapped to the wrong frontier vertex, pool
    # biases that ignore the kind
    "layer_pool_mapping": ("if (start[mid] <= idx[j]) lo = mid; else hi = mid;",
                           "if (start[mid] < idx[j]) lo = mid; else hi = mid;"),
    "layer_pool_unbiased": ("rc = edge_biases(g, F[fi], kind, mult, REF_NONE, b + pos);",
                            "rc = edge_biases(g, F[fi], REF_BIAS_UNIFORM, mult, REF_NONE, b + pos);"),
    # walk key ignores the step
    "walk_key_step": ("uint64_t x = ref_scale(ref_draw(seed, 0, cur, s, inst), run);",
                      "uint64_t x = ref_scale(ref_draw(seed, 0, cur, 0, inst), run);"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name):
    before, after = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, f"mutation site for {name} not found once"
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "mut.c")
        so = os.path.join(td, "libmut.so")
        open(c, "w").write(src.replace(before, after))
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", so, c])
        env = dict(os.environ, CSAW_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                            "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                           capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} not caught:\n{r.stdout[-2000:]}"
