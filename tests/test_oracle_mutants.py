"""Planted mistakes in the oracle are caught by its pins (no GPU).

Each case copies ``oracle/oracle.c``, changes one plausible detail (a dropped
term, a flipped comparison, a wrong index), compiles the copy on the CPU and
checks that at least one pin in ``tests/pins.py`` fails against it.
"""
import json
import os
import subprocess
import sys

import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text, planted text): the original must occur exactly once.
MUTANTS = [
    ("parent_max", "(best == -1 || u < best)", "(best == -1 || u > best)"),
    ("parent_any_level", "if (depth[u] == depth[v] - 1 && (best", "if (depth[u] >= 0 && (best"),
    ("no_dedup", "if (i > b && raw[i] == raw[i - 1]) continue;", ""),
    ("keep_self_loops", ["    if (u == v) continue;\n    bucket[cnt[v]++] = u;", "    if (u == v) continue;\n    cnt[u] += 1;"],
     ["    bucket[cnt[v]++] = u;", "    cnt[u] += 1;"]),
    ("one_direction", "    bucket[cnt[u]++] = v; /* entry v->u */", "    bucket[cnt[u]++] = u; /* entry v->u */"),
    ("rows_unsorted", "  for (int32_t v = 0; v < n; ++v)\n    for (int64_t i = start[v];", "  for (int32_t v = n - 1; v >= 0; --v)\n    for (int64_t i = start[v];"),
    ("depth_plus_two", "depth[v] = depth[u] + 1;", "depth[v] = depth[u] + 2;"),
    ("lifo_queue", "int32_t u = queue[head++];", "int32_t u = queue[--tail];"),
    ("source_parent", "if (v == s) { parent[v] = s; continue; }", "if (v == s) { parent[v] = -1; continue; }"),
    ("delegate_ge", "if (g->off[v + 1] - g->off[v] > th) internal_of[v] = next++;",
     "if (g->off[v + 1] - g->off[v] >= th) internal_of[v] = next++;"),
    ("normal_descending", "for (int32_t v = 0; v < n; ++v) { /* class 1",
     "for (int32_t v = n - 1; v >= 0; --v) { /* class 1"),
    ("component_not_halved", "return ends / 2;", "return ends;"),
    ("u8_unreached_zero", "(uint8_t)(dv < 0 ? 255", "(uint8_t)(dv < 0 ? 0"),
    ("u8_no_overflow", "if (dv > 254) overflow = 1;", ""),
    ("validator_no_canonical", "if (u < p && depth[u] == depth[v] - 1) return 6;", ""),
    ("validator_no_cut", "if ((depth[u] >= 0) != (depth[v] >= 0)) return 2;", ""),
    ("validator_no_parent_depth", "if (depth[p] != depth[v] - 1) return 5;", ""),
    ("validator_union_find_never_unites", "if (a != b) uf[a] = b;", ""),
    ("first_hit_counts_from_zero", "o[5] += first_hit(g, depth, v, L);", "o[5] += first_hit(g, depth, v, L) - 1;"),
    ("subgraph_source_only", "counts[(u_del << 1) | v_del] += 1;", "counts[(u_del << 1) | u_del] += 1;"),
    ("paper_bv_swapped", "bv = sd * (qd + sd) / qd;", "bv = qd * (qd + sd) / sd;"),
    ("paper_back_flipped", "!(fvd < factor1 * bv)", "!(fvd > factor1 * bv)"),
    ("beamer_no_shrink_test", "q[L] * beta < (int64_t)g->n && q[L] < q_prev", "q[L] * beta < (int64_t)g->n"),
    ("beamer_mu_all_edges", "m_u = m_total - seen_m;", "m_u = m_total;"),
    ("stay_guard_dropped", "if (rule == ORC_RULE_BEAMER_STAY && fv[L] * alpha > m_u) next = 1;", ""),
    ("stay_guard_ge", "if (rule == ORC_RULE_BEAMER_STAY && fv[L] * alpha > m_u) next = 1;",
     "if (rule == ORC_RULE_BEAMER_STAY && fv[L] * alpha >= m_u) next = 1;"),
    ("directions_seen_after", "    seen_v += q[L];\n    seen_m += fv[L];\n", ""),
    ("subgraph_U_from_source_class", "if (unvisited && in_x > 0) U += 1;", "if (unvisited && out_x > 0) U += 1;"),
    ("subgraph_q_unfiltered", "if (depth[v] == L && out_x > 0) {", "if (depth[v] == L && is_del == src_del[x]) {"),
    ("subgraph_s_counts_visited", "if (unvisited && out_x > 0) su += 1;", "if (out_x > 0) su += 1;"),
    ("subgraph_dn_nd_swapped", "const int src_del[3] = {1, 1, 0}, dst_del[3] = {1, 0, 1};",
     "const int src_del[3] = {1, 0, 1}, dst_del[3] = {1, 1, 0};"),
    ("subgraph_factor_of_dd_for_all", "(fvd > factor0[x] * bv)", "(fvd > factor0[0] * bv)"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    text = open(SRC).read()
    olds = old if isinstance(old, list) else [old]
    news = new if isinstance(new, list) else [new]
    for o, n in zip(olds, news):
        assert text.count(o) == 1, "mutation anchor for %s not unique" % name
        text = text.replace(o, n)
    src = tmp_path / ("oracle_%s.c" % name)
    src.write_text(text)
    so = tmp_path / ("liboracle_%s.so" % name)
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-I", os.path.dirname(SRC),
                    "-o", str(so), str(src)], check=True)
    # run the pins in a child process: a planted mistake may also crash the library
    code = ("import json, oracle; from tests import pins; "
            "print(json.dumps(pins.run_all(oracle.load(%r))))" % str(so))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return  # the broken oracle crashed: caught
    failed = json.loads(r.stdout.strip().splitlines()[-1])
    assert failed, "planted mistake %s passed every pin" % name
