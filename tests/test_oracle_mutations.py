"""Plants one plausible mistake at a time in a copy of the oracle's C source
(a dropped term, a wrong sign or index, a transposed operand, a missed rule),
rebuilds it on the CPU and checks that the oracle's pins reject it."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = {
    "dropped_teleport_term": ("double r = (1.0 - alpha) / (double)g->n;", "double r = 0.0;"),
    "wrong_sign": ("r = r + alpha * R[u] / (double)outdeg(g, u);",
                   "r = r - alpha * R[u] / (double)outdeg(g, u);"),
    "degree_of_wrong_vertex": ("r = r + alpha * R[u] / (double)outdeg(g, u);",
                               "r = r + alpha * R[u] / (double)outdeg(g, v);"),
    "transposed_gather": ("for (int64_t e = g->in_off[v]; e < g->in_off[v + 1]; ++e) {\n"
                          "    int32_t u = g->in_idx[e];",
                          "for (int64_t e = g->out_off[v]; e < g->out_off[v + 1]; ++e) {\n"
                          "    int32_t u = g->out_idx[e];"),
    "marking_skips_deleted_targets": ("for (int64_t j = lo; j < gt->n_del && key_hi(gt->del_keys[j]) == u; ++j) {",
                                      "for (int64_t j = lo; j < lo; ++j) {"),
    "reinserted_edge_counted_as_deleted": ("    if (has_key(ik, ni, x)) continue;\n    dk[rd++] = x;",
                                           "    dk[rd++] = x;"),
    "frontier_marks_in_neighbours": ("        for (int64_t e = gt->out_off[v]; e < gt->out_off[v + 1]; ++e) VAn[gt->out_idx[e]] = 1;",
                                     "        for (int64_t e = gt->in_off[v]; e < gt->in_off[v + 1]; ++e) VAn[gt->in_idx[e]] = 1;"),
    "jacobi_reads_new_vector": ("Rn[v] = rank_of(g, R, v, alpha, D, dead_end, &s);",
                                "Rn[v] = rank_of(g, Rn, v, alpha, D, dead_end, &s);"),
    "df_bb_reads_new_vector": ("      double r = rank_of(gt, R, v, alpha, 0.0, 0, &s);",
                               "      double r = rank_of(gt, Rn, v, alpha, 0.0, 0, &s);"),
    "teleport_df_ignores_dead_end_mass_change": ("    if (alpha * fabs(D - D_last) / (double)n > tol_f) {",
                                                 "    if (0) {"),
    "teleport_df_drops_dead_end_term": ("      double r = rank_of(gt, R, v, alpha, D, 1, &s);",
                                        "      double r = rank_of(gt, R, v, alpha, 0.0, 1, &s);"),
    "df_lf_expansion_leaves_flags_clear": ("          VA[gt->out_idx[e]] = 1;\n          RC[gt->out_idx[e]] = 1;",
                                           "          VA[gt->out_idx[e]] = 1;"),
    "df_lf_initial_marking_leaves_flags_clear": ("  mark_initial(gt, VA, RC, C);",
                                                 "  mark_initial(gt, VA, NULL, C);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_reject_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation anchor not found: {name}"
    mutated = tmp_path / "oracle_mut.c"
    mutated.write_text(text.replace(old, new, 1))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                           str(mutated), "-o", str(lib), "-lm"])
    env = dict(os.environ, DFPR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins accepted mutation {name}:\n{r.stdout[-2000:]}"
