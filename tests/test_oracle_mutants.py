"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check
that the pins catch every one of them: a dropped term, a wrong index or
offset, a transposed operand, a skipped supply step, a wrong shift."""
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))

# (name, exact text in pm_oracle.c, replacement)
MUTANTS = [
    ("brute_var_drops_last_window", "if (len < 1 || i + len > n) continue;", "if (len < 1 || i + len >= n) continue;"),
    ("brute_var_index_i_not_i_plus_k", "while (k < len && q[k] == T[i + k]) k++;", "while (k < len && q[k] == T[i]) k++;"),
    ("dict_var_lower_bound_skips_equal", "(size_t)L) >= 0) b = h;", "(size_t)L) > 0) b = h;"),
    ("dict_var_ids_descending", "while (y > 0 && jb->found[y - 1] > v)", "while (y > 0 && jb->found[y - 1] < v)"),
    ("dict_var_one_length_group", "if (ng == 0 || glen[ng - 1] != L) {", "if (ng == 0) {"),
    ("brute_drops_last_window", "for (int64_t i = 0; i < n - m + 1; i++) {\n        for (int64_t r = 0; r < d; r++) {",
     "for (int64_t i = 0; i < n - m; i++) {\n        for (int64_t r = 0; r < d; r++) {"),
    ("brute_reversed_pattern", "if (T[i + j] != p[j])", "if (T[i + j] != p[m - 1 - j])"),
    ("brute_index_i_not_i_plus_j", "if (T[i + j] != p[j])", "if (T[i] != p[j])"),
    ("dict_lower_bound_skips_equal", "(size_t)m) < 0) lo = mid + 1;", "(size_t)m) <= 0) lo = mid + 1;"),
    ("dict_worker_gap", "jobs[t].i0 = nwin * t / nthreads;", "jobs[t].i0 = nwin * t / nthreads + (t > 0);"),
    ("ac_restart_at_root", "while ((ns = a->g[(int64_t)state * ORC_SIGMA + T[i]]) == ORC_FAIL)\n            state = a->supply[state];",
     "while ((ns = a->g[(int64_t)state * ORC_SIGMA + T[i]]) == ORC_FAIL)\n            state = 0;"),
    ("ac_supply_one_level_short", "a->supply[s] = a->g[(int64_t)st * ORC_SIGMA + c];", "a->supply[s] = st;"),
    ("ac_report_offset", "occ[total] = ORC_OCC(i - a->m + 1, r);", "occ[total] = ORC_OCC(i - a->m, r);"),
    ("ac_goto_wrong_char", "a->g[(int64_t)state * ORC_SIGMA + p[l]] = q;", "a->g[(int64_t)state * ORC_SIGMA + p[j]] = q;"),
    ("ac_output_on_last_created", "if (a->out_tail[state] < 0) a->out_head[state] = i;\n        else a->out_next[a->out_tail[state]] = i;\n        a->out_tail[state] = i;",
     "if (a->out_tail[a->nstates - 1] < 0) a->out_head[a->nstates - 1] = i;\n        else a->out_next[a->out_tail[a->nstates - 1]] = i;\n        a->out_tail[a->nstates - 1] = i;"),
    ("wm_block_b_plus_one", "int64_t h = orc_wm_h(p + (q - B), B);", "int64_t h = orc_wm_h(p + (q - B - 1 >= 0 ? q - B - 1 : 0), B);"),
    ("wm_shift_init_too_big", "w->shift[h] = m - B + 1;", "w->shift[h] = m - B + 2;"),
    ("dfa_piece_without_overlap", "int64_t end = jb->i1 + m - 1;", "int64_t end = jb->i1;"),
    ("dfa_goto_without_supply", "? dfa[(int64_t)a->supply[q] * ncls + c] : t;", "? 0 : t;"),
    ("dfa_start_off_by_one", "jb->buf[jb->len++] = ORC_OCC(e - m + 1, r);", "jb->buf[jb->len++] = ORC_OCC(e - m, r);"),
    ("wm_overshift", "i += w->shift[h];", "i += w->shift[h] + 1;"),
    ("wm_prefix_wrong_window", "int64_t hp = orc_wm_h(T + (i - m + 1), Bp);", "int64_t hp = orc_wm_h(T + (i - m + 2 <= i ? i - m + 2 : i), Bp);"),
    ("wm_hash_bitshift_3", "for (int32_t k = 0; k < len; k++) h = (h << 2) + s[k];", "for (int32_t k = 0; k < len; k++) h = (h << 3) + s[k];"),
    ("wm_text_block_off_by_one", "int64_t h = orc_wm_h(T + (i - B + 1), B);", "int64_t h = orc_wm_h(T + (i - B + 1 > 0 ? i - B : 0), B);"),
    ("wm_counts_dropped", "                    total++;\n                    counts[r]++;\n                }\n            }\n            i += 1;",
     "                    total++;\n                }\n            }\n            i += 1;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path):
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not unique/found"
    mutated = src.replace(old, new)
    oracle.compile_variant(mutated, str(tmp_path), name)
    so = os.path.join(str(tmp_path), "lib" + name + ".so")
    try:
        res = subprocess.run([sys.executable, os.path.join(HERE, "oracle_mutant_runner.py"), so],
                             capture_output=True, text=True, timeout=120)
        caught = res.returncode != 0
        detail = res.stdout[-2000:] + res.stderr[-2000:]
    except subprocess.TimeoutExpired:
        caught, detail = True, "timed out (caught)"
    assert caught, f"no pin caught the planted mistake {name}: {detail}"


def test_unmutated_oracle_passes_runner(tmp_path):
    oracle.compile_variant(oracle.source_text(), str(tmp_path), "clean")
    so = os.path.join(str(tmp_path), "libclean.so")
    res = subprocess.run([sys.executable, os.path.join(HERE, "oracle_mutant_runner.py"), so],
                         capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
