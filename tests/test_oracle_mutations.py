"""CPU: the oracle's pins catch plausible mistakes.

Each case copies ``oracle/mrpt_oracle.c``, plants one mistake (a dropped
term, a wrong sign, index or comparison, swapped operands or children, a
reordered sum), compiles the copy with the oracle's own flags and runs
``tests/test_oracle_pins.py`` against it in a subprocess (``MRPT_ORACLE_LIB``
points the oracle at the copy).  The pins must fail for every mutant and
pass for the unmodified source.  Nothing here touches the CUDA library.
"""
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "mrpt_oracle.c")

# (name, text in mrpt_oracle.c, replacement); each text occurs exactly once
MUTANTS = [
    # random matrix (Algorithm 1, Sec. II-B)
    ("splitmix_increment", "(i + 1) * 0x9E3779B97F4A7C15ULL", "(i + 1) * 0x9E3779B97F4A7C17ULL"),
    ("bernoulli_inverted", "if (z < a) { /* Bernoulli(a) came up 1 */",
     "if (z >= a) { /* Bernoulli(a) came up 1 */"),
    ("normal_variance_halved", "const double g = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);",
     "const double g = sqrt(-1.0 * log(u1)) * cos(two_pi * u2);"),
    ("fixed_count_floor", "double k = ceil((double)density * (double)d * (1.0 - 1e-6));",
     "double k = floor((double)density * (double)d * (1.0 - 1e-6));"),
    # projection (Algorithms 1 and 3)
    ("projection_descending_order",
     "for (int32_t e = col_off[c]; e < col_off[c + 1]; ++e)\n        acc = fmaf(",
     "for (int32_t e = col_off[c + 1] - 1; e >= col_off[c]; --e)\n        acc = fmaf("),
    ("projection_unfused", "acc = fmaf(x[dim[e]], val[e], acc);", "acc = x[dim[e]] * val[e] + acc;"),
    ("projection_drops_last_term",
     "for (int32_t e = col_off[c]; e < col_off[c + 1]; ++e)\n        acc = fmaf(",
     "for (int32_t e = col_off[c]; e + 1 < col_off[c + 1]; ++e)\n        acc = fmaf("),
    # tree growth (Algorithm 2, Sec. II-A)
    ("median_ties_by_descending_id",
     "if (a->key > b->key) return 1;\n    return (a->id > b->id) - (a->id < b->id);",
     "if (a->key > b->key) return 1;\n    return (a->id < b->id) - (a->id > b->id);"),
    ("split_is_upper_median", "g->split[node] = g->scratch[nl - 1].key;",
     "g->split[node] = g->scratch[nl < c ? nl : nl - 1].key;"),
    ("left_takes_floor_half", "const int32_t nl = (c + 1) / 2;", "const int32_t nl = c > 1 ? c / 2 : 1;"),
    ("children_swapped",
     "grow(g, idx, nl, level + 1, 2 * node + 1);\n    grow(g, idx + nl, c - nl, level + 1, 2 * node + 2);",
     "grow(g, idx, nl, level + 1, 2 * node + 2);\n    grow(g, idx + nl, c - nl, level + 1, 2 * node + 1);"),
    ("leaf_ids_unsorted", "qsort(idx, (size_t)c, sizeof(int32_t), cmp_i32);\n        g->leaf_off",
     "g->leaf_off"),
    # routing (Algorithm 3)
    ("route_strict_less", "node = (p[level] <= split[node]) ?", "node = (p[level] < split[node]) ?"),
    ("route_children_swapped", "? 2 * node + 1 : 2 * node + 2;", "? 2 * node + 2 : 2 * node + 1;"),
    ("route_reads_levels_reversed", "node = (p[level] <= split[node]) ?",
     "node = (p[l - 1 - level] <= split[node]) ?"),
    # votes (Algorithm 4, Sec. III-A)
    ("vote_threshold_off_by_one", "if (votes[point] == v) {", "if (votes[point] == v + 1) {"),
    # exact search (Sec. I-A, knn of Algorithm 4)
    ("distance_drops_first_dim",
     "for (int32_t i = 0; i < d; ++i) {\n            const double diff",
     "for (int32_t i = 1; i < d; ++i) {\n            const double diff"),
    ("distance_sign", "const double diff = (double)q[i] - (double)x[i];",
     "const double diff = (double)q[i] + (double)x[i];"),
    ("knn_ties_by_descending_id",
     "if (a->dist > b->dist) return 1;\n    return (a->id > b->id) - (a->id < b->id);",
     "if (a->dist > b->dist) return 1;\n    return (a->id < b->id) - (a->id > b->id);"),
    ("no_square_root", "out_dists[r] = (mode == 0) ? (float)sqrt(buf[r].dist) :",
     "out_dists[r] = (mode == 0) ? (float)buf[r].dist :"),
    ("padding_id_zero", "out_ids[r] = -1;\n            out_dists[r] = INFINITY;",
     "out_ids[r] = 0;\n            out_dists[r] = INFINITY;"),
]


def _compile(text: str, out_dir: str, name: str) -> str:
    c = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, "lib" + name + ".so")
    with open(c, "w") as f:
        f.write(text)
    subprocess.run(["gcc", *oracle.CFLAGS, c, "-o", so, "-lm"], check=True)
    return so


def _run_pins(so: str) -> subprocess.CompletedProcess:
    env = dict(os.environ, MRPT_ORACLE_LIB=so)
    return subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle_pins.py"),
                           "-x", "-q", "-p", "no:cacheprovider"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_pins_pass_on_the_unmodified_oracle(tmp_path):
    so = _compile(open(SRC).read(), str(tmp_path), "original")
    r = _run_pins(so)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site of {name} not found exactly once"
    so = _compile(src.replace(old, new), str(tmp_path), name)
    r = _run_pins(so)
    # exit code 1: tests ran and at least one pin failed
    assert r.returncode == 1, f"{name} survived the pins:\n" + r.stdout[-2000:] + r.stderr[-2000:]
