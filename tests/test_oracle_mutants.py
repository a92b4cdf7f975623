"""The oracle's pins are sensitive: each test here plants one plausible
mistake in a copy of oracle.c (a dropped term, a wrong comparison, a
transposed stride, a dropped modulo, a wrong bound, ...), compiles it, and
checks that at least one pin of test_oracle.py fails against it.  The
unmodified source passes every pin through the same harness."""
import os
import subprocess

import pytest

import oracle
import test_oracle as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# first fit (the oracle) and a best fit: the fitting mini-bucket whose union
# grows least, ties to the first
BEST_FIT_OLD = """            for (int b = 0; b < nmb && placed < 0; ++b) {
                unsigned char *u = mb_u + (size_t)b * (n + 1);
                memcpy(tmp_u, u, n + 1);
                for (int j = 0; j < f->nv; ++j) tmp_u[f->vars[j]] = 1;
                if (fits(P, mode, z, tmp_u)) {
                    memcpy(u, tmp_u, n + 1);
                    placed = b;
                }
            }"""
BEST_FIT_NEW = """            int bgrow = 1 << 30;
            for (int b = 0; b < nmb; ++b) {
                unsigned char *u = mb_u + (size_t)b * (n + 1);
                memcpy(tmp_u, u, n + 1);
                int grow = 0;
                for (int j = 0; j < f->nv; ++j) {
                    grow += !tmp_u[f->vars[j]];
                    tmp_u[f->vars[j]] = 1;
                }
                if (fits(P, mode, z, tmp_u) && grow < bgrow) {
                    bgrow = grow;
                    placed = b;
                }
            }
            if (placed >= 0)
                for (int j = 0; j < f->nv; ++j) mb_u[(size_t)placed * (n + 1) + f->vars[j]] = 1;"""

# (name, text in oracle.c, replacement)
MUTANTS = [
    ("drop a term of the bucket sum", "for (int k = 0; k < nm; ++k) s += func_eval(&fs[mbf[k]], asg);",
     "for (int k = 1; k < nm; ++k) s += func_eval(&fs[mbf[k]], asg);"),
    ("last argmin instead of first", "                    if (l == 0 || s < best) {",
     "                    if (l == 0 || s <= best) {"),
    ("first scope variable fastest", "for (int j = nv - 1; j >= 0; --j) {\n        f->stride[j] = s;",
     "for (int j = 0; j < nv; ++j) {\n        f->stride[j] = s;"),
    ("no saturation at the top cost", "if (P->saturate && s > P->top) return P->top;", "(void)P;"),
    ("Eq. 3 without its modulo", "r_in += mul * ((r_out / div) % mod);", "r_in += mul * (r_out / div);"),
    ("constant functions ignored", "bound += fs[nfs].tab[0];", "(void)0;"),
    ("separator in ascending elimination order", "for (int tt = n - 1; tt > t; --tt)",
     "for (int tt = t + 1; tt < n; ++tt)"),
    ("min-fill tie to the most neighbours", "(fill == bfill && k < bdeg)", "(fill == bfill && k > bdeg)"),
    ("mini-bucket bound off by one", "if (mode == ORC_MBE_SEP) return k - 1 <= z;",
     "if (mode == ORC_MBE_SEP) return k <= z;"),
    ("pseudo-tree children by ascending degree", "if (g_deg[x] != g_deg[y]) return g_deg[y] - g_deg[x];",
     "if (g_deg[x] != g_deg[y]) return g_deg[x] - g_deg[y];"),
    ("value phase keeps the last variable's value", "        asg[v] = bl;\n    }\n    R->cost",
     "        asg[v] = 0;\n    }\n    R->cost"),
    ("sum-product eliminates by min", "if (semiring == ORC_SUM_PRODUCT && best < INFINITY) {",
     "if (0) {"),
    ("log-sum-exp with the wrong sign", "best = best - log(acc);", "best = best + log(acc);"),
    ("log-sum-exp without the shift", "acc += exp(best - sv[l]);", "acc += exp(-sv[l]);"),
    ("free variables not counted", "bound += -log((double)P->dom[v]);", "(void)0;"),
    ("partition function without the shift", "z += exp(c0 - c);", "z += exp(-c);"),
    ("mini-buckets filled by arity ascending", "if (g_ar[x] != g_ar[y]) return g_ar[y] - g_ar[x];",
     "if (g_ar[x] != g_ar[y]) return g_ar[x] - g_ar[y];"),
    ("equal arities by creation id descending", "return g_id[x] - g_id[y];", "return g_id[y] - g_id[x];"),
    ("best fit instead of first fit", BEST_FIT_OLD, BEST_FIT_NEW),
    ("joint bound strict", "if (mode == ORC_MBE_JOINT) return k <= z;", "if (mode == ORC_MBE_JOINT) return k < z;"),
    ("log2 bound strict", "return entries <= ldexp(1.0, z);", "return entries < ldexp(1.0, z);"),
    ("value phase sums the first mini-bucket only",
     "for (int k = 0; k < nvb[v]; ++k) s += func_eval(&fs[vb[v][k]], asg);",
     "for (int k = 0; k < nvb[v]; ++k) if (vbm[v][k] == 0) s += func_eval(&fs[vb[v][k]], asg);"),
    ("value phase sums the last mini-bucket only",
     "for (int k = 0; k < nvb[v]; ++k) s += func_eval(&fs[vb[v][k]], asg);",
     "for (int k = 0; k < nvb[v]; ++k) { int last = 0; for (int q = 0; q < nvb[v]; ++q) last = vbm[v][q] > last ? "
     "vbm[v][q] : last; if (vbm[v][k] == last) s += func_eval(&fs[vb[v][k]], asg); }"),
]


def _pin_calls():
    calls = [
        ("eq3_example", lambda o: pins.test_eq3_worked_example(o)),
        ("eq3_closed_form", lambda o: pins.test_eq3_is_mixed_radix_projection(o)),
        ("bruteforce_unary", lambda o: pins.test_bruteforce_unary_closed_form(o)),
        ("eval_dense", lambda o: pins.test_eval_matches_numpy_broadcast(o)),
        ("paper_example", lambda o: pins.test_paper_example_structure(o)),
        ("saturation", lambda o: pins.test_saturation_at_top(o)),
        ("argmin_first", lambda o: pins.test_argmin_first_minimum(o)),
        ("grid_dp", lambda o: pins.test_config0_transfer_matrix(o)),
        ("minfill_small", lambda o: pins.test_minfill_small_graphs(o)),
        ("minfill_ties", lambda o: pins.test_minfill_tie_breaks(o)),
        ("components", lambda o: pins.test_components_add_up(o)),
        ("dfs_tree", lambda o: pins.test_dfs_pseudotree_root_and_order(o)),
        ("mpe", lambda o: pins.test_mpe_log_domain_bruteforce(o)),
    ]
    for seed in range(3):
        calls.append((f"be_bruteforce_{seed}", lambda o, s=seed: pins.test_be_equals_bruteforce(o, s, "int")))
    for seed in range(2):
        calls.append((f"mbe_bounds_{seed}", lambda o, s=seed: pins.test_mbe_bounds_and_exactness(o, s)))
    calls.append(("dpop_sep", lambda o: pins.test_dpop_separators(o, 0)))
    calls.append(("mbe_partition", lambda o: pins.test_mbe_partition_golden(o)))
    calls.append(("mbe_value", lambda o: pins.test_mbe_value_sums_every_minibucket(o)))
    calls += [
        ("logz_direct", lambda o: pins.test_logz_bruteforce_is_the_partition_function(o, 1)),
        ("sum_bruteforce", lambda o: pins.test_sum_elimination_equals_bruteforce(o, 0)),
        ("bn_z_one", lambda o: pins.test_bayes_net_partition_function_is_one(o)),
        ("bn_evidence", lambda o: pins.test_bayes_net_probability_of_evidence(o)),
        ("ising", lambda o: pins.test_ising_ring_closed_form(o)),
        ("coloring", lambda o: pins.test_coloring_counts_closed_forms(o)),
        ("sum_mbe", lambda o: pins.test_sum_minibuckets_bound_and_exactness(o, 0)),
    ]
    return calls


def _failing_pins(so_path):
    failed = []
    with oracle.use_library(so_path):
        for name, call in _pin_calls():
            try:
                call(oracle)
            except AssertionError:
                failed.append(name)
    return failed


def _build(tmp_path, src, tag):
    c = tmp_path / f"{tag}.c"
    so = tmp_path / f"{tag}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", str(c), "-o", str(so), "-lm"], check=True)
    return str(so)


def test_unmodified_oracle_passes_the_harness(tmp_path):
    assert _failing_pins(_build(tmp_path, open(SRC).read(), "orig")) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    failed = _failing_pins(_build(tmp_path, src.replace(old, new, 1), "mutant"))
    assert failed, f"no pin caught: {name}"
