"""Planted mistakes in copies of the oracle: each one must fail at least one
pin of tests/test_oracle_*.py.

The pins are meant to be chosen so that a plausible mistake anywhere in the
oracle (a dropped term, a wrong sign or index, a transposed operand, a wrong
normalisation) shows.  This test makes that claim checkable.

* The C estimator (part 1): a copy of ``oracle/mcf_oracle.c`` with one
  textual change is compiled with the oracle's own flags into a temporary
  directory, and the pin modules run against it (``MCF_ORACLE_LIB`` makes
  ``oracle.estimator`` load that build).
* The float64 reference (part 2): a temporary tree holds a copy of
  ``oracle/`` whose ``reference.py`` carries one change, and a copy of
  ``tests/``; the pin modules run from there.

An unchanged copy must pass every pin, and every changed copy must fail one.
The oracle in the tree is never modified.  Each mistake names the passage of
the paper (or the reading, or the mathematics) that it violates.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

from oracle import estimator as E
from paper_2308_01037_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mcf_oracle.c")
REF = os.path.join(ROOT, "oracle", "reference.py")
PINS = ["tests/test_oracle_estimator.py", "tests/test_oracle_general.py", "tests/test_oracle_philox.py"]
REF_PINS = ["tests/test_oracle_reference.py", "tests/test_oracle_estimator.py", "tests/test_oracle_general.py"]

# (name, what it violates, text in mcf_oracle.c, planted replacement)
MUTANTS = [
    ("philox_weyl_constant", "Philox4x32-10 key schedule (Salmon et al.)",
     "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE86u;"),
    ("philox_nine_rounds", "Philox4x32-10: ten rounds",
     "for (int round = 0; round < 10; ++round) {", "for (int round = 0; round < 9; ++round) {"),
    ("uniform_word_layout", "one independent word per transition (reading of SelectNextState)",
     "w[0] = u[k % 4];", "w[0] = u[0];"),
    ("weighted_words_equal", "two independent words per weighted transition",
     "w[1] = u[2 * (k % 2) + 1];", "w[1] = u[2 * (k % 2)];"),
    ("alias_uniform_halved", "alias test x uniform on [0, 1) (Definition 1 transition probabilities)",
     "float x = (float)(w[1] >> 8) * 5.9604644775390625e-08f;",
     "float x = (float)(w[1] >> 9) * 5.9604644775390625e-08f;"),
    ("alias_branch_swapped", "Vose alias sampling of t_ij = |a_ij| / sum_k |a_ik|",
     "return x < c->prob[p] ? b : (int64_t)c->alias[p];", "return x < c->prob[p] ? (int64_t)c->alias[p] : b;"),
    ("alias_residual", "Vose alias table construction",
     "s[g] = (s[g] + s[l]) - 1.0;", "s[g] = s[g] - s[l];"),
    ("zeta_index_f64", "Eq. random_walk_realization: W^(k) carries zeta_(k+2)",
     "zeta[k + 2] * W, 0.0f", "zeta[k + 1] * W, 0.0f"),
    ("zeta_index_f32", "Eq. random_walk_realization, float32 weights",
     "(float)zeta[k + 2] * W32", "(float)zeta[k + 1] * W32"),
    ("cutoff_after_add", "Eq. weight_cutoff: the test precedes the visit (while condition of Algorithms 2/3)",
     "        if (!(wabs > w_cutoff)) break;                   /* Eq. weight_cutoff */\n"
     "        if (precision == 0) visit(ctx, l, zeta[k + 2] * W, 0.0f);\n"
     "        else visit(ctx, l, 0.0, (float)zeta[k + 2] * W32);\n",
     "        if (precision == 0) visit(ctx, l, zeta[k + 2] * W, 0.0f);\n"
     "        else visit(ctx, l, 0.0, (float)zeta[k + 2] * W32);\n"
     "        if (!(wabs > w_cutoff)) break;\n"),
    ("truncation_one_short", "truncation at zeta_K (a walk makes at most K - 2 transitions)",
     "if (k + 2 >= K) break;", "if (k + 3 >= K) break;"),
    ("weight_sign_dropped", "Eq. weights: a_ij / t_ij keeps the sign of a_ij",
     "if (c->val && c->val[pos] < 0.0f) m = -m;", "(void)pos;"),
    ("weight_of_entered_row", "Eq. weights: the ratio uses the row the walk leaves",
     "double m = c->rowabs[l];", "double m = c->rowabs[c->ci[pos]];"),
    ("colnorm_proportional_to_degree", "Eq. initial_prob: p_i proportional to ||C_i||_2",
     "c->colnorm[i] = gamma * sqrt((double)(c->cp[i + 1] - c->cp[i]));",
     "c->colnorm[i] = gamma * (double)(c->cp[i + 1] - c->cp[i]);"),
    ("colnorm_from_row_sums", "Eq. initial_prob: column 2-norms, not row 1-norms",
     "c->colnorm[i] = gamma * sqrt(sq);", "c->colnorm[i] = gamma * sa;"),
    ("column_values_in_row_order", "Definition 1 on a general A: columns read from A, not from its rows",
     "if (val) c->cv[q] = val[p];", "if (val) c->cv[q] = val[q];"),
    ("allocation_without_floor", "reading of N_i = N_s p_i: at least one walk per non-empty column",
     "c->nw[i] = r < 1 ? 1 : (int64_t)r;", "c->nw[i] = (int64_t)r;"),
    ("r_unscaled", "Algorithm 3: r = A'v with A' = gamma A",
     "        r[i] = gamma * s;\n        r32[i] = (float)r[i];\n    }\n    int64_t walks = 0, steps = 0;",
     "        r[i] = s;\n        r32[i] = (float)r[i];\n    }\n    int64_t walks = 0, steps = 0;"),
    ("action_zeta1_dropped", "Algorithm 3: y = zeta_0 v + zeta_1 r + A'q",
     "if (K >= 1) yi += zeta[1] * r[i];", "(void)r;"),
    ("action_Aq_unscaled", "Algorithm 3: the last product is with A' = gamma A",
     "yi += gamma * aq;", "yi += aq;"),
    ("action_q_normalisation", "Algorithm 3: q_i is the mean over N_i walks",
     "q[i] = a.acc / (double)c.nw[i];", "q[i] = a.acc / (double)(c.nw[i] + 1);"),
    ("subset_starts", "Section 4.3: entry i needs the walks of the columns adjacent to i",
     "for (int64_t p = rp[i]; p < rp[i + 1]; ++p) mark[ci[p]] = 1;", "mark[i] = 1;"),
    ("diag_aik_missing", "Eq. rand_funm_formula_diag: d_i sums a'_ik <Q_k, C_i>",
     "acc[i] += (aik * dot) / (double)c.nw[k];", "acc[i] += dot / (double)c.nw[k]; (void)aik;"),
    ("diag_divides_by_N_i", "Eq. rand_funm_Q: row Q_k is the mean over N_k walks",
     "acc[i] += (aik * dot) / (double)c.nw[k];", "acc[i] += (aik * dot) / (double)c.nw[i];"),
    ("diag_dot_with_column_k", "Eq. rand_funm_formula_diag: Q_k is dotted with column i",
     "for (int64_t t = c.cp[i]; t < c.cp[i + 1]; ++t)   /* column i: entries a_ji */",
     "for (int64_t t = c.cp[k]; t < c.cp[k + 1]; ++t)"),
    ("diag_aii_dropped", "Eq. rand_funm_formula_diag: the zeta_1 a'_ii term",
     "if (K >= 1) di += zeta[1] * (gamma * entry(rp, ci, val, i, i));", "(void)entry;"),
    ("diag_Q_not_cleared", "Eq. rand_funm_Q: each Q_k holds only the walks from column k",
     "dc.Q[dc.touched[t]] = 0.0; dc.seen[dc.touched[t]] = 0; }", "dc.seen[dc.touched[t]] = 0; }"),
    ("diag_precision_swapped", "float32-weight reading: visits carry the float32 term",
     "d->Q[l] += d->precision == 1 ? (double)zw32 : zw;", "d->Q[l] += d->precision == 1 ? zw : (double)zw32;"),
    ("full_right_factor_transposed", "Algorithm 2: F = zeta_0 I + zeta_1 A' + (A'Q) A'",
     "for (int64_t i = 0; i < n; ++i) F[i * n + j] += AQ[i * n + m] * a;",
     "for (int64_t i = 0; i < n; ++i) F[j * n + i] += AQ[i * n + m] * a;"),
    ("full_left_factor_row", "Algorithm 2: (A'Q)_i sums a'_im Q_m",
     "const double* qrow = Qm + (int64_t)ci[p] * n;", "const double* qrow = Qm + i * n; (void)ci;"),
    ("full_Q_unnormalised", "Eq. rand_funm_Q: Q_i divided by N_i",
     "Qm[i * n + j] /= (double)c.nw[i];", "Qm[i * n + j] /= 1.0;"),
    ("full_zeta1_dropped", "Algorithm 2: the zeta_1 A' term",
     "if (K >= 1) F[i * n + ci[p]] += zeta[1] * a;", "(void)a;"),
    ("classic_v_of_start", "Algorithm 1: each step adds zeta_k W v at the current state",
     "acc += zeta[k] * W * v[l];", "acc += zeta[k] * W * v[i];"),
    ("classic_truncation", "Algorithm 1: terms zeta_0 .. zeta_K",
     "if (k >= K) break;", "if (k + 1 >= K) break;"),
    ("classic_sign_dropped", "Algorithm 1 with Eq. weights: signed weight ratio",
     "W = W * weight_ratio(&c, l, p);", "W = W * c.rowabs[l];"),
    ("se_not_divided_by_N", "Section 3.5: Var(q_i) = s_i^2 / N_i",
     "w[i] = ss / ((double)(N - 1) * (double)N);", "w[i] = ss / (double)(N - 1);"),
    ("se_sum_of_squares", "sample variance: sum X^2 - N mean^2",
     "double ss = sum2 - (double)N * mean * mean;", "double ss = sum2 - mean * mean;"),
    ("se_weight_not_squared", "Var(y_j) = sum_i a'_ji^2 Var(q_i)",
     "var += a * a * w[ci[p]];", "var += a * w[ci[p]];"),
]


# (name, what it violates, text in reference.py, planted replacement)
REFERENCE_MUTANTS = [
    ("exp_factorial", "zeta_k = 1/k! of the exponential",
     "beta ** k / math.factorial(k)", "beta ** k / math.factorial(k + 1)"),
    ("katz_tail_one_short", "geometric tail rho^(K+1) / (1 - rho) of the Neumann series",
     "/ math.log(rho) - 1.0)))", "/ math.log(rho))))"),
    ("mittag_leffler_beta", "zeta_k = 1 / Gamma(alpha k + beta)",
     "math.exp(-math.lgamma(alpha * k + beta))", "math.exp(-math.lgamma(alpha * k + 1.0))"),
    ("csr_without_gamma", "A' = gamma A (Section 2.2)",
     "return sp.csr_matrix((gamma * data,", "return sp.csr_matrix((data,"),
    ("lambda_second_largest", "scale 1/lambda_max",
     "return float(np.linalg.eigvalsh(csr_matrix(g, values).toarray())[-1])",
     "return float(np.linalg.eigvalsh(csr_matrix(g, values).toarray())[-2])"),
    ("arpack_smallest", "scale 1/lambda_max (large graphs)", 'which="LA"', 'which="SA"'),
    ("gershgorin_signed_sum", "Gershgorin bound max_i sum_k |a_ik| (Section 4.5)",
     "np.abs(A).sum(axis=1).max()", "A.sum(axis=1).max()"),
    ("eigen_reconstruction", "f(A) = V f(Lambda) V^T",
     "return (V * f) @ V.T", "return (V * f) @ V"),
    ("powers_not_accumulated", "Eq. power_series: A^k by repeated products",
     "            P = P @ A\n", "            P = A\n"),
    ("series_zeta0_dropped", "Eq. power_series: the zeta_0 v term",
     "y = coeffs[0] * t\n", "y = 0.0 * t\n"),
    ("series_diag_entries", "diagonal entries (e_i^T f(A') e_i)",
     "out[b0:b0 + block] = D[idx, np.arange(len(idx))]",
     "out[b0:b0 + block] = D[np.arange(len(idx)), np.arange(len(idx))]"),
    ("walk_zeta_index", "Lemma 2: W^(k) carries zeta_(k+2)",
     "X = X + coeffs[k + 2] * W * contrib(l)", "X = X + coeffs[k + 1] * W * contrib(l)"),
    ("walk_truncation", "truncation at zeta_K",
     "leaf = (k + 2 >= K) or len(nbr[l]) == 0", "leaf = (k + 3 >= K) or len(nbr[l]) == 0"),
    ("walk_weight_without_t", "Eq. weights: W multiplied by a_ij / t_ij",
     "stack.append((j, k + 1, W * (a / t), P * t, X))", "stack.append((j, k + 1, W * a, P * t, X))"),
    ("walk_probability_without_t", "Definition 1: a path has probability prod t",
     "stack.append((j, k + 1, W * (a / t), P * t, X))", "stack.append((j, k + 1, W * (a / t), P, X))"),
    ("walk_cutoff_after_add", "Eq. weight_cutoff: the test precedes the visit",
     "        if not (abs(W) > w_cutoff):\n            leaf = True\n        else:\n"
     "            X = X + coeffs[k + 2] * W * contrib(l)\n            leaf = (k + 2 >= K) or len(nbr[l]) == 0\n",
     "        X = X + coeffs[k + 2] * W * contrib(l)\n        if not (abs(W) > w_cutoff):\n"
     "            leaf = True\n        else:\n            leaf = (k + 2 >= K) or len(nbr[l]) == 0\n"),
    ("enum_action_zeta1_dropped", "Algorithm 3: y = zeta_0 v + zeta_1 r + A'q",
     "y = coeffs[0] * v + (coeffs[1] * r if K >= 1 else 0.0)", "y = coeffs[0] * v"),
    ("action_variance_not_squared", "Var(y_j) = sum_i a'_ji^2 Var(X_i) / N_i",
     'var[j] += a * a * ex["var_walk"][i] / nw[i]', 'var[j] += a * ex["var_walk"][i] / nw[i]'),
    ("action_variance_N_of_j", "Var(y_j) = sum_i a'_ji^2 Var(X_i) / N_i",
     'var[j] += a * a * ex["var_walk"][i] / nw[i]', 'var[j] += a * a * ex["var_walk"][i] / nw[j]'),
    ("enum_diag_row_k", "Eq. rand_funm_formula_diag: the rows i of column k",
     "for i in np.nonzero(Arow[:, k])[0]:", "for i in np.nonzero(Arow[k, :])[0]:"),
    ("enum_diag_aik_missing", "Eq. rand_funm_formula_diag: a'_ik <Q_k, C_i>",
     "mean[i] += a * e1[i]", "mean[i] += e1[i]"),
    ("enum_diag_aii_dropped", "Eq. rand_funm_formula_diag: the zeta_1 a'_ii term",
     "coeffs[1] * Arow[i, i] if K >= 1 else 0.0", "0.0 * Arow[i, i] if K >= 1 else 0.0"),
    ("enum_diag_variance_N_of_i", "Var(d_i) = sum_k a'_ik^2 Var(Y_k,i) / N_k",
     "var[i] += a * a * max(e2[i] - e1[i] ** 2, 0.0) / nw[k]",
     "var[i] += a * a * max(e2[i] - e1[i] ** 2, 0.0) / nw[i]"),
    ("enum_rows_transposed", "a visit of l adds row l of A'",
     "Arow[i, j] += a\n", "Arow[j, i] += a\n"),
    ("moment_signed_entries", "second moments carry |a'_ij| (Definition 1, Eq. weights)",
     "A = abs(csr_matrix(g, values, gamma))", "A = csr_matrix(g, values, gamma)"),
    ("moment_without_row_sums", "M = diag(s') |A'|: the weight multiplier s'_l",
     "S = sp.diags(r) @ A @ sp.diags(r)", "S = A"),
    ("moment_rows_squared", "M = diag(s') |A'| is similar to D^1/2 |A'| D^1/2",
     "r = np.sqrt(s)", "r = s"),
]


def _pytest(pins, cwd, env):
    r = subprocess.run([sys.executable, "-m", "pytest", *pins, "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=cwd, env=env, capture_output=True, text=True, timeout=900)
    lines = r.stdout.splitlines()
    failed = [ln for ln in lines if ln.startswith(("FAILED", "ERROR"))]
    return r.returncode, failed[0] if failed else (lines[-1] if lines else r.stderr[-300:])


def _run_reference_pins(text, lib):
    """Runs the pin modules from a temporary tree whose oracle/reference.py is ``text``."""
    with tempfile.TemporaryDirectory(prefix="reference_mutant_") as d:
        skip = shutil.ignore_patterns("__pycache__", "_build")
        shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"), ignore=skip)
        shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(d, "tests"), ignore=skip)
        os.symlink(os.path.join(ROOT, "paper_2308_01037_gb300"), os.path.join(d, "paper_2308_01037_gb300"))
        with open(os.path.join(d, "oracle", "reference.py"), "w") as f:
            f.write(text)
        env = dict(os.environ, MCF_ORACLE_LIB=lib, OMP_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1")
        return _pytest(REF_PINS, d, env)


def _run_pins(text):
    """Compiles ``text`` as the oracle and runs the pin modules against it;
    returns (pytest exit code, first failing test or last line)."""
    with tempfile.TemporaryDirectory(prefix="oracle_mutant_") as d:
        src = os.path.join(d, "mcf_oracle.c")
        so = os.path.join(d, "liboracle.so")
        with open(src, "w") as f:
            f.write(text)
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", src,
                        "-o", so, "-lm"], check=True, capture_output=True)
        env = dict(os.environ, MCF_ORACLE_LIB=so, OMP_NUM_THREADS="1")
        return _pytest(PINS, ROOT, env)


def _jobs(path, mutants, what):
    with open(path) as f:
        text = f.read()
    for name, _, old, _ in mutants:
        assert text.count(old) == 1, f"{name}: the text to change must occur exactly once in {what}"
    return [("unchanged", text)] + [(name, text.replace(old, new)) for name, _, old, new in mutants]


@pytest.fixture(scope="module")
def outcomes():
    I.build()
    lib = E.build()
    jobs = [("c", name, text) for name, text in _jobs(SRC, MUTANTS, "mcf_oracle.c")]
    jobs += [("py", name, text) for name, text in _jobs(REF, REFERENCE_MUTANTS, "reference.py")]

    def run(job):
        kind, _, text = job
        return _run_pins(text) if kind == "c" else _run_reference_pins(text, lib)

    with cf.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        res = list(ex.map(run, jobs))
    return {(kind, name): r for (kind, name, _), r in zip(jobs, res)}


@pytest.mark.parametrize("kind", ["c", "py"])
def test_unchanged_copy_passes_every_pin(outcomes, kind):
    rc, info = outcomes[(kind, "unchanged")]
    assert rc == 0, info


@pytest.mark.parametrize("kind", ["c", "py"])
def test_every_planted_mistake_fails_a_pin(outcomes, kind):
    survived = {name: info for (k, name), (rc, info) in outcomes.items()
                if k == kind and name != "unchanged" and rc != 1}
    assert not survived, f"planted mistakes that no pin caught (or that broke the run): {survived}"
