"""The oracle's pins catch plausible mistakes: each case plants one mistake
in a copy of oracle.c (a dropped factor, an overwrite instead of a sum, an
off-by-one in the product count, a signed error scale, a wrong operand in
either gradient, repeated columns counted twice, an inclusive prune
threshold, top-k keeping the smallest, no inflation, no normalisation) and
runs the pin tests against it; every mutant must fail
them, and the unmodified copy must pass. CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "dropped_a_factor": ("double prod = a * (double)valB[t];", "double prod = (double)valB[t];"),
    "overwrite_not_add": ("spa[c] += prod;", "spa[c] = prod;"),
    "ip_off_by_one": ("count += (int64_t)(rptB[k + 1] - rptB[k]);",
                      "count += (int64_t)(rptB[k + 1] - rptB[k] - 1);"),
    "signed_error_scale": ("mag[c] += fabs(prod);", "mag[c] += prod;"),
    "dA_wrong_operand": ("acc += g[c] * (double)valB[t];", "acc += g[c] * (double)valA[j];"),
    "dB_wrong_operand": ("if (dB) dB[t] += (double)valA[j] * g[c];",
                         "if (dB) dB[t] += (double)valB[t] * g[c];"),
    "symbolic_counts_repeats": ("if (seen[c] != (int64_t)r) { seen[c] = (int64_t)r; ++nnz; }",
                                "{ seen[c] = (int64_t)r; ++nnz; }"),
    "mcl_prune_inclusive": ("if (decide < (float)theta) continue;",
                            "if (decide <= (float)theta) continue;"),
    "mcl_topk_keeps_smallest": ("if (x[0] > y[0]) return -1;\n    if (x[0] < y[0]) return 1;",
                                "if (x[0] < y[0]) return -1;\n    if (x[0] > y[0]) return 1;"),
    "mcl_no_inflation": ("double w = pow(v, r);", "double w = v;"),
    "normalise_unscaled": ("out[q] = s > 0 ? (double)val[q] / s : 0.0;",
                           "out[q] = (double)val[q];"),
}


def run_pins(tmp_path, text):
    d = tmp_path / "src"
    d.mkdir()
    (d / "oracle.c").write_text(text)
    env = dict(os.environ, ORACLE_C_SOURCE=str(d / "oracle.c"))
    p = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle.py", "-q", "-x",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert (d / "liboracle.so").exists()          # the copy was built and used
    return p


def test_unmodified_copy_passes(tmp_path):
    p = run_pins(tmp_path, open(SRC).read())
    assert p.returncode == 0, p.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1
    p = run_pins(tmp_path, text.replace(old, new))
    assert p.returncode == 1 and " failed" in p.stdout, p.stdout[-2000:]


# The numpy oracles (pruned layer, Eqs. 1-3; bulk sampling): a mistake is
# planted in a copy of the oracle package beside a copy of the tests, whose
# path setup then imports the copy.
PY_MUTANTS = {
    "topk_ties_to_larger_column": (
        "layers.py", "order = np.lexsort((cols, 0xFFFFFFFF - key[i]))",
        "order = np.lexsort((-cols, 0xFFFFFFFF - key[i]))"),
    "topk_keeps_smallest": (
        "layers.py", "order = np.lexsort((cols, 0xFFFFFFFF - key[i]))",
        "order = np.lexsort((cols, key[i]))"),
    "topk_negative_order": (
        "layers.py", "return np.where(neg, 0xFFFFFFFF - b, b | 0x80000000)",
        "return np.where(neg, b, b | 0x80000000)"),
    "forward_unpruned": (
        "layers.py", "T = np.where(M, np.asarray(X, dtype=np.float64), 0.0)\n"
                     "    C = np.asarray(A, dtype=np.float64) @ T",
        "T = np.asarray(X, dtype=np.float64)\n    C = np.asarray(A, dtype=np.float64) @ T"),
    "dX_unmasked": (
        "layers.py", "dX = np.where(M, A64.T @ dY64 @ W64.T, 0.0)", "dX = A64.T @ dY64 @ W64.T"),
    "dX_untransposed_A": (
        "layers.py", "dX = np.where(M, A64.T @ dY64 @ W64.T, 0.0)",
        "dX = np.where(M, A64 @ dY64 @ W64.T, 0.0)"),
    "dW_without_A": ("layers.py", "dW = (A64 @ T).T @ dY64", "dW = T.T @ dY64"),
    "sample_uniform_rounds": (
        "sampling.py", "idx = min(n - 1, int(np.floor(ut * n)))",
        "idx = min(n - 1, int(np.round(ut * n)))"),
    "sample_left_boundary": ("sampling.py", 'side="right"', 'side="left"'),
    "sample_mode2_abs": (
        "sampling.py", "w = w * w if mode == 2 else np.maximum(w, 0.0)",
        "w = np.abs(w) if mode == 2 else np.maximum(w, 0.0)"),
    "sample_negative_weights": (
        "sampling.py", "w = w * w if mode == 2 else np.maximum(w, 0.0)",
        "w = w * w if mode == 2 else w"),
    "sample_short_rows": ("sampling.py", "if n <= s:", "if n < s:"),
    "select_inclusive_rank": (
        "sampling.py", "rank = np.concatenate([[0], np.cumsum(flag)])",
        "rank = np.concatenate([np.cumsum(flag), [flag.sum()]])"),
}
PY_TESTS = {"layers.py": "tests/test_oracle_layers.py", "sampling.py": "tests/test_oracle_sampling.py"}


def run_py_pins(tmp_path, fname, text):
    import shutil
    root = tmp_path / "tree"
    shutil.copytree(os.path.join(ROOT, "oracle"), root / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    (root / "tests").mkdir()
    for f in ("conftest.py", os.path.basename(PY_TESTS[fname])):
        shutil.copy(os.path.join(ROOT, "tests", f), root / "tests" / f)
    (root / "oracle" / fname).write_text(text)
    return subprocess.run([sys.executable, "-m", "pytest", PY_TESTS[fname], "-q", "-x",
                           "-p", "no:cacheprovider"], cwd=root, capture_output=True, text=True,
                          timeout=600)


@pytest.mark.parametrize("fname", sorted(PY_TESTS))
def test_unmodified_numpy_oracle_copy_passes(tmp_path, fname):
    p = run_py_pins(tmp_path, fname, open(os.path.join(ROOT, "oracle", fname)).read())
    assert p.returncode == 0, p.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_planted_numpy_oracle_mistake_is_caught(tmp_path, name):
    fname, old, new = PY_MUTANTS[name]
    text = open(os.path.join(ROOT, "oracle", fname)).read()
    assert text.count(old) == 1
    p = run_py_pins(tmp_path, fname, text.replace(old, new))
    assert p.returncode == 1 and " failed" in p.stdout, p.stdout[-2000:]
