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
