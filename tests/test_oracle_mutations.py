"""Plant plausible mistakes in a copy of the oracle (CPU only) and check that
the pins in test_oracle_pins.py catch every one of them."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "elm_oracle.c")

MUTANTS = {
    "bias_dropped": ("z[j] = s * orc_g(z[j] + b[j], act);", "z[j] = s * orc_g(z[j], act);"),
    "sigmoid_sign": ("1.0 / (1.0 + exp(-z))", "1.0 / (1.0 + exp(z))"),
    "gram_operand": ("s[l] += hj * h[l];", "s[l] += hj * h[j];"),
    "pivot_min": ("if (aj > ap ||", "if (aj < ap ||"),
    "update_sign": ("A[j * L + l] -= R[k * L + j] * R[k * L + l];",
                    "A[j * L + l] += R[k * L + j] * R[k * L + l];"),
    "unscale_index": ("R[i * L + j] *= sqrt(d[perm[j]]);", "R[i * L + j] *= sqrt(d[j]);"),
    "no_min_norm_solve": ("rc = orc_chol(M, r, U);\n        if (rc == 0) {",
                          "rc = orc_chol(M, r, U);\n        if (0) {"),
    "beta2_transposed": ("v += K[i * q + j] * y[i * m + t];", "v += K[j * q + i % q] * y[i * m + t];"),
    "refine_sign": ("Y[i] = T[i] - Y[i];", "Y[i] = Y[i] - T[i];"),
    "forward_solve_index": ("v -= U[j * ldu + i] * B[j * q + c];", "v -= U[i * ldu + j] * B[j * q + c];"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, name
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(before, after))
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                    "-o", str(lib), str(mut), "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "mutant %s survived the pins:\n%s" % (name, r.stdout[-2000:])
