"""Plant plausible mistakes in a copy of the oracle and check the pins catch each.

Every mutation is applied to a temporary copy of ``oracle/qai_oracle.c``
(never to the committed file), compiled with gcc, and loaded in a child
process through ``QAI_ORACLE_LIB``. The child runs the pin tests of
``test_oracle_pins.py``; each mutation must make at least one of them fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "qai_oracle.c")

MUTATIONS = {
    "remove_edt_drops_abc": ("return c * g2 - b * g1 - a * f - a * b * c > 0;",
                             "return c * g2 - b * g1 - a * f > 0;"),
    "query_tie_goes_right": ("g[k] + (h[k] - i) * (h[k] - i) > g[k + 1]",
                             "g[k] + (h[k] - i) * (h[k] - i) >= g[k + 1]"),
    "pass_order_z_first": ("for (int a = 2; a >= 0; a--) {",
                           "for (int a = 0; a < 3; a++) {"),
    "sign_flipped": ("int sign = (p->sign_rule == 1) ? first : sgn64(sum);",
                     "int sign = (p->sign_rule == 1) ? first : -sgn64(sum);"),
    "threshold_strict": ("if (d >= p->grad_threshold) zero_sign = 1;",
                         "if (d > p->grad_threshold) zero_sign = 1;"),
    "propagate_off_by_one": ("S[i] = (I1[i] >= 0) ? S[I1[i]] : 0;",
                             "S[i] = (I1[i] > 0) ? S[I1[i] - 1] : 0;"),
    "b2_rule_inverted": ("if (p->b2_rule == 0 && Q[nb[k]] != Q[i]) continue;",
                         "if (p->b2_rule == 0 && Q[nb[k]] == Q[i]) continue;"),
    "idw_weight_swapped": ("return b / (a + b);", "return a / (a + b);"),
    "interior_too_wide": ("if (c[a] < 1 || c[a] > s->n[a] - 2) return 0;",
                          "if (c[a] < 1 || c[a] > s->n[a] - 1) return 0;"),
    "dequantize_missing_2": ("double dprime = 2.0 * (double)Q[i] * eb;",
                             "double dprime = (double)Q[i] * eb;"),
    "adjoint_dw_missing_factor": ("double dw = w * (1.0 - w) * (0.5 * log((double)b) - 0.5 * log((double)a));",
                                  "double dw = w * (0.5 * log((double)b) - 0.5 * log((double)a));"),
    "adjoint_eta_missing_eb": ("ge += G[i] * S[i] * w * eb;", "ge += G[i] * S[i] * w;"),
    "k2_zero_precedence": ("    if (d1 == 0) return 1.0;                /* on a quantization boundary     */\n"
                           "    if (d2 == 0) return 0.0;",
                           "    if (d2 == 0) return 0.0;\n    if (d1 == 0) return 1.0;"),
    # Section VII-B approximate strategy
    "approx_index_not_global": ("if (I1[i] >= 0) I1[i] += off;", ""),
    "approx_slabs_overlap": ("*z1 = (k + 1) * n0 / nparts;", "*z1 = (k + 1) * n0 / nparts + (k + 1 < nparts);"),
    "approx_edt2_whole_field": ("edt(B2 + off, &sl, D2 + off, I2 + off);", "edt(B2, &s, D2, I2);"),
    "approx_s_not_propagated": ("S[i] = B1[i] ? SB[i] : (I1[i] >= 0 ? SB[I1[i]] : 0);", "S[i] = SB[i];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found: {name}"
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o",
                    str(lib), str(mutated), "-lm"], check=True)
    env = dict(os.environ, QAI_ORACLE_LIB=str(lib), OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_adjoint.py"),
                        os.path.join(ROOT, "tests", "test_oracle_sharded.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutation {name} survived the pins:\n{r.stdout[-2000:]}"
