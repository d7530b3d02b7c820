"""The oracle's pins must catch plausible mistakes. Each case plants one mistake (a dropped term,
a wrong sign, an off-by-one index, a transposed operand, a wrong format boundary) in a temporary
copy of oracle.c, builds it, and runs the relevant pin tests against it in a subprocess: they
must fail. The planted copies live in a temporary directory; oracle.c itself is never changed."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    # (name, original text, planted text, pin test files that must catch it)
    ("subnormal_effective_exponent", "uint32_t ebar = e_max > 1 ? e_max : 1;\n  for (int i = 0; i < BS; ++i) {\n    uint64_t u",
     "uint32_t ebar = e_max;\n  for (int i = 0; i < BS; ++i) {\n    uint64_t u", "test_oracle_codec.py"),
    ("significand_index", "int pos = 52 - (int)((uint32_t)t - k);", "int pos = 51 - (int)((uint32_t)t - k);",
     "test_oracle_codec.py"),
    ("decode_exponent", "int32_t e = ebar - k;", "int32_t e = ebar - k + 1;", "test_oracle_codec.py"),
    ("stream_order", "int t = i * l + b;\n        words", "int t = (BS - 1 - i) * l + b;\n        words",
     "test_oracle_codec.py"),
    ("fp16_subnormal_boundary", "round_rne(x, 11, -14, 15)", "round_rne(x, 11, -15, 15)", "test_oracle_cast.py"),
    ("bf16_precision", "round_rne(x, 8, -126, 127)", "round_rne(x, 9, -126, 127)", "test_oracle_cast.py"),
    ("update_wrong_coefficient", "for (int32_t k = 0; k < n; ++k) ws->w[k] -= vi[k] * ws->h[i];",
     "for (int32_t k = 0; k < n; ++k) ws->w[k] -= vi[k] * ws->h[0];", "test_oracle_gmres.py"),
    ("reorth_dropped_correction", "for (int i = 0; i <= j; ++i) ws->h[i] += ws->u[i];", "",
     "test_oracle_gmres.py"),
    ("givens_sign", "Rj[i + 1] = -ws->sn[i] * Rj[i] + ws->cs[i] * Rj[i + 1];",
     "Rj[i + 1] = ws->sn[i] * Rj[i] + ws->cs[i] * Rj[i + 1];", "test_oracle_gmres.py"),
    ("rhs_rotation_sign", "ws->g[j + 1] = -s * ws->g[j];", "ws->g[j + 1] = s * ws->g[j];", "test_oracle_gmres.py"),
    ("backsub_transposed", "t -= ws->R[(size_t)i * ld + k] * ws->y[i];", "t -= ws->R[(size_t)k * ld + i] * ws->y[i];",
     "test_oracle_gmres.py"),
    ("solution_update_dropped_vector",
     "for (int i = 0; i < mls; ++i) {\n      const double* vi = ws->vhat + (size_t)i * n;\n      for (int32_t k = 0; k < n; ++k) x[k]",
     "for (int i = 1; i < mls; ++i) {\n      const double* vi = ws->vhat + (size_t)i * n;\n      for (int32_t k = 0; k < n; ++k) x[k]",
     "test_oracle_gmres.py"),
    ("spmv_dropped_last_entry", "for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) s +=",
     "for (int32_t p = row_ptr[i]; p + 1 < row_ptr[i + 1]; ++p) s +=", "test_oracle_gmres.py"),
    ("jacobi_step3_unpreconditioned", "orc_spmv_csr(n, ws->row_ptr, ws->col, ws->vals, ws->t, ws->w);",
     "orc_spmv_csr(n, ws->row_ptr, ws->col, ws->vals, ws->v, ws->w);", "test_oracle_gmres.py"),
    ("jacobi_step17_unscaled", "for (int32_t k = 0; k < n; ++k) x[k] += ws->dinv[k] * ws->t[k];",
     "for (int32_t k = 0; k < n; ++k) x[k] += ws->t[k];", "test_oracle_gmres.py"),
    ("jacobi_m_not_inverted", "ws->dinv[i] = 1.0 / d;", "ws->dinv[i] = d;", "test_oracle_gmres.py"),
    # the second Gram-Schmidt pass of steps 7-11 and the breakdown exit of step 12
    ("reorth_trigger_flipped", "    if (hn < ws->eta * omega) {", "    if (hn > ws->eta * omega) {",
     "test_oracle_gmres.py"),
    ("reorth_trigger_eta_squared", "    if (hn < ws->eta * omega) {", "    if (hn < ws->eta * ws->eta * omega) {",
     "test_oracle_gmres.py"),
    ("breakdown_literal_step12", "int breakdown = (hn == 0.0) || (did_reorth && hn < ws->eta * h_before);",
     "int breakdown = (hn == 0.0) || (hn < ws->eta * omega);", "test_oracle_gmres.py"),
    ("breakdown_eta_on_omega", "int breakdown = (hn == 0.0) || (did_reorth && hn < ws->eta * h_before);",
     "int breakdown = (hn == 0.0) || (did_reorth && hn < ws->eta * omega);", "test_oracle_gmres.py"),
    ("breakdown_stagnation_dropped", "if (broke_down && res->true_rrn >= cycle_start_rrn) { /* R18 */",
     "if (0) { /* R18 */", "test_oracle_gmres.py"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,orig,planted,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, orig, planted, pins):
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert src.count(orig) == 1, f"mutation anchor for {name} not unique"
    shutil.copy(os.path.join(ROOT, "oracle", "oracle.h"), tmp_path / "oracle.h")
    (tmp_path / "oracle.c").write_text(src.replace(orig, planted))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                    str(tmp_path / "oracle.c"), "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} was not caught by {pins}:\n{r.stdout[-2000:]}"
