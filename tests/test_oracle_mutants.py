"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle.c (on the CPU, in a
temporary directory), builds it, and runs the pin suite against that build
in a child process: the suite has to fail.  The committed oracle is never
modified.
"""
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "sample_std": ("*sigma = sqrt(v / (double)m);", "*sigma = sqrt(v / (double)(m - 1));"),
    "dropped_term": ("for (int32_t k = 0; k < m; ++k) {\n        double d = zi[k] - zj[k];",
                     "for (int32_t k = 1; k < m; ++k) {\n        double d = zi[k] - zj[k];"),
    "dg_sign": ("dg[i] = (x[i + m - 1] - mu) + (x[i - 1] - prev_mu);",
                "dg[i] = (x[i + m - 1] - mu) - (x[i - 1] - prev_mu);"),
    "df_index": ("df[i] = (x[i + m - 1] - x[i - 1]) / 2.0;", "df[i] = (x[i + m] - x[i - 1]) / 2.0;"),
    "exclusion_off_by_one": ("return J->inclusive ? (d > J->excl) : (d >= J->excl);",
                             "return J->inclusive ? (d > J->excl) : (d > J->excl);"),
    "floor_zone": ("return (int64_t)ceil(ez * (double)m);", "return (int64_t)floor(ez * (double)m);"),
    "tie_to_last": ("if (d < best) {", "if (d <= best) {"),
    "grad_transposed": ("grad_x[i + k] += -g[i] * (zj[k] - rho * zi[k]) / (si * d);",
                        "grad_x[i + k] += -g[i] * (zi[k] - rho * zj[k]) / (si * d);"),
    "flat_distance": ("if (fi || J->cflat[j]) {\n                d = flatd;",
                      "if (fi || J->cflat[j]) {\n                d = 2.0 * sqrt((double)m);"),
    "arc_end_inclusive": ("if (a <= k && k < b) ++c;", "if (a <= k && k <= b) ++c;"),
    "iac_scale": ("double iac = 2.0 * (double)k * (double)(l - k) / (double)l;",
                  "double iac = 1.0 * (double)k * (double)(l - k) / (double)l;"),
    "diag_mask_signed": ("if (J->diag_ok && !J->diag_ok[d]) return 0;",
                         "if (J->diag_ok && !J->diag_ok[j > i ? j - i : 0]) return 0;"),
    "raw_unsquared": ("                    acc += e * e;", "                    acc += fabs(e);"),
    "lr_sides_swapped": ("if ((J->side < 0 && j >= i) || (J->side > 0 && j <= i)) return 0;",
                         "if ((J->side > 0 && j >= i) || (J->side < 0 && j <= i)) return 0;"),
    "cac_edge_off_by_one": ("if (k >= edge && k < l - edge && iac > 0.0) {",
                            "if (k > edge && k < l - edge && iac > 0.0) {"),
    "cac_unclamped": ("c = r < 1.0 ? r : 1.0;", "c = r;"),
    "segment_tie_to_last": ("if (best < 0 || cac[k] < cac[best]) best = k;",
                            "if (best < 0 || cac[k] <= cac[best]) best = k;"),
    "second_not_shifted": ("                second = best;\n", ""),
    "raw_missing_sqrt": ("                d = sqrt(acc);", "                d = acc;"),
    "distance_uncapped": ("    return d > cap ? cap : d;", "    return d;"),
    "segment_zone_inclusive": ("if (d < seg_excl || d == 0) masked = 1;",
                               "if (d <= seg_excl || d == 0) masked = 1;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mut_c = tmp_path / "oracle_mut.c"
    mut_c.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-pthread", str(mut_c), "-o", str(so), "-lm"])
    env = dict(os.environ, ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_oracle_pins.py"),
                        os.path.join(HERE, "test_oracle_fluss.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"
