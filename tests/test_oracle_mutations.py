"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/exact_oracle.c`` (on the
CPU), rebuilds that copy in a temporary directory and runs the pin tests
against it in a subprocess; the run must fail.  The unmodified source must
pass the same selection (checked by the rest of the suite).
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "exact_oracle.c")

MUTATIONS = {
    "transposed_pixel_index": ("return axis == 0 ? x[k * g->nx + j] : x[j * g->nx + k];",
                               "return axis == 0 ? x[j * g->nx + k] : x[k * g->nx + j];"),
    "swapped_interp_weights": ("double w = q == 0 ? 1.0 - f : f;", "double w = q == 0 ? f : 1.0 - f;"),
    "step_length_inverted": ("*delta = g->pixel / fabs(dx);", "*delta = g->pixel * fabs(dx);"),
    "bin_centre_off_by_half": ("double u = ((double)b - 0.5 * (double)(g->n_bins - 1))",
                               "double u = ((double)b - 0.5 * (double)(g->n_bins))"),
    "relu_dropped": ("double tp = t > 0.0 ? t : 0.0;", "double tp = t;"),
    "residual_sign": ("acc += y[(long)w * n + i] - I0 * ora_h_bg(z[i], K, S + (long)w * K, mu, M, mu_bg, p + i, n);",
                      "acc += I0 * ora_h_bg(z[i], K, S + (long)w * K, mu, M, mu_bg, p + i, n) - y[(long)w * n + i];"),
    "background_sign": ("for (int m = 0; m < M; ++m) e += mu_bg[m * K + k] * p[m * stride];",
                        "for (int m = 0; m < M; ++m) e -= mu_bg[m * K + k] * p[m * stride];"),
    "normalisation_drops_windows": ("double inv_m = 1.0 / ((double)W * (double)n);",
                                    "double inv_m = 1.0 / (double)n;"),
    "full_step_from_half_point": ("for (long q = 0; q < d; ++q) xn[q] = clampd(x[q] - eta * F[q], lo, hi);",
                                  "for (long q = 0; q < d; ++q) xn[q] = clampd(xh[q] - eta * F[q], lo, hi);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mut = tmp_path / "exact_oracle.c"
    mut.write_text(src.replace(old, new))
    env = dict(os.environ, EXACT_ORACLE_SRC=str(mut), OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           "tests/test_oracle_projector.py", "tests/test_oracle_operator.py", "tests/test_oracle_background.py"]
    proc = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert proc.returncode == 1, f"mutation {name} was not caught:\n{proc.stdout[-2000:]}"
    assert " failed" in proc.stdout
