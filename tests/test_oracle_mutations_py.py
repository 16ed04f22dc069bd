"""The pins of the Python parts of the oracle (TV projection, running-average
rule, dense operator) must catch plausible mistakes.

Each case copies the oracle, the input generators, the package's Python
binding and the pin tests into a temporary tree, plants one mistake in the
copied oracle (on the CPU), and runs the pins there in a subprocess; the run
must fail.  The unmodified oracle passes the same pins in the rest of the
suite.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# file, old, new, pin test files that must catch it
MUTATIONS = {
    "tv_backward_differences": ("oracle/tv.py", "gx[:, :-1] = x[:, 1:] - x[:, :-1]", "gx[:, 1:] = x[:, 1:] - x[:, :-1]",
                                ["tests/test_oracle_tv.py"]),
    "tv_div_sign": ("oracle/tv.py", "d[:-1, :] += py[:-1, :]\n    d[1:, :] -= py[:-1, :]",
                    "d[:-1, :] -= py[:-1, :]\n    d[1:, :] += py[:-1, :]", ["tests/test_oracle_tv.py"]),
    "tv_anisotropic_norm": ("oracle/tv.py", "return float(np.sqrt(gx * gx + gy * gy).sum())",
                            "return float((np.abs(gx) + np.abs(gy)).sum())", ["tests/test_oracle_tv.py"]),
    "prox_theta_not_halved": ("oracle/tv.py", "theta = 0.5 * lam", "theta = lam", ["tests/test_oracle_tv.py"]),
    "prox_projection_anisotropic": ("oracle/tv.py", "nrm = np.maximum(1.0, np.sqrt(qx * qx + qy * qy))",
                                    "nrm = np.maximum(1.0, np.maximum(np.abs(qx), np.abs(qy)))",
                                    ["tests/test_oracle_tv.py"]),
    "bisection_direction": ("oracle/tv.py", "        if T > tau:\n            lo = lam\n        else:\n            hi = lam",
                            "        if T < tau:\n            lo = lam\n        else:\n            hi = lam",
                            ["tests/test_oracle_tv.py"]),
    "dykstra_q_dropped": ("oracle/tv.py", "        q = y + q - zn", "        q = q * 0.0", ["tests/test_oracle_tv.py"]),
    "dykstra_p_dropped": ("oracle/tv.py", "        p = w - y", "        p = p * 0.0", ["tests/test_oracle_tv.py"]),
    "window_one_too_long": ("oracle/__init__.py", "    return max(1, t // 2)", "    return max(1, t // 2 + 1)",
                            ["tests/test_oracle_running_average.py"]),
    "window_slice_off_by_one": ("oracle/__init__.py", "        out.append(sum(xs[t - m:t]) / m)",
                                "        out.append(sum(xs[t - m - 1:t - 1]) / m)",
                                ["tests/test_oracle_running_average.py"]),
    "dense_relu_dropped": ("oracle/dense.py", "tp = np.maximum(np.asarray(t, dtype=np.float64), 0.0)",
                           "tp = np.asarray(t, dtype=np.float64)", ["tests/test_oracle_operator.py"]),
    "dense_normalisation_drops_windows": ("oracle/dense.py", "return A.T @ r / (S.shape[0] * A.shape[0])",
                                          "return A.T @ r / A.shape[0]", ["tests/test_oracle_operator.py"]),
}


def _tree(dst):
    for d in ("oracle", "synth", "paper_2503_19925_gb300", "tests"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d),
                        ignore=shutil.ignore_patterns("_build", "__pycache__", "*.so"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), dst)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_python_oracle_pins_catch_mutation(name, tmp_path):
    rel, old, new, tests = MUTATIONS[name]
    _tree(str(tmp_path))
    path = tmp_path / rel
    src = path.read_text()
    assert src.count(old) == 1, name
    path.write_text(src.replace(old, new))
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"] + tests
    proc = subprocess.run(cmd, cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=900)
    assert proc.returncode == 1, f"mutation {name} was not caught:\n{proc.stdout[-2000:]}"
    assert " failed" in proc.stdout
