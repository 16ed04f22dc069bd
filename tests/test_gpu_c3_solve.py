"""Whole-solve parity on the 512^2 fan-beam workload (720 views x 736 bins over
360 deg, 4 windows over 64 energies, BF16-rounded Poisson counts, I0 = 1e4):
the CUDA path's projected extragradient iterates (Eq. (11)) after 100 and 500
iterations against the FP64 oracle's, from the same counts, step and x_1 = 0,
in the launch configuration the benchmark times (autotuned adjoint split).

The oracle iterates are stored in tests/golden/c3_oracle.npz by
tests/golden/make_c3_oracle.py (about 45 min of oracle time); the counts are
regenerated here with the oracle's projector and link from the same seeds.
Bar: relative L2 error <= 1e-3 and |PSNR difference| <= 0.05 dB (PSNR of each
image against the phantom)."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "c3_oracle.npz")
sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
import make_c3_oracle  # noqa: E402

sys.path.pop(0)


def _golden():
    data = np.load(GOLDEN)
    return data, json.loads(str(data["meta"]))


def test_stored_oracle_iterates_are_current():
    """The stored iterates were computed by the current oracle and input
    sources, at the step and checkpoints the file records."""
    data, meta = _golden()
    assert meta["sources_sha256"] == make_c3_oracle.source_digest(), \
        "tests/golden/c3_oracle.npz is stale: rerun tests/golden/make_c3_oracle.py"
    assert meta["checkpoints"] == [100, 500]
    for t in meta["checkpoints"]:
        x = data[f"x{t}"]
        assert x.shape == (512, 512) and np.isfinite(x).all() and x.min() >= 0.0
    # the iteration makes progress between the checkpoints (not a stored zero image)
    assert np.linalg.norm(data["x500"] - data["x100"]) > 1e-3 * np.linalg.norm(data["x500"])


@pytest.mark.gpu
def test_c3_solve_matches_oracle_after_100_and_500_iterations():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import bench
    import paper_2503_19925_gb300 as ex

    data, meta = _golden()
    assert meta["sources_sha256"] == make_c3_oracle.source_digest()
    _, cfg, _, S, mu, y, _ = bench.oracle_inputs("C3", norm_iters=0)
    _, _, _, xs, _ = bench.workload("C3")
    plan = ex.Plan(ex.Geometry(**cfg["geometry"]), mu, S)
    plan.autotune()  # as the benchmark does
    yb = torch.as_tensor(y, dtype=torch.bfloat16, device="cuda:0").contiguous()
    # the counts are BF16 values already: the conversion is exact
    assert np.array_equal(yb.double().cpu().numpy(), y)
    x = torch.zeros((512, 512), dtype=torch.float32, device="cuda:0")

    def psnr(a):
        return 20.0 * np.log10(1.0 / np.sqrt(np.mean((np.asarray(a, np.float64) - xs) ** 2)))

    done = 0
    for t in meta["checkpoints"]:
        _, info = plan.solve(yb, meta["I0"], meta["eta"], t - done, x=x)
        assert info.status == 0 and info.iters_done == t - done
        done = t
        ref = data[f"x{t}"].astype(np.float64)
        got = x.double().cpu().numpy()
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 1e-3, (t, rel)
        assert abs(psnr(got) - psnr(ref)) <= 0.05, (t, psnr(got), psnr(ref))
    plan.close()
