"""Writes tests/golden/c3_oracle.npz: the FP64 oracle's projected
extragradient iterates (Eq. (11), box [0, inf)) on the 512^2 fan-beam workload
(720 views x 736 bins over 360 deg, 4 windows over 64 energies, BF16-rounded
Poisson counts at I0 = 1e4), from x_1 = 0 with step eta = 1/(4L), L the
Lipschitz bound of Sec. 4.2 with ||A||^2 from 20 oracle power iterations.

Stored: x after 100 and after 500 iterations (FP32 copies of the FP64
iterates), eta, and SHA-256 digests of the oracle and input-generator sources
the values were computed with (a test that finds them changed reports the file
as stale).  Inputs come from bench.oracle_inputs (synth draws, oracle
projector and link); nothing here touches the CUDA path.

    python tests/golden/make_c3_oracle.py      # about 45 min on 8 cores
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "c3_oracle.npz")
CHECKPOINTS = (100, 500)
NORM_ITERS = 20
SOURCES = ("oracle/exact_oracle.c", "oracle/__init__.py", "synth/__init__.py", "synth/configs.py")


def source_digest() -> str:
    h = hashlib.sha256()
    for rel in SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def main():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    t0 = time.time()
    oracle, cfg, g, S, mu, y, eta, = bench.oracle_inputs("C3", norm_iters=NORM_ITERS)
    x = np.zeros((g.ny, g.nx))
    out, done = {}, 0
    for t in CHECKPOINTS:
        x = oracle.solve(g, S, mu, cfg["I0"], y, eta, t - done, x1=x).x
        done = t
        out[f"x{t}"] = x.astype(np.float32)
        print(f"{t} iterations after {time.time() - t0:.0f} s", flush=True)
    meta = {"workload": bench.describe(cfg), "eta": eta, "I0": cfg["I0"], "norm_iters": NORM_ITERS,
            "checkpoints": list(CHECKPOINTS), "x1": "zeros", "box": [0.0, None],
            "sources_sha256": source_digest(), "command": "python tests/golden/make_c3_oracle.py"}
    np.savez_compressed(OUT, meta=np.array(json.dumps(meta)), **out)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
