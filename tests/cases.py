"""Seeded test problems: inputs from ``synth``, expected counts from the oracle."""
import numpy as np

import oracle
import synth
from synth import configs
import paper_2503_19925_gb300 as ex


def spectrum(K, W, seed, n, kind="partition"):
    e = synth.energy_grid(K)
    phi = synth.smooth_spectrum(e, seed)
    D = synth.window_partition(K, W) if kind == "partition" else synth.window_trapezoids(K, W, seed)
    return D * phi[None, :], synth.power_law_mu(e, configs.mu_scale(n))


def problem(geom: dict, K=10, W=1, I0=1e4, n_ellipses=6, seed=0, noise=True, bf16=False):
    """Returns dict(g_or, g_gpu, S, mu, xs, y, I0) with y [W][V][B] float64
    (rounded to BF16 values when bf16=True)."""
    g_or = oracle.Geometry(**geom)
    g_gpu = ex.Geometry(**geom)
    n = max(g_or.nx, g_or.ny)
    S, mu = spectrum(K, W, seed, n)
    xs = synth.rasterize_ellipses(synth.random_ellipses(n, n_ellipses, seed), g_or.nx, g_or.ny,
                                  supersample=2)
    lam = oracle.expected_counts(oracle.forward(g_or, xs), S, mu, I0)
    y = synth.poisson_counts(lam, seed + 1) if noise else lam
    if bf16:
        import torch
        y = torch.from_numpy(y).to(torch.bfloat16).to(torch.float64).numpy()
    return dict(g_or=g_or, g_gpu=g_gpu, S=S, mu=mu, xs=xs, y=y, I0=I0)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def psnr(x, ref):
    """PSNR in dB for images with range [0, 1]: 20 log10(1 / RMSE)."""
    rmse = np.sqrt(np.mean((np.asarray(x, np.float64) - ref) ** 2))
    return float(20 * np.log10(1.0 / rmse))
