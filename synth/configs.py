"""Workload configurations (shapes and recipe numbers only).

C1..C3 are the plain/mixed-precision reconstructions, C4 the batched mix and C5
the serving stream.  Each entry gives the scan geometry fields (same names as
``exact_geometry``), the energy/window recipe and the solver settings.  The
paper's own experiments use a 25^2 phantom with 3 windows and 50 energies
(Sec. 3.1) and a 512^2 image with about 10^6 rays (Fig. 1); these synthetic
cases take those shapes and scale them.
"""
import math

C1 = dict(name="C1", geometry=dict(beam=0, nx=64, ny=64, n_views=90, n_bins=91, angle_range=math.pi),
          n_ellipses=6, K=10, W=1, windows="partition", I0=1e4, iters=200, y_dtype="f32")

C2 = dict(name="C2", geometry=dict(beam=0, nx=256, ny=256, n_views=180, n_bins=367, angle_range=math.pi),
          n_ellipses=6, K=32, W=3, windows="partition", I0=1e4, I0_sweep=(1e3, 1e4, 1e5), iters=300,
          y_dtype="f32")

C3 = dict(name="C3", geometry=dict(beam=1, nx=512, ny=512, n_views=720, n_bins=736, angle_range=2 * math.pi,
                                   bin_pitch=1.5, src_to_center=1000.0, src_to_det=1500.0),
          n_ellipses=6, K=64, W=4, windows="partition", I0=1e4, iters=500, y_dtype="bf16")

ALL = {"C1": C1, "C2": C2, "C3": C3}


def mu_scale(n: int) -> float:
    """mu_k = c (E_k/60 keV)^-3 with c = 2/N per unit length: a full-width path
    at density 1 gives mu z = 2 at 60 keV."""
    return 2.0 / n
