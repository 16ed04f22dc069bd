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


def c4_jobs(n_jobs: int = 64, seed: int = 4, sizes=(128, 192, 256, 384, 512), views=(60, 360),
            windows=(1, 4), K: int = 32, I0_range=(1e3, 1e5)):
    """The batched mix: per job an image size from `sizes`, a parallel-beam view
    count uniform in `views` over 180 degrees, B = ceil(N sqrt 2) rounded up to
    odd bins, a window count uniform in `windows`, K energies and I0
    log-uniform in `I0_range`.  Returns a list of dicts (geometry, W, K, I0,
    seed)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n_jobs):
        n = int(rng.choice(sizes))
        v = int(rng.integers(views[0], views[1] + 1))
        b = int(np.ceil(n * np.sqrt(2.0)))
        b += (b + 1) % 2
        w = int(rng.integers(windows[0], windows[1] + 1))
        i0 = float(np.exp(rng.uniform(np.log(I0_range[0]), np.log(I0_range[1]))))
        out.append(dict(geometry=dict(beam=0, nx=n, ny=n, n_views=v, n_bins=b, angle_range=math.pi),
                        W=w, K=K, I0=i0, seed=int(rng.integers(1 << 31))))
    return out


C4 = dict(name="C4", n_jobs=64, iters=100)


def c5_requests(n_jobs: int, seed: int = 5, sizes=(128, 1024), views=(90, 1440), windows=(1, 4),
                energies=(16, 64), I0_range=(1e3, 1e5)):
    """The serving stream: per request an image size uniform in `sizes`
    (multiples of 32), views uniform in `views`, parallel or fan beam 50/50,
    B = ceil(N sqrt 2) (parallel) or the fan's detector coverage, windows
    uniform in `windows`, energies uniform in `energies`, I0 log-uniform."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n_jobs):
        n = int(rng.integers(sizes[0] // 32, sizes[1] // 32 + 1)) * 32
        v = int(rng.integers(views[0], views[1] + 1))
        fan = bool(rng.integers(0, 2))
        w = int(rng.integers(windows[0], windows[1] + 1))
        k = int(rng.integers(energies[0], energies[1] + 1))
        k = max(k, w)
        i0 = float(np.exp(rng.uniform(np.log(I0_range[0]), np.log(I0_range[1]))))
        if fan:
            rs = 2.0 * n
            rd = 3.0 * n
            half = 0.5 * n * np.sqrt(2.0) + 2
            # detector coverage of the image's circumscribed circle, pitch 1.5 at the detector
            cover = 2 * rd * np.tan(np.arcsin(half / rs))
            b = int(np.ceil(cover / 1.5)) | 1
            g = dict(beam=1, nx=n, ny=n, n_views=v, n_bins=b, angle_range=2 * math.pi, bin_pitch=1.5,
                     src_to_center=rs, src_to_det=rd)
        else:
            b = int(np.ceil(n * np.sqrt(2.0))) | 1
            g = dict(beam=0, nx=n, ny=n, n_views=v, n_bins=b, angle_range=math.pi)
        out.append(dict(geometry=g, W=w, K=k, I0=i0, seed=int(rng.integers(1 << 31))))
    return out


C5 = dict(name="C5", tol=1e-4, max_iters=2000, budget_bytes=150e9)
