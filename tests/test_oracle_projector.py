"""Pins for the oracle's projector (A), adjoint (A^T) and norm estimate.

The paper leaves the discretisation of A open (it only asks for nonnegative
entries derived from the Radon transform, Sec. 1 and Sec. 2.1), so the pins
here are: (i) a dense matrix assembled pixel by pixel from two points on
each ray (a different route to the same Joseph weights); (ii) exact row and
column sums for axis-aligned views; (iii) the chord length of the square image
support for a constant image; (iv) analytic line integrals of ellipses, which
the discrete projector must approach as the grid is refined; (v) the adjoint
identity <Ax, r> = <x, A^T r>; (vi) the spectral norm from numpy's SVD.
"""
import numpy as np
import pytest

import oracle
from oracle import Geometry
import synth
from tests.geom_cases import tiny_geometries


def _two_points(g: Geometry, v: int, b: int):
    th = g.angle0 + v * g.angle_range / g.n_views
    es = np.array([np.cos(th), np.sin(th)])
    eu = np.array([-np.sin(th), np.cos(th)])
    u = (b - (g.n_bins - 1) / 2) * g.bin_pitch + g.det_offset
    if g.beam == 0:
        P = u * eu
        return P, P - es
    return g.src_to_center * es, (g.src_to_center - g.src_to_det) * es + u * eu


def dense_A(g: Geometry) -> np.ndarray:
    """Joseph matrix assembled entry by entry: for every ray and every pixel
    centre line of the driving axis, intersect the line through two points of
    the ray with it and give the two nearest pixel centres the weights
    step * (1 - distance/pixel)."""
    Xc = (np.arange(g.nx) - (g.nx - 1) / 2) * g.pixel
    Yc = (np.arange(g.ny) - (g.ny - 1) / 2) * g.pixel
    A = np.zeros((g.n_rays, g.d))
    for v in range(g.n_views):
        for b in range(g.n_bins):
            P, Q = _two_points(g, v, b)
            D = Q - P
            L = np.hypot(*D)
            i = v * g.n_bins + b
            if abs(D[0]) >= abs(D[1]):
                step = g.pixel * L / abs(D[0])
                for ix in range(g.nx):
                    y = P[1] + (Xc[ix] - P[0]) / D[0] * D[1]
                    for iy in range(g.ny):
                        w = max(0.0, 1.0 - abs(y - Yc[iy]) / g.pixel)
                        A[i, iy * g.nx + ix] += step * w
            else:
                step = g.pixel * L / abs(D[1])
                for iy in range(g.ny):
                    x = P[0] + (Yc[iy] - P[1]) / D[1] * D[0]
                    for ix in range(g.nx):
                        w = max(0.0, 1.0 - abs(x - Xc[ix]) / g.pixel)
                        A[i, iy * g.nx + ix] += step * w
    return A


@pytest.mark.parametrize("gi", range(len(tiny_geometries())))
def test_dense_matrix_equals_ray_walk(gi):
    g = tiny_geometries()[gi]
    A = dense_A(g)
    assert (A >= 0).all()
    # columns of the walk: A e_k
    W = np.zeros_like(A)
    for k in range(g.d):
        e = np.zeros(g.d)
        e[k] = 1.0
        W[:, k] = oracle.forward(g, e.reshape(g.ny, g.nx)).ravel()
    np.testing.assert_allclose(W, A, rtol=0, atol=1e-11 * max(1.0, A.max()))
    # rows of the scatter: A^T e_i
    T = np.zeros_like(A)
    for i in range(g.n_rays):
        e = np.zeros(g.n_rays)
        e[i] = 1.0
        T[i, :] = oracle.adjoint(g, e.reshape(g.n_views, g.n_bins)).ravel()
    np.testing.assert_allclose(T, A, rtol=0, atol=1e-11 * max(1.0, A.max()))


@pytest.mark.parametrize("n", [8, 11, 32])
def test_axis_aligned_views_give_row_and_column_sums(n):
    """Bins on pixel centres: view 0 sums image rows, view pi/2 sums columns
    (in reverse order of the detector axis)."""
    g = Geometry(beam=0, nx=n, ny=n, n_views=2, n_bins=n, angle_range=np.pi, pixel=1.0)
    x = synth.random_image(n, n, seed=5)
    z = oracle.forward(g, x)
    np.testing.assert_allclose(z[0], x.sum(axis=1), rtol=1e-12)
    np.testing.assert_allclose(z[1], x.sum(axis=0)[::-1], rtol=1e-12)


@pytest.mark.parametrize("beam", [0, 1])
def test_constant_image_gives_support_chord(beam):
    """For x = 1, a ray whose crossings all lie between the first and last
    pixel centre of the cross axis has Joseph value N * pixel / |cos|, the
    length of its chord through the square [-N p/2, N p/2]^2 measured along
    the driving axis."""
    n = 32
    g = Geometry(beam=beam, nx=n, ny=n, n_views=24, n_bins=9, angle0=0.11, angle_range=2 * np.pi,
                 pixel=0.75, bin_pitch=0.6, src_to_center=60.0, src_to_det=90.0)
    z = oracle.forward(g, np.ones((n, n)))
    checked = 0
    for v in range(g.n_views):
        for b in range(g.n_bins):
            P, Q = _two_points(g, v, b)
            D = (Q - P) / np.hypot(*(Q - P))
            drive = 0 if abs(D[0]) >= abs(D[1]) else 1
            # cross coordinates at the first and last driving-axis pixel centres
            c_end = []
            for s in (-(n - 1) / 2 * g.pixel, (n - 1) / 2 * g.pixel):
                lam = (s - P[drive]) / D[drive]
                c_end.append(P[1 - drive] + lam * D[1 - drive])
            lim = (n - 1) / 2 * g.pixel
            if max(abs(c) for c in c_end) <= lim:
                assert z[v, b] == pytest.approx(n * g.pixel / abs(D[drive]), rel=1e-12)
                checked += 1
    assert checked > g.n_views * 3


def _ellipse_line_integral(e: synth.Ellipse, n_vec, s):
    """Analytic line integral of rho * 1{ellipse} along {p : p . n = s}
    (n unit): 2 rho a b sqrt(q - s'^2) / q with q = (a n1')^2 + (b n2')^2,
    n' the normal in the ellipse frame and s' = s - c . n."""
    c, sn = np.cos(e.phi), np.sin(e.phi)
    n1 = n_vec[0] * c + n_vec[1] * sn
    n2 = -n_vec[0] * sn + n_vec[1] * c
    q = (e.a * n1) ** 2 + (e.b * n2) ** 2
    sp = s - (e.cx * n_vec[0] + e.cy * n_vec[1])
    return np.where(q > sp ** 2, 2.0 * e.rho * e.a * e.b * np.sqrt(np.maximum(q - sp ** 2, 0)) / q, 0.0)


def _analytic_sinogram(g: Geometry, ells):
    out = np.zeros((g.n_views, g.n_bins))
    for v in range(g.n_views):
        for b in range(g.n_bins):
            P, Q = _two_points(g, v, b)
            D = (Q - P) / np.hypot(*(Q - P))
            nv = np.array([-D[1], D[0]])
            out[v, b] = sum(_ellipse_line_integral(e, nv, nv @ P) for e in ells)
    return out


@pytest.mark.parametrize("beam", [0, 1])
def test_ellipse_chords_converge(beam):
    """Joseph projections of a finely rasterised ellipse phantom approach the
    analytic line integrals; the error shrinks as pixels shrink."""
    errs = []
    # same physical object (radius-40 field of view), grids of 64 and 256 pixels
    ells = [synth.Ellipse(5.0, -3.0, 22.0, 13.0, 0.4, 0.7), synth.Ellipse(-8.0, 9.0, 7.0, 11.0, 1.1, 0.3)]
    for n in (64, 256):
        pix = 80.0 / n
        g = Geometry(beam=beam, nx=n, ny=n, n_views=16, n_bins=41, angle0=0.05, angle_range=2 * np.pi,
                     pixel=pix, bin_pitch=1.7, src_to_center=150.0, src_to_det=220.0)
        x = synth.rasterize_ellipses(ells, n, n, pixel=pix, supersample=4, clip=False)
        z = oracle.forward(g, x)
        ref = _analytic_sinogram(g, ells)
        errs.append(np.abs(z - ref).mean() / ref.max())
    assert errs[1] < errs[0] / 2.5
    assert errs[1] < 2e-3


@pytest.mark.parametrize("gi", range(len(tiny_geometries())))
def test_adjoint_identity(gi):
    g = tiny_geometries()[gi]
    rng = np.random.default_rng(gi)
    for _ in range(3):
        x = rng.standard_normal((g.ny, g.nx))
        r = rng.standard_normal((g.n_views, g.n_bins))
        lhs = float((oracle.forward(g, x) * r).sum())
        rhs = float((x * oracle.adjoint(g, r)).sum())
        assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)


def test_adjoint_identity_medium():
    g = Geometry(beam=1, nx=96, ny=80, n_views=45, n_bins=131, angle_range=2 * np.pi, bin_pitch=1.5,
                 src_to_center=300.0, src_to_det=450.0)
    x = synth.random_image(96, 80, seed=1)
    r = synth.random_sinogram(45, 131, seed=2)
    lhs = float((oracle.forward(g, x) * r).sum())
    rhs = float((x * oracle.adjoint(g, r)).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("gi", [0, 3, 4])
def test_norm_estimate_matches_svd(gi):
    g = tiny_geometries()[gi]
    lam, it = oracle.norm_estimate(g, max_iters=2000, rtol=1e-13)
    ref = np.linalg.norm(dense_A(g), 2) ** 2
    assert lam == pytest.approx(ref, rel=1e-9)
    assert it < 2000
