/*
 * exact_oracle.c -- plain FP64 CPU oracle for the EXACT hot path.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library.  It shares no code with the CUDA path
 * (paper_2503_19925_gb300/csrc) and the CUDA path never calls it.
 *
 * Everything here is written for clarity, not speed: FP64 throughout, fixed
 * loop orders, the adjoint as a ray-driven scatter (the plain transpose of the
 * forward walk), the polychromatic link evaluated literally per window.
 * Paper: "Extragradient algorithm for computed tomography" (EXACT).
 *
 * Projector discretisation.  The paper only says that A is a nonnegative
 * matrix derived from the Radon transform (Sec. 1, notation list; Sec. 2.1).
 * We use Joseph's ray-driven method with these conventions:
 *   - pixel (ix, iy) of an nx x ny image (stored x[iy*nx + ix]) has its centre
 *     at X(ix) = (ix - (nx-1)/2) * pixel, Y(iy) = (iy - (ny-1)/2) * pixel;
 *   - view v has angle th = angle0 + v * angle_range / n_views (end point
 *     excluded), source-side unit vector es = (cos th, sin th) and detector
 *     axis eu = (-sin th, cos th); bin b sits at
 *     u_b = (b - (n_bins-1)/2) * bin_pitch + det_offset along eu;
 *   - parallel beam: the ray passes through u_b * eu with direction -es;
 *   - fan beam (flat detector): the ray goes from the source S = R_s * es to
 *     the detector point (R_s - R_d) * es + u_b * eu;
 *   - the driving axis is x when |dir_x| >= |dir_y| (ties drive x), else y;
 *     at every pixel centre line j of the driving axis the ray's crossing has
 *     cross-axis index coordinate t_j = alpha + beta * j, and the sample is the
 *     linear interpolation between the two nearest pixel centres, pixels
 *     outside the image counting as 0;
 *   - the sample step is delta = pixel / |dir_drive|, so
 *     A[i][pixel(j,k)] = delta * max(0, 1 - |t_j - k|).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int beam;               /* 0 parallel, 1 fan (flat detector) */
    int nx, ny;
    double pixel;
    int n_views;
    double angle0, angle_range;
    int n_bins;
    double bin_pitch, det_offset;
    double src_to_center, src_to_det;
} ora_geometry;

/* A ray: a point p on it and a unit direction d. */
static void ray_line(const ora_geometry *g, int v, int b,
                     double *px, double *py, double *dx, double *dy)
{
    double th = g->angle0 + (double)v * g->angle_range / (double)g->n_views;
    double c = cos(th), s = sin(th);
    double u = ((double)b - 0.5 * (double)(g->n_bins - 1)) * g->bin_pitch + g->det_offset;
    if (g->beam == 0) {
        *px = -s * u;
        *py = c * u;
        *dx = -c;
        *dy = -s;
    } else {
        double sx = g->src_to_center * c, sy = g->src_to_center * s;
        double qx = (g->src_to_center - g->src_to_det) * c - s * u;
        double qy = (g->src_to_center - g->src_to_det) * s + c * u;
        double ex = qx - sx, ey = qy - sy;
        double len = sqrt(ex * ex + ey * ey);
        *px = sx;
        *py = sy;
        *dx = ex / len;
        *dy = ey / len;
    }
}

/* Joseph parameters of ray (v, b): driving axis (0 = x, 1 = y), the
 * cross-axis index coordinate t_j = alpha + beta * j at driving index j, and
 * the step length delta. */
static void ray_joseph(const ora_geometry *g, int v, int b,
                       int *axis, double *alpha, double *beta, double *delta)
{
    double px, py, dx, dy;
    ray_line(g, v, b, &px, &py, &dx, &dy);
    double x0 = -0.5 * (double)(g->nx - 1) * g->pixel;
    double y0 = -0.5 * (double)(g->ny - 1) * g->pixel;
    if (fabs(dx) >= fabs(dy)) {
        /* crossing with the column line x = X(j): y = py + (X(j) - px) dy/dx */
        *axis = 0;
        *beta = dy / dx;
        *alpha = (py + (x0 - px) * (dy / dx)) / g->pixel + 0.5 * (double)(g->ny - 1);
        *delta = g->pixel / fabs(dx);
    } else {
        *axis = 1;
        *beta = dx / dy;
        *alpha = (px + (y0 - py) * (dx / dy)) / g->pixel + 0.5 * (double)(g->nx - 1);
        *delta = g->pixel / fabs(dy);
    }
}

int ora_num_rays(const ora_geometry *g) { return g->n_views * g->n_bins; }

/* Ray table (for inspection by tests). */
void ora_rays(const ora_geometry *g, int *axis, double *alpha, double *beta, double *delta)
{
    for (int v = 0; v < g->n_views; ++v)
        for (int b = 0; b < g->n_bins; ++b) {
            long i = (long)v * g->n_bins + b;
            ray_joseph(g, v, b, &axis[i], &alpha[i], &beta[i], &delta[i]);
        }
}

/* Value of pixel (drive index j, cross index k) for a ray with the given
 * driving axis; 0 outside the image. */
static double pix(const ora_geometry *g, const double *x, int axis, long j, double kf)
{
    long nc = axis == 0 ? g->ny : g->nx;
    if (kf < 0.0 || kf >= (double)nc) return 0.0;
    long k = (long)kf;
    return axis == 0 ? x[k * g->nx + j] : x[j * g->nx + k];
}

/* z = A x: the projection <a_i, x> of Eq. (5), one Joseph walk per ray. */
void ora_forward(const ora_geometry *g, const double *x, double *z)
{
    long n = (long)g->n_views * g->n_bins;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        int v = (int)(i / g->n_bins), b = (int)(i % g->n_bins);
        int axis;
        double alpha, beta, delta;
        ray_joseph(g, v, b, &axis, &alpha, &beta, &delta);
        long nd = axis == 0 ? g->nx : g->ny;
        double sum = 0.0;
        for (long j = 0; j < nd; ++j) {
            double t = alpha + beta * (double)j;
            double k0 = floor(t);
            double f = t - k0;
            sum += (1.0 - f) * pix(g, x, axis, j, k0) + f * pix(g, x, axis, j, k0 + 1.0);
        }
        z[i] = delta * sum;
    }
}

/* g = A^T r as a ray-driven scatter: every sample of every ray adds its two
 * interpolation weights times r_i into the two pixels it touched.  Serial, in
 * ray order, so the result does not depend on the thread count. */
void ora_adjoint(const ora_geometry *g, const double *r, double *out)
{
    long n = (long)g->n_views * g->n_bins;
    memset(out, 0, sizeof(double) * (size_t)g->nx * (size_t)g->ny);
    for (long i = 0; i < n; ++i) {
        int v = (int)(i / g->n_bins), b = (int)(i % g->n_bins);
        int axis;
        double alpha, beta, delta;
        ray_joseph(g, v, b, &axis, &alpha, &beta, &delta);
        long nd = axis == 0 ? g->nx : g->ny;
        long nc = axis == 0 ? g->ny : g->nx;
        for (long j = 0; j < nd; ++j) {
            double t = alpha + beta * (double)j;
            double k0 = floor(t);
            double f = t - k0;
            for (int q = 0; q < 2; ++q) {
                double kf = k0 + q;
                double w = q == 0 ? 1.0 - f : f;
                if (kf < 0.0 || kf >= (double)nc) continue;
                long k = (long)kf;
                long p = axis == 0 ? k * g->nx + j : j * g->nx + k;
                out[p] += delta * w * r[i];
            }
        }
    }
}

/* h(t) for window w: sum_k S[w][k] exp(-mu_k max(t, 0)), Eq. (7), with the
 * window's intensity folded into S (Sec. 1, Eq. (2)), for a ray that may also
 * cross M known materials (Appendix A.1, single-material recovery against a
 * known background): their projections p[m * stride] attenuate energy k by
 * exp(-mu_bg[m][k] p_m) on top of the unknown material, i.e. Eq. (1) with the
 * known terms moved into the ray's effective intensity and spectrum. */
double ora_h_bg(double t, int K, const double *S_w, const double *mu, int M, const double *mu_bg,
                const double *p, long stride)
{
    double tp = t > 0.0 ? t : 0.0;
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        double e = mu[k] * tp;
        for (int m = 0; m < M; ++m) e += mu_bg[m * K + k] * p[m * stride];
        s += S_w[k] * exp(-e);
    }
    return s;
}

double ora_h(double t, int K, const double *S_w, const double *mu)
{
    return ora_h_bg(t, K, S_w, mu, 0, NULL, NULL, 0);
}

/* Expected counts lam[w][i] = I0 h_w(z_i) (Eq. (2) with one material), with
 * an optional known background (M materials, projections p[m][i]). */
void ora_expected_counts_bg(long n, const double *z, int W, int K, const double *S, const double *mu, double I0,
                            int M, const double *mu_bg, const double *p, double *lam)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i)
        for (int w = 0; w < W; ++w)
            lam[(long)w * n + i] = I0 * ora_h_bg(z[i], K, S + (long)w * K, mu, M, mu_bg, p + i, n);
}

void ora_expected_counts(long n, const double *z, int W, int K, const double *S,
                         const double *mu, double I0, double *lam)
{
    ora_expected_counts_bg(n, z, W, K, S, mu, I0, 0, NULL, NULL, lam);
}

/* Residual r_i = sum_w (y[w][i] - I0 h_w(z_i)): the bracket of Eq. (8), every
 * (window, ray) pair a measurement with the ray's vector a_i. */
void ora_residual_bg(long n, const double *z, int W, int K, const double *S, const double *mu, double I0, int M,
                     const double *mu_bg, const double *p, const double *y, double *r)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int w = 0; w < W; ++w)
            acc += y[(long)w * n + i] - I0 * ora_h_bg(z[i], K, S + (long)w * K, mu, M, mu_bg, p + i, n);
        r[i] = acc;
    }
}

void ora_residual(long n, const double *z, int W, int K, const double *S,
                  const double *mu, double I0, const double *y, double *r)
{
    ora_residual_bg(n, z, W, K, S, mu, I0, 0, NULL, NULL, y, r);
}

/* F(x) = (1/m) sum_{w,i} (y_{w,i} - I0 h_w(<a_i,x>)) a_i with m = W * n, Eq. (8).
 * z and r are caller-provided scratch of n entries. */
void ora_operator_bg(const ora_geometry *g, const double *x, int W, int K, const double *S, const double *mu,
                     double I0, int M, const double *mu_bg, const double *p, const double *y, double *F,
                     double *z, double *r)
{
    long n = (long)g->n_views * g->n_bins;
    long d = (long)g->nx * g->ny;
    ora_forward(g, x, z);
    ora_residual_bg(n, z, W, K, S, mu, I0, M, mu_bg, p, y, r);
    ora_adjoint(g, r, F);
    double inv_m = 1.0 / ((double)W * (double)n);
    for (long q = 0; q < d; ++q) F[q] *= inv_m;
}

void ora_operator(const ora_geometry *g, const double *x, int W, int K, const double *S,
                  const double *mu, double I0, const double *y, double *F,
                  double *z, double *r)
{
    ora_operator_bg(g, x, W, K, S, mu, I0, 0, NULL, NULL, y, F, z, r);
}

/* Projection onto the box [lo, hi]^d; lo = 0, hi = +inf is the projection onto
 * the nonnegative orthant of Sec. 3.1. */
static double clampd(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Projected extragradient, Eq. (11):
 *   x_{t+1/2} = P(x_t - eta F(x_t)),  x_{t+1} = P(x_t - eta F(x_{t+1/2})).
 * x holds x_1 on entry and the last iterate on exit.  After each iteration
 * rel_res = ||x_{t+1} - x_t|| / max(||x_t||, 1e-30) is stored in hist[t] (if
 * hist is not NULL); when tol > 0 and check_every > 0 the loop stops after the
 * first iteration t+1 that is a multiple of check_every with rel_res <= tol.
 * If avg is not NULL it receives the mean of the iterates x_{t+1} for
 * t = floor(iters/2) .. T-1, T the number of iterations run (the last
 * ceil(iters/2) iterates when the loop runs to the end; the last iterate if it
 * stopped before iters/2).  Returns T. */
int ora_solve_bg(const ora_geometry *g, int W, int K, const double *S, const double *mu, double I0, int M,
                 const double *mu_bg, const double *p, const double *y, double eta, int iters, double lo,
                 double hi, double tol, int check_every, double *x, double *hist, double *avg)
{
    long n = (long)g->n_views * g->n_bins;
    long d = (long)g->nx * g->ny;
    double *F = malloc(sizeof(double) * d);
    double *xh = malloc(sizeof(double) * d);
    double *xn = malloc(sizeof(double) * d);
    double *z = malloc(sizeof(double) * n);
    double *r = malloc(sizeof(double) * n);
    double *acc = avg ? calloc((size_t)d, sizeof(double)) : NULL;
    int done = 0;
    int t_avg0 = iters / 2;
    long n_avg = 0;
    for (int t = 0; t < iters; ++t) {
        ora_operator_bg(g, x, W, K, S, mu, I0, M, mu_bg, p, y, F, z, r);
        for (long q = 0; q < d; ++q) xh[q] = clampd(x[q] - eta * F[q], lo, hi);
        ora_operator_bg(g, xh, W, K, S, mu, I0, M, mu_bg, p, y, F, z, r);
        for (long q = 0; q < d; ++q) xn[q] = clampd(x[q] - eta * F[q], lo, hi);
        double num = 0.0, den = 0.0;
        for (long q = 0; q < d; ++q) {
            double e = xn[q] - x[q];
            num += e * e;
            den += x[q] * x[q];
        }
        double rel = sqrt(num) / fmax(sqrt(den), 1e-30);
        if (hist) hist[t] = rel;
        memcpy(x, xn, sizeof(double) * d);
        if (acc && t >= t_avg0) {
            for (long q = 0; q < d; ++q) acc[q] += x[q];
            ++n_avg;
        }
        done = t + 1;
        if (tol > 0.0 && check_every > 0 && (t + 1) % check_every == 0 && rel <= tol) break;
    }
    if (avg) {
        for (long q = 0; q < d; ++q) avg[q] = n_avg > 0 ? acc[q] / (double)n_avg : x[q];
        free(acc);
    }
    free(F); free(xh); free(xn); free(z); free(r);
    return done;
}

int ora_solve(const ora_geometry *g, int W, int K, const double *S, const double *mu,
              double I0, const double *y, double eta, int iters, double lo, double hi,
              double tol, int check_every, double *x, double *hist, double *avg)
{
    return ora_solve_bg(g, W, K, S, mu, I0, 0, NULL, NULL, y, eta, iters, lo, hi, tol, check_every, x, hist,
                        avg);
}

/* Power iteration for ||A||_op^2 = lambda_max(A^T A) (the quantity behind
 * lambda_max(Sigma) of Theorem 2 and the Lipschitz bound of Sec. 4.2):
 * v_1 = 1/sqrt(d); lam_k = ||A v_k||^2 (Rayleigh quotient of A^T A at the unit
 * vector v_k); v_{k+1} = A^T A v_k / ||A^T A v_k||.  Stops when
 * |lam_k - lam_{k-1}| <= rtol * lam_k (rtol > 0) or after max_iters.  Returns lam. */
double ora_norm_estimate(const ora_geometry *g, int max_iters, double rtol, int *iters_done)
{
    long n = (long)g->n_views * g->n_bins;
    long d = (long)g->nx * g->ny;
    double *v = malloc(sizeof(double) * d);
    double *w = malloc(sizeof(double) * d);
    double *z = malloc(sizeof(double) * n);
    for (long p = 0; p < d; ++p) v[p] = 1.0 / sqrt((double)d);
    double lam = 0.0, prev = 0.0;
    int it = 0;
    for (it = 1; it <= max_iters; ++it) {
        ora_forward(g, v, z);
        lam = 0.0;
        for (long i = 0; i < n; ++i) lam += z[i] * z[i];
        ora_adjoint(g, z, w);
        double nw = 0.0;
        for (long p = 0; p < d; ++p) nw += w[p] * w[p];
        nw = sqrt(nw);
        if (nw == 0.0) break;
        for (long p = 0; p < d; ++p) v[p] = w[p] / nw;
        if (it > 1 && rtol > 0.0 && fabs(lam - prev) <= rtol * lam) break;
        prev = lam;
    }
    if (iters_done) *iters_done = it > max_iters ? max_iters : it;
    free(v); free(w); free(z);
    return lam;
}
