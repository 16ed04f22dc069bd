// k_adjoint.cu -- pixel-driven adjoint g = A^T r (the exact transpose of the
// Joseph projector in k_forward.cu) with the fused extragradient epilogue of
// Eq. (11) and the FP64 partial norms of the stopping rule.
//
// One thread owns one pixel (kx, ky) and loops over the views in a fixed
// order, so each output is a fixed-order sum: deterministic, no atomics.  For
// each view it finds the detector bins whose rays can give the pixel a
// nonzero Joseph weight:
//   - an x-driven ray samples column kx, and touches the pixel iff its
//     crossing lies strictly between the points (kx, ky-1) and (kx, ky+1);
//   - a y-driven ray samples row ky, and touches it iff its crossing lies
//     strictly between (kx-1, ky) and (kx+1, ky).
// Projecting the two end points onto the detector (a ratio of affine forms of
// (kx, ky), stored per view) bounds the candidate bins; each candidate's weight
// is then evaluated from the same ray record as the forward walk.  A small margin widens the candidate range; candidates that
// do not touch the pixel get weight 0.
//
// The FP32 weights are formed from the split ray coordinate of k_forward.cu
// (see weight_f); both kernels reproduce the FP64 matrix entries to ~1e-6, so
// the gather is the transpose of the forward walk up to FP32 rounding.
#include "exact_internal.h"

namespace exact {

namespace {

constexpr int TX = 32, TY = 8;
constexpr float kBinEps = 0.01f;

template <bool FAN>
__device__ __forceinline__ void bin_range(float num, float den, float dn, float dd, float c, int n_bins,
                                          int &b0, int &b1)
{
    float u1, u2;
    if (FAN) {
        u1 = __fdividef(num + dn, den + dd);
        u2 = __fdividef(num - dn, den - dd);
    } else {
        u1 = num + dn;
        u2 = num - dn;
    }
    float lo = fminf(u1, u2) + c - kBinEps;
    float hi = fmaxf(u1, u2) + c + kBinEps;
    lo = fminf(fmaxf(lo, -1.0f), (float)n_bins);
    hi = fminf(fmaxf(hi, -1.0f), (float)n_bins);
    b0 = max(0, (int)ceilf(lo));
    b1 = min(n_bins - 1, (int)floorf(hi));
}

// FP32 Joseph weight of ray `rec` at driving index jf for the pixel at cross
// index kc: max(0, 1 - |u|) with u = t(jf) - kc formed from the split
// coordinate (t = A + a + (bh + bl) jf): the product bh*jf is split exactly by
// fmaf, and (A - kc) + bh*jf cancels exactly whenever the ray can touch the
// pixel, so u carries only FP32 rounding at magnitude ~1.
__device__ __forceinline__ float weight_f(const RayF &rec, float jf, float kc)
{
    const float p = rec.bh * jf;
    const float e = fmaf(rec.bh, jf, -p);
    const float u = ((rec.A - kc) + p) + (rec.a + fmaf(rec.bl, jf, e));
    return fmaxf(0.0f, 1.0f - fabsf(u));
}

// FP64 Joseph weight: t = fma(beta, j, alpha), entries (1 - |t - k|)_+.
__device__ __forceinline__ double weight_d(const RayD &rec, double jf, double kc)
{
    const double u = fma(rec.beta, jf, rec.alpha) - kc;
    return fmax(0.0, 1.0 - fabs(u)) * rec.delta;
}

__device__ __forceinline__ float weight_of(const RayF &rec, float jf, float kc) { return weight_f(rec, jf, kc); }
__device__ __forceinline__ double weight_of(const RayD &rec, double jf, double kc) { return weight_d(rec, jf, kc); }

// A^T r at pixel (kx, ky): the fixed-order sum over views, and within a view
// over the candidate bins, of weight * r.  For FP32 r must already carry each
// ray's delta (or `delta` is given); RayD weights include delta.
template <typename T, typename R, bool FAN>
__device__ __forceinline__ T gather_pixel(const R *__restrict__ rays, const ViewRec *__restrict__ views,
                                          const T *__restrict__ r, const float *__restrict__ delta, int n_views,
                                          int n_bins, int kx, int ky)
{
    const float fx = (float)kx, fy = (float)ky;
    const T tx = (T)kx, ty = (T)ky;
    T acc = T(0);
    for (int v = 0; v < n_views; ++v) {
        const ViewRec vr = views[v];
        const long long vb = (long long)v * n_bins;
        const float num = fmaf(vr.n2, fy, fmaf(vr.n1, fx, vr.n0));
        const float den = FAN ? fmaf(vr.d2, fy, fmaf(vr.d1, fx, vr.d0)) : 1.0f;
        if (vr.xb1 > vr.xb0) {  // x-driven rays sample column kx
            int b0, b1;
            bin_range<FAN>(num, den, vr.n2, vr.d2, vr.c, n_bins, b0, b1);
            b0 = max(b0, vr.xb0);
            b1 = min(b1, vr.xb1 - 1);
            for (int b = b0; b <= b1; ++b) {
                const T w = weight_of(rays[vb + b], tx, ty);
                const T rv = delta ? (T)(r[vb + b] * delta[vb + b]) : r[vb + b];
                acc = fma(w, rv, acc);
            }
        }
        if (vr.yb1 > vr.yb0) {  // y-driven rays sample row ky
            int b0, b1;
            bin_range<FAN>(num, den, vr.n1, vr.d1, vr.c, n_bins, b0, b1);
            b0 = max(b0, vr.yb0);
            b1 = min(b1, vr.yb1 - 1);
            for (int b = b0; b <= b1; ++b) {
                const T w = weight_of(rays[vb + b], ty, tx);
                const T rv = delta ? (T)(r[vb + b] * delta[vb + b]) : r[vb + b];
                acc = fma(w, rv, acc);
            }
        }
    }
    return acc;
}

// Fixed-order block sum of two doubles; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double &a, double &b)
{
    __shared__ double sa[TX * TY / 32], sb[TX * TY / 32];
    const int lane = (threadIdx.y * TX + threadIdx.x) & 31;
    const int warp = (threadIdx.y * TX + threadIdx.x) >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (warp == 0 && lane == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < TX * TY / 32; ++w) {
            ta += sa[w];
            tb += sb[w];
        }
        a = ta;
        b = tb;
    }
}

template <int MODE, bool FAN>
__global__ void __launch_bounds__(TX *TY) k_adjoint(AdjArgs a)
{
    if (a.state && a.state->done) return;
    const int kx = blockIdx.x * TX + threadIdx.x;
    const int ky = blockIdx.y * TY + threadIdx.y;
    const bool inside = kx < a.nx && ky < a.ny;
    float g = 0.0f;
    if (inside) g = gather_pixel<float, RayF, FAN>(a.rays, a.views, a.r, a.delta, a.n_views, a.n_bins, kx, ky);

    if (MODE == ADJ_PLAIN) {
        if (inside) a.out[(long long)ky * a.nx + kx] = a.scale * g;
        return;
    }

    // extragradient step from the base iterate, projected onto [lo, hi]
    const long long pr = (long long)ky * a.ldr + kx + kPad;
    const float xb = inside ? a.base_r[pr] : 0.0f;
    // projection onto [lo, hi] that keeps a NaN (so the stopping rule sees it)
    const float step = fmaf(a.scale, g, xb);
    const float xn = inside ? (step < a.lo ? a.lo : (step > a.hi ? a.hi : step)) : 0.0f;
    if (inside) a.out_r[pr] = xn;

    // column-major copy through shared memory: 8 consecutive ky per kx row
    __shared__ float tile[TY][TX + 1];
    tile[threadIdx.y][threadIdx.x] = xn;
    __syncthreads();
    {
        const int l = threadIdx.y * TX + threadIdx.x;
        const int col = l / TY, row = l % TY;
        const int ox = blockIdx.x * TX + col, oy = blockIdx.y * TY + row;
        if (ox < a.nx && oy < a.ny) a.out_c[(long long)ox * a.ldc + oy + kPad] = tile[row][col];
    }

    if (MODE == ADJ_EG_FINAL) {
        if (inside && a.avg && a.iter >= a.avg_from) a.avg[(long long)ky * a.nx + kx] += (double)xn;
        const double dd = (double)xn - (double)xb;
        double s0 = inside ? dd * dd : 0.0;
        double s1 = inside ? (double)xb * (double)xb : 0.0;
        block_sum2(s0, s1);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
            a.partials[2 * blk] = s0;
            a.partials[2 * blk + 1] = s1;
        }
    }
}

// FP64 adjoint of the power iteration: w = A^T z into both padded copies,
// plus per-block partial sums of ||w||^2.
template <bool FAN>
__global__ void __launch_bounds__(TX *TY) k_adjoint_d(const RayD *rays, const ViewRec *views, int n_views,
                                                     int n_bins, int nx, int ny, const double *zd, double *xrd,
                                                     double *xcd, long long ldr, long long ldc,
                                                     double *partials, const DevState *st)
{
    if (st->done) return;
    const int kx = blockIdx.x * TX + threadIdx.x;
    const int ky = blockIdx.y * TY + threadIdx.y;
    const bool inside = kx < nx && ky < ny;
    double w = 0.0;
    if (inside) {
        w = gather_pixel<double, RayD, FAN>(rays, views, zd, nullptr, n_views, n_bins, kx, ky);
        xrd[(long long)ky * ldr + kx + kPad] = w;
        xcd[(long long)kx * ldc + ky + kPad] = w;
    }
    double s0 = w * w, s1 = 0.0;
    block_sum2(s0, s1);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = s0;
}

}  // namespace

int adjoint_blocks(int nx, int ny) { return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY); }

cudaError_t launch_adjoint(const AdjArgs &a, int mode, bool fan, cudaStream_t s)
{
    const dim3 block(TX, TY);
    const dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
    if (fan) {
        if (mode == ADJ_PLAIN) k_adjoint<ADJ_PLAIN, true><<<grid, block, 0, s>>>(a);
        else if (mode == ADJ_EG) k_adjoint<ADJ_EG, true><<<grid, block, 0, s>>>(a);
        else k_adjoint<ADJ_EG_FINAL, true><<<grid, block, 0, s>>>(a);
    } else {
        if (mode == ADJ_PLAIN) k_adjoint<ADJ_PLAIN, false><<<grid, block, 0, s>>>(a);
        else if (mode == ADJ_EG) k_adjoint<ADJ_EG, false><<<grid, block, 0, s>>>(a);
        else k_adjoint<ADJ_EG_FINAL, false><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_d(const RayD *rays, const ViewRec *views, int n_views, int n_bins, int nx, int ny,
                             const double *zd, double *xrd, double *xcd, long long ldr, long long ldc,
                             double *partials, DevState *st, bool fan, cudaStream_t s)
{
    const dim3 block(TX, TY);
    const dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY);
    if (fan)
        k_adjoint_d<true><<<grid, block, 0, s>>>(rays, views, n_views, n_bins, nx, ny, zd, xrd, xcd, ldr, ldc,
                                                 partials, st);
    else
        k_adjoint_d<false><<<grid, block, 0, s>>>(rays, views, n_views, n_bins, nx, ny, zd, xrd, xcd, ldr, ldc,
                                                  partials, st);
    return cudaGetLastError();
}

}  // namespace exact
