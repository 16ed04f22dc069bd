// k_forward.cu -- Joseph forward projector z = A x with the fused
// polychromatic link and residual (Eq. (7), Eq. (8)).
//
// One thread walks one ray.  Consecutive threads take consecutive detector
// bins of one view, so at a given driving index j the lanes of a warp read
// neighbouring cross-axis pixels of the same image line: x-driven rays read the
// column-major copy, y-driven rays the row-major copy, and each lane's two
// interpolation taps sit next to each other.  Both copies carry kPad zero
// columns on each side, so the taps need no bounds test; the per-ray driving
// range [j_lo, j_hi] (computed on the host) leaves out samples that cannot
// touch the image.  The image (1 MB at 512^2) stays in L1/L2.
//
// Cross-axis coordinate: t(j) = A + a + (bh + bl) j is re-anchored every
// kChunk samples.  At the anchor j0 the integer part K and the fraction tau0
// are formed with an exact product split (fmaf), then inside the chunk
// tau = fmaf(bh, j - j0, tau0) stays below ~kChunk in magnitude, so FP32 keeps
// t to ~1e-6 pixel even for 16k-pixel images (a plain fmaf(beta, j, alpha)
// loses ~3e-5 pixel at 512).
//
// Link epilogue: r_i = delta_i (Y_i - sum_k c_k 2^(-mu2_k max(z_i, 0))) with
// c_k = I0 sum_w S[w][k] and Y_i = sum_w y[w][i] (F is linear in y, so summing
// the windows first is exact algebra); the per-energy coefficients live in the
// kernel parameter space (uniform access).  The residual leaves the kernel
// already multiplied by the ray's step length, the factor every entry of the
// ray's row of A carries.
#include "exact_internal.h"

namespace exact {

namespace {

constexpr int kChunk = 32;

// Sum of the Joseph samples of one ray (without the step length delta).
// Bounds: the host range [j_lo, j_hi] keeps the exact crossing t(j) inside
// (-1.5, n_cross + 0.5) and the FP32 evaluation below is within 1e-5 of it,
// so k0 = floor(t) lies in [-2, n_cross] and the taps k0, k0 + 1 stay inside the
// padded row [-kPad, n_cross + kPad - 1]; exact_plan_create re-checks this for
// every chunk anchor and chunk end with the same FP32 operations.
__device__ __forceinline__ float joseph_sum_f(const ImgF &img, const RayF rec, int bits)
{
    const int axis = ray_axis(bits);
    const int jlo = ray_jlo(bits), jhi = ray_jhi(bits);
    const float *__restrict__ base = (axis ? img.xr : img.xc) + kPad;
    const int ld = (int)(axis ? img.ldr : img.ldc);
    const int A = (int)rec.A;
    float acc = 0.0f;
    for (int j0 = jlo; j0 <= jhi; j0 += kChunk) {
        // anchor: t(j0) = K + tau0 with tau0 accurate to FP32 rounding at ~1
        const float jf = (float)j0;
        const float p = rec.bh * jf;
        const float e = fmaf(rec.bh, jf, -p);
        const float P = floorf(p);
        const float tau0 = ((p - P) + rec.a) + fmaf(rec.bl, jf, e);
        // element offset of the row start plus K, minus the bias of the
        // float-to-int trick below
        int off = j0 * ld + A + (int)P - kFloorBias;
        const int cnt = min(kChunk, jhi - j0 + 1);
        float di = 0.0f;
#pragma unroll 4
        for (int i = 0; i < cnt; ++i) {
            const float tau = fmaf(rec.bh, di, tau0);
            // floor(tau) for |tau| < 2^22: round-down add of 1.5 * 2^23 leaves
            // floor(tau) in the low mantissa bits
            const float r = __fadd_rd(tau, kFloorMagic);
            const float f = tau - (r - kFloorMagic);
            const int idx = off + __float_as_int(r);
            const float a0 = __ldg(base + idx);
            const float a1 = __ldg(base + idx + 1);
            acc += fmaf(f, a1 - a0, a0);
            off += ld;
            di += 1.0f;
        }
    }
    return acc;
}

__global__ void __launch_bounds__(256, 8) k_forward(FwdArgs a)
{
    if (a.state && a.state->done) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    a.z[i] = a.delta[i] * joseph_sum_f(a.img, a.rays[i], a.bits[i]);
}

__global__ void __launch_bounds__(256, 8) k_forward_link(FwdArgs a, const LinkCoef coef)
{
    if (a.state && a.state->done) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const float delta = a.delta[i];
    const float z = delta * joseph_sum_f(a.img, a.rays[i], a.bits[i]);
    const float zp = fmaxf(z, 0.0f);
    float lam = 0.0f;
    for (int k = 0; k < a.K; ++k) lam = fmaf(coef.c[k], exp2f(-coef.mu2[k] * zp), lam);
    a.r[i] = delta * (a.Y[i] - lam);
}

// FP64 forward of the power iteration: z = inv_norm * A w, plus per-block
// partial sums of ||z||^2 (fixed order).  t(j) = fma(beta, j, alpha) in double.
__global__ void __launch_bounds__(256) k_forward_d(const RayD *rays, long long n, const double *xrd,
                                                   const double *xcd, int nx, int ny, long long ldr,
                                                   long long ldc, double *zd, double *partials,
                                                   const DevState *st)
{
    if (st->done) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double z = 0.0;
    if (i < n) {
        const RayD rec = rays[i];
        const int axis = ray_axis(rec.bits);
        const int jlo = ray_jlo(rec.bits), jhi = ray_jhi(rec.bits);
        const double *row = (axis ? xrd : xcd) + (long long)jlo * (axis ? ldr : ldc) + kPad;
        const long long ld = axis ? ldr : ldc;
        const int ncross = axis ? nx : ny;
        double acc = 0.0;
        for (int j = jlo; j <= jhi; ++j) {
            const double t = fma(rec.beta, (double)j, rec.alpha);
            const double kf = floor(t);
            const double f = t - kf;
            int k = (int)kf;
            k = min(max(k, -kPad), ncross);
            const double a0 = row[k], a1 = row[k + 1];
            acc += fma(f, a1 - a0, a0);
            row += ld;
        }
        z = st->inv_norm * (rec.delta * acc);
        zd[i] = z;
    }
    double s = z * z;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double sw[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sw[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sw[w];
        partials[blockIdx.x] = t;
    }
}

}  // namespace

int forward_d_blocks(long long n) { return (int)((n + 255) / 256); }

cudaError_t launch_forward(const FwdArgs &a, bool link, const LinkCoef *coef, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    const int threads = 256;
    const unsigned blocks = (unsigned)((a.n + threads - 1) / threads);
    if (link)
        k_forward_link<<<blocks, threads, 0, s>>>(a, *coef);
    else
        k_forward<<<blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_forward_d(const RayD *rays, long long n, const double *xrd, const double *xcd, int nx,
                             int ny, long long ldr, long long ldc, double *zd, double *partials,
                             DevState *st, cudaStream_t s)
{
    k_forward_d<<<forward_d_blocks(n), 256, 0, s>>>(rays, n, xrd, xcd, nx, ny, ldr, ldc, zd, partials, st);
    return cudaGetLastError();
}

}  // namespace exact
