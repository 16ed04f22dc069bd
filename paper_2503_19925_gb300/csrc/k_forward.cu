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
// Link epilogue: r_i = Y_i - sum_k c_k 2^(-mu2_k max(z_i, 0)) with
// c_k = I0 sum_w S[w][k] and Y_i = sum_w y[w][i] (F is linear in y, so summing
// the windows first is exact algebra); the per-energy coefficients live in the
// kernel parameter space (uniform access).
#include "exact_internal.h"

namespace exact {

namespace {

// Sum of the Joseph samples of one ray (without the step length delta).
// T is the arithmetic type (float on the hot path, double in the power
// iteration); t = fma(beta, j, alpha) is the same expression the adjoint uses.
template <typename T, typename R>
__device__ __forceinline__ T joseph_sum(const T *xr, const T *xc, int nx, int ny, long long ldr, long long ldc,
                                        const R &rec)
{
    const int axis = ray_axis(rec.bits);
    const int jlo = ray_jlo(rec.bits), jhi = ray_jhi(rec.bits);
    const T *base = axis ? xr : xc;
    const long long ld = axis ? ldr : ldc;
    const int ncross = axis ? nx : ny;
    const T *row = base + (long long)jlo * ld + kPad;
    T acc = T(0);
    T jf = (T)jlo;
#pragma unroll 4
    for (int j = jlo; j <= jhi; ++j) {
        const T t = fma(rec.beta, jf, rec.alpha);
        const T kf = floor(t);
        const T f = t - kf;
        int k = (int)kf;
        k = min(max(k, -kPad), ncross);
        const T a0 = __ldg(row + k);
        const T a1 = __ldg(row + k + 1);
        acc += fma(f, a1 - a0, a0);
        row += ld;
        jf += T(1);
    }
    return acc;
}

__device__ __forceinline__ float joseph_ray(const ImgF &img, const RayF &rec)
{
    return rec.delta * joseph_sum<float, RayF>(img.xr, img.xc, img.nx, img.ny, img.ldr, img.ldc, rec);
}

__global__ void __launch_bounds__(256) k_forward(FwdArgs a)
{
    if (a.state && a.state->done) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const RayF rec = a.rays[i];
    a.z[i] = joseph_ray(a.img, rec);
}

__global__ void __launch_bounds__(256) k_forward_link(FwdArgs a, const LinkCoef coef)
{
    if (a.state && a.state->done) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const RayF rec = a.rays[i];
    const float z = joseph_ray(a.img, rec);
    const float zp = fmaxf(z, 0.0f);
    float lam = 0.0f;
    for (int k = 0; k < a.K; ++k) lam = fmaf(coef.c[k], exp2f(-coef.mu2[k] * zp), lam);
    a.r[i] = a.Y[i] - lam;
}

// FP64 forward of the power iteration: z = inv_norm * A w, plus per-block
// partial sums of ||z||^2 (fixed order).
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
        z = st->inv_norm * (rec.delta * joseph_sum<double, RayD>(xrd, xcd, nx, ny, ldr, ldc, rec));
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
