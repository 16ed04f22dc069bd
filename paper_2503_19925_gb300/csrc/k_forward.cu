// k_forward.cu -- Joseph forward projector z = A x with the fused
// polychromatic link and residual (Eq. (7), Eq. (8)).
//
// One CTA takes a work unit: up to kFR adjacent rays of one view that share a
// driving axis, one ray per thread.  The unit walks the driving axis in chunks
// of kFC pixel lines; for every chunk the band of the image its rays cross
// (kFHB cross-axis rows, computed on the host) is brought into shared memory
// by one 2D tensor-map copy (cp.async.bulk.tensor) from the padded copy of the
// image read along that axis: x-driven rays read the column-major copy,
// y-driven rays the row-major one.  Copies are double-buffered on two
// mbarriers, so the copy of chunk c + 1 overlaps the samples of chunk c, and
// each thread's two interpolation taps are shared-memory loads.  Every thread
// waits on the mbarrier of its chunk; one CTA barrier per chunk then both
// agrees on the outcome and frees the other buffer for the next copy.  Out-of-range
// parts of a box are zero-filled by the copy, which is the projector's
// zero-outside-the-image rule.  Every mbarrier wait is bounded: on a timeout the
// CTA records EXACT_ERR_TIMEOUT, waits (bounded) for its copy in flight and
// returns.
//
// Cross-axis coordinate: t(j) = A + a + (bh + bl) j is re-anchored at every
// chunk start j0.  The integer part K and the fraction tau0 are formed with an
// exact product split (fmaf); inside the chunk tau = fmaf(bh, j - j0, tau0)
// stays small, so FP32 keeps t to ~1e-6 pixel at any image size (a plain
// fmaf(beta, j, alpha) loses ~3e-5 pixel at 512).
//
// Every ray that samples a chunk walks all kFC of its lines in a fully
// unrolled loop (line offset a compile-time constant, no per-line range test
// or clamp): lines outside the ray's driving range put its crossing more than
// a pixel outside the image, where both taps read zeros, so the sum is the
// same bit for bit as a walk over the range alone.  The band rows of the
// chunk's first and last line are checked once; the row is monotone in the
// line, so that bounds every read.
//
// Link epilogue: r_i = delta_i (Y_i - sum_k c_k 2^(-mu2_k max(z_i, 0))) with
// c_k = I0 sum_w S[w][k] and Y_i = sum_w y[w][i] (F is linear in y, so summing
// the windows first is exact algebra); the per-energy coefficients live in the
// kernel parameter space (uniform access).  The residual leaves the kernel
// already multiplied by the ray's step length, the factor every entry of the
// ray's row of A carries.
//
// The walk itself (forward_unit) is in joseph.cuh, shared with the persistent
// multi-job kernel of k_batch.cu.
#include "joseph.cuh"

namespace exact {

namespace {

template <bool LINK>
__global__ void __launch_bounds__(kFR) k_forward_tma(FwdArgs a, const __grid_constant__ CUtensorMap map_r,
                                                     const __grid_constant__ CUtensorMap map_c,
                                                     const __grid_constant__ LinkCoef coef)
{
    if (a.state && a.state->done) return;
    __shared__ __align__(128) FwdSmem sm;
    __shared__ __align__(8) uint64_t bar[kFStages];
    if (threadIdx.x == 0) {
        for (int q = 0; q < kFStages; ++q) mbar_init(&bar[q]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0u;
    forward_unit<LINK, false>(a, blockIdx.x, &map_r, &map_c, &coef, sm, bar, phase);
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

cudaError_t launch_forward(const FwdArgs &a, bool link, const LinkCoef *coef, const CUtensorMap &map_r,
                           const CUtensorMap &map_c, cudaStream_t s)
{
    if (a.n_units <= 0) return cudaSuccess;
    if (link) {
        k_forward_tma<true><<<a.n_units, kFR, 0, s>>>(a, map_r, map_c, *coef);
    } else {
        LinkCoef none;
        none.mu2[0] = 0.0f;
        none.c[0] = 0.0f;
        k_forward_tma<false><<<a.n_units, kFR, 0, s>>>(a, map_r, map_c, none);
    }
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
