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
// each thread's two interpolation taps are shared-memory loads.  Out-of-range
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
// Link epilogue: r_i = delta_i (Y_i - sum_k c_k 2^(-mu2_k max(z_i, 0))) with
// c_k = I0 sum_w S[w][k] and Y_i = sum_w y[w][i] (F is linear in y, so summing
// the windows first is exact algebra); the per-energy coefficients live in the
// kernel parameter space (uniform access).  The residual leaves the kernel
// already multiplied by the ray's step length, the factor every entry of the
// ray's row of A carries.
#include "exact_internal.h"

namespace exact {

namespace {

constexpr unsigned kBoxBytes = kFC * kFHB * sizeof(float);
constexpr int kWaitSpins = 1 << 20;  // bounded mbarrier wait (try_wait also suspends briefly)

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for the given phase parity; true when the phase completed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t addr = smem_u32(bar);
    for (int it = 0; it < kWaitSpins; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// One kFC x kFHB box of the tensor map at (x = padded cross index, y = line).
__device__ __forceinline__ void tma_box(float *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    const uint32_t b = smem_u32(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(kBoxBytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(b)
        : "memory");
}

template <bool LINK>
__global__ void __launch_bounds__(kFR) k_forward_tma(FwdArgs a, const __grid_constant__ CUtensorMap map_r,
                                                     const __grid_constant__ CUtensorMap map_c, const LinkCoef coef)
{
    if (a.state && a.state->done) return;
    __shared__ __align__(128) float buf[2][kFC * kFHB];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_ok;

    const FwdUnit u = a.units[blockIdx.x];
    const int t = threadIdx.x;
    const bool has_ray = t < u.count;
    const long long i = (long long)u.ray0 + t;
    RayF rec = {0.f, 0.f, 0.f, 0.f};
    int bits = 1;  // empty driving range (j_lo = 1 > j_hi = 0)
    if (has_ray) {
        rec = a.rays[i];
        bits = a.bits[i];
    }
    const int jlo = ray_jlo(bits), jhi = ray_jhi(bits);
    const CUtensorMap *map = u.axis ? &map_r : &map_c;
    const int A = (int)rec.A;
    const int *kst = a.kstart + u.koff;

    if (t == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (u.nchunks > 0) tma_box(buf[0], map, kst[0] + kPad, u.jc0 * kFC, &bar[0]);
    }
    __syncthreads();

    float acc = 0.0f;
    for (int c = 0; c < u.nchunks; ++c) {
        if (t == 0) {
            const bool ok = mbar_wait(&bar[c & 1], (uint32_t)(c >> 1) & 1u);
            s_ok = ok ? 1 : 0;
            if (ok && c + 1 < u.nchunks) {
                // the other buffer was last read before the barrier that ended
                // chunk c - 1; order those reads before the async-proxy write
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_box(buf[(c + 1) & 1], map, kst[c + 1] + kPad, (u.jc0 + c + 1) * kFC, &bar[(c + 1) & 1]);
            }
        }
        __syncthreads();
        if (!s_ok) {
            // the copy of chunk c never completed: report, wait (bounded) for
            // it once more so no copy lands after exit, and leave
            if (t == 0) {
                mbar_wait(&bar[c & 1], (uint32_t)(c >> 1) & 1u);
                if (a.err) {
                    a.err->status = EXACT_ERR_TIMEOUT;
                    a.err->done = 1;
                }
            }
            return;
        }
        const int j0 = (u.jc0 + c) * kFC;
        const int ja = max(jlo, j0), jb = min(jhi, j0 + kFC - 1);
        if (ja <= jb) {
            // anchor: t(j0) = K + tau0 with tau0 accurate to FP32 rounding at ~1
            const float jf = (float)j0;
            const float p = rec.bh * jf;
            const float e = fmaf(rec.bh, jf, -p);
            const float P = floorf(p);
            const float tau0 = ((p - P) + rec.a) + fmaf(rec.bl, jf, e);
            // local row = K + floor(tau) - kstart, with the bias of the
            // float-to-int floor folded in
            const int off = A + (int)P - kst[c] - kFloorBias;
            const float *sb = buf[c & 1] + (ja - j0) * kFHB;
            float di = (float)(ja - j0);
#pragma unroll 4
            for (int j = ja; j <= jb; ++j) {
                const float tau = fmaf(rec.bh, di, tau0);
                // floor(tau) for |tau| < 2^22: a round-down add of 1.5 * 2^23
                // leaves floor(tau) in the low mantissa bits
                const float r = __fadd_rd(tau, kFloorMagic);
                const float f = tau - (r - kFloorMagic);
                // the host sized the band with a row of margin; the clamp only
                // keeps a damaged table inside the buffer
                const int row = min(max(off + __float_as_int(r), 0), kFHB - 2);
                const float a0 = sb[row], a1 = sb[row + 1];
                acc += fmaf(f, a1 - a0, a0);
                sb += kFHB;
                di += 1.0f;
            }
        }
        __syncthreads();
    }
    if (!has_ray) return;
    const float delta = a.delta[i];
    const float z = delta * acc;
    if (!LINK) {
        a.z[i] = z;
        return;
    }
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
