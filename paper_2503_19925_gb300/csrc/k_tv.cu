// k_tv.cu -- projection onto X = {x : ||x||_TV <= tau} ∩ [lo, hi]^d, the
// feasible set of the experiments of Sec. 3.1 (there lo = 0, hi = +inf).
//
// Dykstra's alternating projections between the TV ball X1 and the box X2, in
// the paper's order:
//   y_k = P_X1(z_k + p_k),  p_{k+1} = z_k + p_k - y_k,
//   z_{k+1} = P_X2(y_k + q_k),  q_{k+1} = y_k + q_k - z_{k+1},
// until ||z_{k+1} - z_k|| <= tol_dykstra.  P_X1(w) is the TV-regularised point
// argmin_x ||x - w||^2 + lam ||x||_TV with lam found by bisection until
// | ||x||_TV - tau | <= tol_tv (the identity when ||w||_TV <= tau already).
// The regularised problem is the ROF problem with theta = lam / 2, solved by
// the fast gradient projection method (FISTA on the dual
// min_{|p_ij| <= 1} 1/2 ||w + theta div p||^2, step 1/(8 theta)), the dual
// carried from one solve to the next.  TV is isotropic with forward
// differences, zero past the last row / column.
//
// All of it runs as one persistent cooperative launch: every CTA owns a
// grid-stride share of the pixels, phases are separated by a grid barrier
// (bounded spin: on a timeout the kernel records EXACT_ERR_TIMEOUT and
// returns; the dual steps run kTvK at a time between barriers, see
// fgp_block), and every decision (bisection branch, stop tests) is taken by all
// CTAs on the same FP64 sum, reduced in a fixed order, so the run is
// deterministic.  Pixel arrays are FP32; data rewritten during the launch is
// read through L2 (__ldcg), since L1 is not coherent across CTAs.
#include "exact_internal.h"

#include <math.h>
#include <string.h>

namespace exact {

namespace {

constexpr int kTvThreads = 384;  // 8 rows x 48 columns of a dual-step region
constexpr long long kTvBarrierSpins = 1LL << 22;

struct TvArgs {
    int nx, ny;
    long long d;
    const float *z;
    float *out;            // [ny][nx] result, or null
    float *out_r, *out_c;  // padded row- / column-major copies of the result, or null
    long long ldr, ldc;
    const float *old_r;    // padded row-major previous iterate: partial norms of the solve, or null
    double *norm_part;     // [kPartStride * grid] when old_r is set
    double *avg;           // running-average rule: FP64 window sum (null hist: off)
    float *hist;
    int hist_put, hist_drop;
    double inv_m, inv_m_prev;
    float *zk, *pk, *qk, *w, *xt;
    float *dual[8];        // px, py, rx, ry and their second buffers
    double *part;          // [2][grid] FP64 partial sums
    unsigned *bar;         // [0] arrivals, [1] generation
    long long bar_polls;   // polls before a barrier wait gives up
    int *err;              // status word (EXACT_ERR_TIMEOUT on a barrier timeout)
    int *done;             // solve path: set with err on a timeout, and checked on entry
    double *lam_io;        // in: starting lam (<= 0: 1); out: last lam
    int *stats;            // out: [0] Dykstra rounds, [1] regularised solves
    double tau, tol_tv, tol_dyk;
    int fgp_iters, max_bisect, max_dyk;
    float lo, hi;
    int fixed_lam;         // proximal mode: one regularised solve with lam, no constraint
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int *p)
{
    return *reinterpret_cast<const volatile int *>(p);
}

// Grid-wide barrier with a bounded wait.  Returns false (uniformly within the
// CTA) if it gave up; the status word then holds EXACT_ERR_TIMEOUT.
__device__ bool grid_barrier(unsigned *bar, int *err, int *done, long long polls)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = ld_acquire_u32(bar + 1);
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (ld_acquire_u32(bar + 1) == gen) {
                if (++spins > polls || ld_volatile_i32(err) != 0) {
                    ok = 0;
                    atomicCAS(err, 0, (int)EXACT_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        if (!ok && done) atomicExch(done, 1);
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Fixed-order CTA sum of one double per thread (result valid in every thread):
// the entries past the largest power of two kTvPow2 are folded in first.
constexpr int kTvPow2 = 256;
static_assert(kTvThreads >= kTvPow2 && kTvThreads <= 2 * kTvPow2, "one fold step");

__device__ double block_sum(double v)
{
    __shared__ double s[kTvThreads];
    s[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < kTvThreads - kTvPow2) s[threadIdx.x] += s[threadIdx.x + kTvPow2];
    __syncthreads();
    for (int h = kTvPow2 / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    const double r = s[0];
    __syncthreads();
    return r;
}

// Grid sum of one double per thread: CTA partials to slot `slot`, a barrier,
// then every CTA adds all partials in the same order.  ok = false on timeout.
__device__ double grid_sum(const TvArgs &a, double v, int slot, bool &ok)
{
    const double b = block_sum(v);
    if (threadIdx.x == 0) a.part[(long long)slot * gridDim.x + blockIdx.x] = b;
    ok = grid_barrier(a.bar, a.err, a.done, a.bar_polls);
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kTvThreads)
        s += __ldcg(a.part + (long long)slot * gridDim.x + i);
    return block_sum(s);
}

// Row and column of flat pixel index q (32-bit division while q fits).
__device__ __forceinline__ int tv_row(long long q, int nx)
{
    return q <= 0x7fffffffLL ? (int)q / nx : (int)(q / nx);
}

__device__ __forceinline__ int tv_col(long long q, int nx)
{
    return q <= 0x7fffffffLL ? (int)q % nx : (int)(q % nx);
}

// Isotropic TV term of pixel (i, j) of image v.
__device__ __forceinline__ double tv_term(const float *v, int i, int j, int nx, int ny)
{
    const long long q = (long long)i * nx + j;
    const float c = __ldcg(v + q);
    const float gx = j < nx - 1 ? __ldcg(v + q + 1) - c : 0.0f;
    const float gy = i < ny - 1 ? __ldcg(v + q + nx) - c : 0.0f;
    return sqrt((double)gx * gx + (double)gy * gy);
}

// x = w + theta div r at pixel (i, j).
__device__ __forceinline__ float prox_x(const float *w, const float *rx, const float *ry, float theta, int i, int j,
                                        int nx, int ny)
{
    const long long q = (long long)i * nx + j;
    float dv = 0.0f;
    if (j < nx - 1) dv += __ldcg(rx + q);
    if (j > 0) dv -= __ldcg(rx + q - 1);
    if (i < ny - 1) dv += __ldcg(ry + q);
    if (i > 0) dv -= __ldcg(ry + q - nx);
    return fmaf(theta, dv, __ldcg(w + q));
}

// Up to kTvK dual steps of the fast gradient projection method between two
// grid barriers (temporal blocking).  A CTA stages a kTvT x kTvT tile of the
// image with a halo of kTvK pixels (w, r and p) and runs the steps on the whole
// staged region: every step needs r at distance one, so the garbage that
// enters from the region's edge moves in by one pixel per step and the tile
// itself stays exact; the tile's new p and r are then written to the second
// buffers.  Per pixel the arithmetic is that of one step over the whole image,
// so the result does not depend on kTvK.
//
// Thread (tr, c) of the CTA owns region column c and rows tr + kTvRows m
// (m < kTvM); its w, r, p and x stay in registers, and only r and x, which
// the neighbours read, go through shared memory.  The boundary rule needs no
// branch in the divergence: r_x is zero at the last image column and r_y at
// the last row (their gradient components are zero there, so they keep the
// zero every dual starts with, and p carried between solves keeps it too),
// and every position outside the image is staged as zero with its gradient
// components masked, so the terms the rule drops are exact zeros.
// The shared arrays are flat with row stride kTvR (= 16 mod 32 words, no bank
// conflicts across the two rows a warp touches); r has one leading pad row and
// column, x one trailing (zeroed once per launch, never written): region-edge
// reads land on the pad or on another edge position, and feed only the
// garbage ring.
constexpr int kTvT = 32, kTvK = 8, kTvR = kTvT + 2 * kTvK;
constexpr int kTvRows = kTvThreads / kTvR;  // rows of the region per pass of the CTA
constexpr int kTvM = kTvR / kTvRows;        // region positions per thread
static_assert(kTvRows * kTvR == kTvThreads && kTvM * kTvRows == kTvR, "threads tile the region");

struct TvSmem {
    float rx[(kTvR + 1) * kTvR + 1];  // r_x at (li, lj): [(li + 1) kTvR + lj + 1], li, lj >= -1
    float ry[(kTvR + 1) * kTvR + 1];
    float x[(kTvR + 1) * kTvR + 1];   // x at (li, lj): [li kTvR + lj], li, lj <= kTvR
};

__device__ __forceinline__ int tv_ri(int li, int lj) { return (li + 1) * kTvR + lj + 1; }

__device__ void fgp_block(const TvArgs &a, TvSmem &sm, const float *rxg, const float *ryg, const float *pxg,
                          const float *pyg, float *px2, float *py2, float *rx2, float *ry2, float theta, float step,
                          double &t, int nsteps)
{
    const int nx = a.nx, ny = a.ny;
    const int tiles_x = (nx + kTvT - 1) / kTvT, tiles = tiles_x * ((ny + kTvT - 1) / kTvT);
    // momentum of the fast gradient method, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
    // and beta_k = (t_k - 1) / t_{k+1}, in FP64 by one thread (FP64 runs at a
    // small fraction of the FP32 rate) and shared with the CTA
    __shared__ float s_beta[kTvK];
    __shared__ double s_t;
    if (threadIdx.x == 0) {
        double tt = t;
        for (int k = 0; k < nsteps; ++k) {
            const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tt * tt));
            s_beta[k] = (float)((tt - 1.0) / tn);
            tt = tn;
        }
        s_t = tt;
    }
    __syncthreads();
    const int tr = threadIdx.x / kTvR, lj = threadIdx.x - tr * kTvR;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int i0 = (tile / tiles_x) * kTvT - kTvK, j0 = (tile % tiles_x) * kTvT - kTvK;  // region origin
        const int gj = j0 + lj;
        const bool jin = gj >= 0 && gj < nx;
        const bool fx = gj >= 0 && gj < nx - 1;  // x-gradient kept (forward difference inside the image)
        float w[kTvM], rx[kTvM], ry[kTvM], px[kTvM], py[kTvM], xv[kTvM];
        unsigned fy = 0u;  // bit m: y-gradient kept at row tr + kTvRows m
#pragma unroll
        for (int m = 0; m < kTvM; ++m) {
            const int li = tr + kTvRows * m, gi = i0 + li;
            if (gi >= 0 && gi < ny - 1) fy |= 1u << m;
            w[m] = rx[m] = ry[m] = px[m] = py[m] = 0.0f;
            if (jin && gi >= 0 && gi < ny) {
                const long long q = (long long)gi * nx + gj;
                w[m] = __ldcg(a.w + q);
                rx[m] = __ldcg(rxg + q);
                ry[m] = __ldcg(ryg + q);
                px[m] = __ldcg(pxg + q);
                py[m] = __ldcg(pyg + q);
            }
            sm.rx[tv_ri(li, lj)] = rx[m];
            sm.ry[tv_ri(li, lj)] = ry[m];
        }
        __syncthreads();
        for (int k = 0; k < nsteps; ++k) {
            const float beta = s_beta[k];
            // x = w + theta div r
#pragma unroll
            for (int m = 0; m < kTvM; ++m) {
                const int li = tr + kTvRows * m;
                const float dv = ((rx[m] - sm.rx[tv_ri(li, lj - 1)]) + ry[m]) - sm.ry[tv_ri(li - 1, lj)];
                xv[m] = fmaf(theta, dv, w[m]);
                sm.x[li * kTvR + lj] = xv[m];
            }
            __syncthreads();
            // (p, r) update from grad x
#pragma unroll
            for (int m = 0; m < kTvM; ++m) {
                const int li = tr + kTvRows * m;
                const float x0 = xv[m];
                // neighbours loaded unconditionally (always inside the arrays), then masked
                const float xe = sm.x[li * kTvR + lj + 1], xs = sm.x[(li + 1) * kTvR + lj];
                const float gx = fx ? xe - x0 : 0.0f;
                const float gy = (fy >> m) & 1u ? xs - x0 : 0.0f;
                const float qx = fmaf(step, gx, rx[m]);
                const float qy = fmaf(step, gy, ry[m]);
                // projection onto the unit disc: q / max(1, |q|), with the
                // hardware reciprocal square root where |q| > 1
                const float s2 = fmaf(qx, qx, qy * qy);
                const float inv = s2 > 1.0f ? rsqrtf(s2) : 1.0f;
                const float nx_ = qx * inv, ny_ = qy * inv;
                rx[m] = fmaf(beta, nx_ - px[m], nx_);
                ry[m] = fmaf(beta, ny_ - py[m], ny_);
                px[m] = nx_;
                py[m] = ny_;
                // read by the neighbours in the next x update, after the barrier
                sm.rx[tv_ri(li, lj)] = rx[m];
                sm.ry[tv_ri(li, lj)] = ry[m];
            }
            __syncthreads();
        }
        // the tile (exact after nsteps <= kTvK steps) to the second buffers
        if (jin && lj >= kTvK && lj < kTvK + kTvT) {
#pragma unroll
            for (int m = 0; m < kTvM; ++m) {
                const int li = tr + kTvRows * m, gi = i0 + li;
                if (li >= kTvK && li < kTvK + kTvT && gi < ny) {
                    const long long q = (long long)gi * nx + gj;
                    px2[q] = px[m];
                    py2[q] = py[m];
                    rx2[q] = rx[m];
                    ry2[q] = ry[m];
                }
            }
        }
    }
    t = s_t;
    __syncthreads();  // s_t and s_beta are rewritten by the next call
}

__global__ void __launch_bounds__(kTvThreads, 2) k_tv_project(TvArgs a)
{
    if (a.done && ld_volatile_i32(a.done)) return;
    extern __shared__ __align__(16) unsigned char tv_smem[];
    TvSmem &sm = *reinterpret_cast<TvSmem *>(tv_smem);
    // the pads of the dual-step arrays are never written after this
    for (int e = threadIdx.x; e < (int)(sizeof(TvSmem) / sizeof(float)); e += kTvThreads)
        reinterpret_cast<float *>(tv_smem)[e] = 0.0f;
    __syncthreads();
    const long long stride = (long long)gridDim.x * kTvThreads;
    const long long first = (long long)blockIdx.x * kTvThreads + threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    float *px = a.dual[0], *py = a.dual[1], *rx = a.dual[2], *ry = a.dual[3];
    float *px2 = a.dual[4], *py2 = a.dual[5], *rx2 = a.dual[6], *ry2 = a.dual[7];
    bool ok = true;
    int slot = 0;

    for (long long q = first; q < a.d; q += stride) {
        a.zk[q] = a.z[q];
        a.pk[q] = 0.0f;
        a.qk[q] = 0.0f;
        px[q] = 0.0f;
        py[q] = 0.0f;
    }
    double lam = *a.lam_io > 0.0 ? *a.lam_io : 1.0;
    int rounds = 0, solves = 0;
    for (int k = 1; k <= a.max_dyk; ++k) {
        for (long long q = first; q < a.d; q += stride) a.w[q] = __ldcg(a.zk + q) + __ldcg(a.pk + q);
        if (!grid_barrier(a.bar, a.err, a.done, a.bar_polls)) return;
        double part = 0.0;
        double tw = 0.0;
        if (!a.fixed_lam) {
            for (long long q = first; q < a.d; q += stride)
                part += tv_term(a.w, tv_row(q, nx), tv_col(q, nx), nx, ny);
            tw = grid_sum(a, part, slot, ok);
            slot ^= 1;
            if (!ok) return;
        }
        const float *ysrc = a.w;
        if (tw > a.tau || a.fixed_lam) {
            double lo = 0.0, hi = INFINITY;
            for (int s = 0; s < a.max_bisect; ++s) {
                const float theta = (float)(0.5 * lam);
                const float step = (float)(1.0 / (4.0 * lam));  // 1 / (8 theta)
                double t = 1.0;
                for (int it = 0; it < a.fgp_iters; it += kTvK) {
                    const int ns = a.fgp_iters - it < kTvK ? a.fgp_iters - it : kTvK;
                    // the first block starts r at p, the carried dual
                    fgp_block(a, sm, it == 0 ? px : rx, it == 0 ? py : ry, px, py, px2, py2, rx2, ry2, theta, step,
                              t, ns);
                    if (!grid_barrier(a.bar, a.err, a.done, a.bar_polls)) return;
                    float *tp;
                    tp = px; px = px2; px2 = tp;
                    tp = py; py = py2; py2 = tp;
                    tp = rx; rx = rx2; rx2 = tp;
                    tp = ry; ry = ry2; ry2 = tp;
                }
                // x = w + theta div p, and its TV from the neighbours' x
                // recomputed in place (the same FP32 values), so no barrier
                // separates the two; later phases read xt only at the pixel
                // each thread wrote
                part = 0.0;
                for (long long q = first; q < a.d; q += stride) {
                    const int i = tv_row(q, nx), j = tv_col(q, nx);
                    const float c = prox_x(a.w, px, py, theta, i, j, nx, ny);
                    a.xt[q] = c;
                    if (!a.fixed_lam) {
                        const float gx = j < nx - 1 ? prox_x(a.w, px, py, theta, i, j + 1, nx, ny) - c : 0.0f;
                        const float gy = i < ny - 1 ? prox_x(a.w, px, py, theta, i + 1, j, nx, ny) - c : 0.0f;
                        part += sqrt((double)gx * gx + (double)gy * gy);
                    }
                }
                if (a.fixed_lam) {
                    ++solves;
                    break;
                }
                const double tx = grid_sum(a, part, slot, ok);
                slot ^= 1;
                if (!ok) return;
                ++solves;
                if (fabs(tx - a.tau) <= a.tol_tv) break;
                if (tx > a.tau) lo = lam;
                else hi = lam;
                lam = isinf(hi) ? 2.0 * lam : 0.5 * (lo + hi);
            }
            ysrc = a.xt;
        }
        part = 0.0;
        for (long long q = first; q < a.d; q += stride) {
            const float y = __ldcg(ysrc + q), wv = __ldcg(a.w + q), qv = __ldcg(a.qk + q), zo = __ldcg(a.zk + q);
            const float yq = y + qv;
            const float zn = fminf(fmaxf(yq, a.lo), a.hi);
            a.pk[q] = wv - y;
            a.qk[q] = yq - zn;
            a.zk[q] = zn;
            const double dz = (double)zn - (double)zo;
            part += dz * dz;
        }
        const double chg = grid_sum(a, part, slot, ok);
        slot ^= 1;
        if (!ok) return;
        rounds = k;
        if (sqrt(chg) <= a.tol_dyk) break;
    }
    // result, padded copies and (solve path) the partial norms of the step
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (long long q = first; q < a.d; q += stride) {
        const float v = __ldcg(a.zk + q);
        const int i = tv_row(q, nx), j = tv_col(q, nx);
        if (a.old_r) {  // read before out_r, which may be the same image
            const double xb = (double)__ldcg(a.old_r + (long long)i * a.ldr + j + kPad);
            const double dd = (double)v - xb;
            s0 += dd * dd;
            s1 += xb * xb;
            if (a.hist) {  // running average of Sec. 3.1, as in the extragradient epilogue
                const double sp = a.avg[q];
                double sn = sp + (double)v;
                if (a.hist_drop >= 0) sn -= (double)a.hist[(long long)a.hist_drop * a.d + q];
                a.hist[(long long)a.hist_put * a.d + q] = v;
                a.avg[q] = sn;
                const double dv = sn * a.inv_m - sp * a.inv_m_prev;
                s2 += dv * dv;
            }
        }
        if (a.out) a.out[q] = v;
        if (a.out_r) a.out_r[(long long)i * a.ldr + j + kPad] = v;
        if (a.out_c) a.out_c[(long long)j * a.ldc + i + kPad] = v;
    }
    if (a.old_r) {
        const double b0 = block_sum(s0), b1 = block_sum(s1), b2 = block_sum(s2);
        if (threadIdx.x == 0) {
            a.norm_part[kPartStride * blockIdx.x] = b0;
            a.norm_part[kPartStride * blockIdx.x + 1] = b1;
            a.norm_part[kPartStride * blockIdx.x + 2] = b2;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.lam_io = lam;
        a.stats[0] = rounds;
        a.stats[1] = solves;
    }
}

int g_tv_grid[64] = {};  // cooperative grid per device (0: not queried yet)

size_t tv_align(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

size_t tv_workspace_bytes(int nx, int ny, int grid)
{
    const size_t d = (size_t)nx * ny;
    return tv_align(sizeof(float) * d) * 13 + tv_align(sizeof(double) * 2 * (size_t)grid) + tv_align(sizeof(TvTail));
}

int tv_grid(long long d)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!g_tv_grid[dev]) {
        int sms = 0, per = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (cudaFuncSetAttribute(k_tv_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TvSmem)) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tv_project, kTvThreads, sizeof(TvSmem)) !=
                cudaSuccess)
            return 0;
        if (per < 1) return 0;
        g_tv_grid[dev] = sms * (per < 4 ? per : 4);
    }
    const long long need = (d + kTvThreads - 1) / kTvThreads;
    return (int)(need < g_tv_grid[dev] ? (need > 0 ? need : 1) : g_tv_grid[dev]);
}

TvTail *tv_tail(void *ws, int nx, int ny, int grid)
{
    const size_t d = (size_t)nx * ny;
    return reinterpret_cast<TvTail *>(static_cast<char *>(ws) + tv_align(sizeof(float) * d) * 13 +
                                      tv_align(sizeof(double) * 2 * (size_t)grid));
}

cudaError_t launch_tv_project(const TvLaunch &L, cudaStream_t s)
{
    TvArgs a;
    memset(&a, 0, sizeof(a));
    a.nx = L.nx;
    a.ny = L.ny;
    a.d = (long long)L.nx * L.ny;
    a.z = L.z;
    a.out = L.out;
    a.out_r = L.out_r;
    a.out_c = L.out_c;
    a.ldr = L.ldr;
    a.ldc = L.ldc;
    a.old_r = L.old_r;
    a.norm_part = L.norm_part;
    a.avg = L.avg;
    a.hist = L.hist;
    a.hist_put = L.hist_put;
    a.hist_drop = L.hist_drop;
    a.inv_m = L.inv_m;
    a.inv_m_prev = L.inv_m_prev;
    // workspace layout: 13 pixel arrays, partial sums, tail words
    char *p = static_cast<char *>(L.ws);
    const size_t fb = tv_align(sizeof(float) * (size_t)a.d);
    float **arrs[5] = {&a.zk, &a.pk, &a.qk, &a.w, &a.xt};
    for (int i = 0; i < 5; ++i, p += fb) *arrs[i] = reinterpret_cast<float *>(p);
    for (int i = 0; i < 8; ++i, p += fb) a.dual[i] = reinterpret_cast<float *>(p);
    a.part = reinterpret_cast<double *>(p);
    TvTail *tail = tv_tail(L.ws, L.nx, L.ny, L.grid);
    a.bar = tail->bar;
    a.err = L.state ? &L.state->status : &tail->status;
    a.done = L.state ? &L.state->done : nullptr;
    a.lam_io = L.lam_io ? L.lam_io : &tail->lam;
    a.stats = tail->stats;
    a.tau = L.tau;
    a.tol_tv = L.tol_tv;
    a.tol_dyk = L.tol_dykstra;
    a.fgp_iters = L.fgp_iters;
    a.max_bisect = L.max_bisect;
    a.max_dyk = L.max_dykstra;
    a.lo = L.fixed_lam ? -INFINITY : L.lo;
    a.hi = L.fixed_lam ? INFINITY : L.hi;
    a.fixed_lam = L.fixed_lam;
    if (L.fixed_lam) a.max_dyk = 1;
    a.bar_polls = debug_wait_polls() > 0 ? debug_wait_polls() : kTvBarrierSpins;
    cudaError_t e = cudaMemsetAsync(tail->bar, 0, sizeof(tail->bar), s);
    if (e != cudaSuccess) return e;
    if (debug_take_tv_block()) {
        // fault injection: arrivals start at the grid size, so no arrival
        // completes the first barrier and every CTA's wait runs out
        const unsigned g = (unsigned)L.grid;
        e = cudaMemcpyAsync(tail->bar, &g, sizeof(g), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // g lives on this stack frame
        if (e != cudaSuccess) return e;
    }
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel((const void *)k_tv_project, dim3(L.grid), dim3(kTvThreads), args,
                                       sizeof(TvSmem), s);
}

}  // namespace exact

using namespace exact;

extern "C" {

exact_tv_opts exact_tv_opts_default(void)
{
    exact_tv_opts o;
    o.fgp_iters = 40;
    o.max_bisect = 40;
    o.max_dykstra = 50;
    o.pad = 0;
    o.tol_tv = 0.01;
    o.tol_dykstra = 1e-4;
    o.lam0 = 0.0;
    return o;
}

size_t exact_tv_workspace_bytes(int nx, int ny)
{
    if (nx < 1 || ny < 1) return 0;
    const int grid = tv_grid((long long)nx * ny);
    return grid > 0 ? tv_workspace_bytes(nx, ny, grid) : 0;
}

exact_status exact_tv_project(int nx, int ny, const float *z, double tau, double lo, double hi,
                              const exact_tv_opts *opts, float *x, void *workspace, size_t workspace_bytes,
                              exact_tv_info *info, exact_stream_t stream)
{
    if (nx < 1 || ny < 1 || nx > 16384 || ny > 16384 || !z || !x || !workspace || z == x) return EXACT_ERR_INVALID_ARG;
    if (!(tau >= 0.0) || !(tau < INFINITY) || isnan(lo) || isnan(hi) || lo > hi || lo == INFINITY ||
        hi == -INFINITY)
        return EXACT_ERR_INVALID_ARG;
    const exact_tv_opts o = opts ? *opts : exact_tv_opts_default();
    if (o.fgp_iters < 1 || o.max_bisect < 1 || o.max_dykstra < 0 || !(o.tol_tv >= 0.0) || !(o.tol_dykstra >= 0.0) ||
        !(o.lam0 < INFINITY) || isnan(o.lam0))
        return EXACT_ERR_INVALID_ARG;
    const int grid = tv_grid((long long)nx * ny);
    if (grid <= 0) return EXACT_ERR_CUDA;
    if (workspace_bytes < tv_workspace_bytes(nx, ny, grid)) return EXACT_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TvTail *tail = tv_tail(workspace, nx, ny, grid);
    TvTail h;
    memset(&h, 0, sizeof(h));
    h.lam = o.lam0;
    if (cudaMemcpyAsync(tail, &h, sizeof(h), cudaMemcpyHostToDevice, s) != cudaSuccess) return EXACT_ERR_CUDA;
    TvLaunch L;
    memset(&L, 0, sizeof(L));
    L.nx = nx;
    L.ny = ny;
    L.grid = grid;
    L.z = z;
    L.out = x;
    L.ws = workspace;
    L.tau = tau;
    L.tol_tv = o.tol_tv;
    L.tol_dykstra = o.tol_dykstra;
    L.fgp_iters = o.fgp_iters;
    L.max_bisect = o.max_bisect;
    L.max_dykstra = o.max_dykstra;
    L.lo = (float)lo;
    L.hi = (float)hi;
    cudaError_t e = launch_tv_project(L, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, tail, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? EXACT_ERR_OOM : EXACT_ERR_CUDA;
    if (info) {
        info->rounds = h.stats[0];
        info->solves = h.stats[1];
        info->lam = h.lam;
        info->status = (exact_status)h.status;
    }
    return h.status == 0 ? EXACT_OK : (exact_status)h.status;
}

exact_status exact_tv_prox(int nx, int ny, const float *z, double lam, int fgp_iters, float *x, void *workspace,
                           size_t workspace_bytes, exact_stream_t stream)
{
    if (nx < 1 || ny < 1 || nx > 16384 || ny > 16384 || !z || !x || !workspace || z == x) return EXACT_ERR_INVALID_ARG;
    if (!(lam > 0.0) || !(lam < INFINITY) || fgp_iters < 1) return EXACT_ERR_INVALID_ARG;
    const int grid = tv_grid((long long)nx * ny);
    if (grid <= 0) return EXACT_ERR_CUDA;
    if (workspace_bytes < tv_workspace_bytes(nx, ny, grid)) return EXACT_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TvTail *tail = tv_tail(workspace, nx, ny, grid);
    TvTail h;
    memset(&h, 0, sizeof(h));
    h.lam = lam;
    if (cudaMemcpyAsync(tail, &h, sizeof(h), cudaMemcpyHostToDevice, s) != cudaSuccess) return EXACT_ERR_CUDA;
    TvLaunch L;
    memset(&L, 0, sizeof(L));
    L.nx = nx;
    L.ny = ny;
    L.grid = grid;
    L.z = z;
    L.out = x;
    L.ws = workspace;
    L.fgp_iters = fgp_iters;
    L.max_bisect = 1;
    L.max_dykstra = 1;
    L.fixed_lam = 1;
    cudaError_t e = launch_tv_project(L, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, tail, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? EXACT_ERR_OOM : EXACT_ERR_CUDA;
    return h.status == 0 ? EXACT_OK : (exact_status)h.status;
}

}  // extern "C"
