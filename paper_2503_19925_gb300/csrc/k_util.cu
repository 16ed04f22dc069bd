// k_util.cu -- small kernels around the hot path: image packing into the
// padded row- and column-major copies, the window sum of the counts, the
// fixed-order FP64 reductions that drive stopping (solve) and convergence
// (power iteration), and state resets.  None of these loops over rays.
#include "exact_internal.h"

#include <math.h>

namespace exact {

namespace {

__device__ __forceinline__ float proj(float v, float lo, float hi, bool project)
{
    return project ? (v < lo ? lo : (v > hi ? hi : v)) : v;
}

// Row-major copy with kPad zero columns on each side (values times *scale
// when scale is given).
__global__ void k_pack_rows(const float *x, float *xr, int nx, int ny, long long ldr, float lo, float hi,
                            bool project, const double *scale)
{
    const long long total = (long long)ny * ldr;
    const float sc = scale ? (float)*scale : 1.0f;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / ldr;
        const long long k = e - j * ldr - kPad;
        xr[e] = (k >= 0 && k < nx) ? sc * proj(x[j * nx + k], lo, hi, project) : 0.0f;
    }
}

// Column-major copy (x transposed) with kPad zero entries on each side,
// through a shared-memory tile.
__global__ void k_pack_cols(const float *x, float *xc, int nx, int ny, long long ldc, float lo, float hi,
                            bool project, const double *scale)
{
    __shared__ float tile[32][33];
    const float sc = scale ? (float)*scale : 1.0f;
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int iy = by + r, ix = bx + threadIdx.x;
        tile[r][threadIdx.x] = (ix < nx && iy < ny) ? sc * proj(x[(long long)iy * nx + ix], lo, hi, project) : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int ix = bx + r, iy = by + threadIdx.x;
        if (ix < nx && iy < ny) xc[(long long)ix * ldc + iy + kPad] = tile[threadIdx.x][r];
    }
    // pads (and the alignment tail) of the rows this block owns
    if (blockIdx.y == 0 && threadIdx.y == 0 && threadIdx.x < 32) {
        const int ix = bx + threadIdx.x;
        if (ix < nx) {
            for (int p = 0; p < kPad; ++p) xc[(long long)ix * ldc + p] = 0.0f;
            for (long long p = kPad + ny; p < ldc; ++p) xc[(long long)ix * ldc + p] = 0.0f;
        }
    }
}

__global__ void k_unpack(const float *xr, long long ldr, int nx, int ny, float *x, const double *avg,
                         const DevState *st, int avg_from)
{
    const long long d = (long long)nx * ny;
    long long cnt = 0;
    // avg_from >= 0: tail average of the iterates after avg_from; avg_from < 0:
    // running-average window sum of the last max(1, floor(T/2)) iterates
    if (avg) cnt = avg_from >= 0 ? (long long)st->iters_done - avg_from : max(1, st->iters_done / 2);
    if (avg && avg_from < 0 && st->iters_done == 0) cnt = 0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < d;
         p += (long long)gridDim.x * blockDim.x) {
        const long long j = p / nx, k = p - j * nx;
        if (avg && cnt > 0)
            x[p] = (float)(avg[p] / (double)cnt);
        else
            x[p] = xr[j * ldr + k + kPad];
    }
}

template <typename Tin>
__device__ __forceinline__ float to_f(Tin v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename Tin>
__global__ void k_collapse(const Tin *y, int W, long long n, float *Y)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int w = 0; w < W; ++w) s += to_f<Tin>(y[(long long)w * n + i]);
        Y[i] = s;
    }
}

constexpr int RT = 256;  // threads of the single-block reductions

// Fixed-order sum over `count` values with stride `stride` starting at `src`,
// result in thread 0.
__device__ double block_sum_fixed(const double *src, int count, int stride)
{
    __shared__ double s[RT];
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += RT) acc += src[(long long)i * stride];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = RT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    const double r = s[0];
    __syncthreads();
    return r;
}

// COND: launched inside a CUDA graph's WHILE loop; the iteration index is
// st->iters_done and thread 0 sets the loop condition on every launch (also
// when the solve already stopped), so the loop always ends: iters_done grows by
// one per iteration up to st->iter_end.
template <bool COND>
__global__ void __launch_bounds__(RT) k_solve_reduce(const double *partials, int nparts, DevState *st, int iter,
                                                     cudaGraphConditionalHandle cond)
{
    if (st->done) {
        if (COND && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    const int rule = st->rule;
    const double num = block_sum_fixed(partials, nparts, kPartStride);
    const double den = block_sum_fixed(partials + 1, nparts, kPartStride);
    const double chg = rule == EXACT_STOP_AVERAGE ? block_sum_fixed(partials + 2, nparts, kPartStride) : 0.0;
    if (threadIdx.x == 0) {
        const double rel = sqrt(num) / fmax(sqrt(den), 1e-30);
        const int t = (COND ? st->iters_done : iter) + 1;  // iterations run
        const double tol = st->tol;
        const int check_every = st->check_every;
        st->rel_res = rel;
        st->avg_change = (rule == EXACT_STOP_AVERAGE && t >= 2) ? sqrt(chg) : 0.0;
        st->iters_done = t;
        const double crit = rule == EXACT_STOP_AVERAGE ? st->avg_change : rel;
        const bool may_stop = rule == EXACT_STOP_AVERAGE ? t >= 2 : true;
        if (!isfinite(rel) || !isfinite(crit)) {
            st->status = EXACT_ERR_NONFINITE;
            st->done = 1;
        } else if (may_stop && tol > 0.0 && check_every > 0 && t % check_every == 0 && crit <= tol) {
            st->done = 1;
        }
        if (COND) cudaGraphSetConditional(cond, (!st->done && t < st->iter_end) ? 1u : 0u);
    }
}

__global__ void k_reset_state(DevState *st, int t0, int t_end, double tol, int check_every, int rule, int avg_from)
{
    st->done = 0;
    st->iters_done = t0;
    st->status = EXACT_OK;
    st->rel_res = 0.0;
    st->lam = 0.0;
    st->lam_prev = 0.0;
    st->inv_norm = 1.0;
    st->avg_change = 0.0;
    st->iter_end = t_end;
    st->check_every = check_every;
    st->rule = rule;
    st->avg_from = avg_from;
    st->tol = tol;
}

__global__ void k_power_init(double *xrd, double *xcd, int nx, int ny, long long ldr, long long ldc, DevState *st)
{
    const long long tr = (long long)ny * ldr, tc = (long long)nx * ldc;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tr + tc;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < tr) {
            const long long k = e % ldr - kPad;
            xrd[e] = (k >= 0 && k < nx) ? 1.0 : 0.0;
        } else {
            const long long k = (e - tr) % ldc - kPad;
            xcd[e - tr] = (k >= 0 && k < ny) ? 1.0 : 0.0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->done = 0;
        st->iters_done = 0;
        st->status = EXACT_OK;
        st->lam = 0.0;
        st->lam_prev = 0.0;
        st->inv_norm = 1.0 / sqrt((double)nx * (double)ny);
    }
}

__global__ void __launch_bounds__(RT) k_power_reduce(const double *pz, int nz, const double *pw, int nw,
                                                     DevState *st, int iter, double rtol)
{
    if (st->done) return;
    const double lam = block_sum_fixed(pz, nz, 1);
    const double w2 = block_sum_fixed(pw, nw, 1);
    if (threadIdx.x == 0) {
        st->lam = lam;
        st->iters_done = iter + 1;
        const double nrm = sqrt(w2);
        if (!(nrm > 0.0) || !isfinite(nrm)) {
            if (!isfinite(nrm)) st->status = EXACT_ERR_NONFINITE;
            st->done = 1;
        } else {
            st->inv_norm = 1.0 / nrm;
            if (iter > 0 && rtol > 0.0 && fabs(lam - st->lam_prev) <= rtol * lam) st->done = 1;
            st->lam_prev = lam;
        }
    }
}

// Per-block FP64 partial sums of v[i]^2 over fixed contiguous chunks.
__global__ void __launch_bounds__(256) k_sumsq(const float *v, long long n, double *partials)
{
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long b0 = (long long)blockIdx.x * per, b1 = b0 + per < n ? b0 + per : n;
    double acc = 0.0;
    for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const double d = (double)v[i];
        acc += d * d;
    }
    __shared__ double s[256];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = s[0];
}

// FP32 power iteration start: w = 1 (so v_1 = 1/sqrt(d) after scaling).
__global__ void k_power_init_f(float *w, long long d, DevState *st)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (long long)gridDim.x * blockDim.x)
        w[i] = 1.0f;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->done = 0;
        st->iters_done = 0;
        st->status = EXACT_OK;
        st->lam = 0.0;
        st->lam_prev = 0.0;
        st->inv_norm = 1.0 / sqrt((double)d);
    }
}

unsigned grid_for(long long work, int threads)
{
    long long b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

}  // namespace

cudaError_t launch_pack(const float *x, float *xr, float *xc, int nx, int ny, long long ldr, long long ldc,
                        float lo, float hi, bool project, cudaStream_t s, const double *scale)
{
    k_pack_rows<<<grid_for((long long)ny * ldr, 256), 256, 0, s>>>(x, xr, nx, ny, ldr, lo, hi, project, scale);
    const dim3 grid((nx + 31) / 32, (ny + 31) / 32);
    k_pack_cols<<<grid, dim3(32, 8), 0, s>>>(x, xc, nx, ny, ldc, lo, hi, project, scale);
    return cudaGetLastError();
}

cudaError_t launch_sumsq(const float *v, long long n, double *partials, int nparts, cudaStream_t s)
{
    k_sumsq<<<nparts, 256, 0, s>>>(v, n, partials);
    return cudaGetLastError();
}

cudaError_t launch_power_init_f(float *w, long long d, DevState *st, cudaStream_t s)
{
    k_power_init_f<<<grid_for(d, 256), 256, 0, s>>>(w, d, st);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const float *xr, long long ldr, int nx, int ny, float *x, const double *avg,
                          const DevState *state, int avg_from, cudaStream_t s)
{
    k_unpack<<<grid_for((long long)nx * ny, 256), 256, 0, s>>>(xr, ldr, nx, ny, x, avg, state, avg_from);
    return cudaGetLastError();
}

cudaError_t launch_collapse(const void *y, int dtype, int W, long long n, float *Y, cudaStream_t s)
{
    if (dtype == EXACT_BF16)
        k_collapse<__nv_bfloat16><<<grid_for(n, 256), 256, 0, s>>>((const __nv_bfloat16 *)y, W, n, Y);
    else
        k_collapse<float><<<grid_for(n, 256), 256, 0, s>>>((const float *)y, W, n, Y);
    return cudaGetLastError();
}

cudaError_t launch_solve_reduce(const double *partials, int nparts, DevState *st, int iter, cudaStream_t s)
{
    k_solve_reduce<false><<<1, RT, 0, s>>>(partials, nparts, st, iter, cudaGraphConditionalHandle{});
    return cudaGetLastError();
}

cudaError_t launch_solve_reduce_cond(const double *partials, int nparts, DevState *st,
                                     cudaGraphConditionalHandle cond, cudaStream_t s)
{
    k_solve_reduce<true><<<1, RT, 0, s>>>(partials, nparts, st, -1, cond);
    return cudaGetLastError();
}

cudaError_t launch_reset_state(DevState *st, int t0, int t_end, double tol, int check_every, int rule, int avg_from,
                               cudaStream_t s)
{
    k_reset_state<<<1, 1, 0, s>>>(st, t0, t_end, tol, check_every, rule, avg_from);
    return cudaGetLastError();
}

cudaError_t launch_power_init(double *xrd, double *xcd, int nx, int ny, long long ldr, long long ldc,
                              DevState *st, cudaStream_t s)
{
    k_power_init<<<grid_for((long long)ny * ldr + (long long)nx * ldc, 256), 256, 0, s>>>(xrd, xcd, nx, ny, ldr,
                                                                                        ldc, st);
    return cudaGetLastError();
}

cudaError_t launch_power_reduce(const double *pz, int nz, const double *pw, int nw, DevState *st, int iter,
                                double rtol, cudaStream_t s)
{
    k_power_reduce<<<1, RT, 0, s>>>(pz, nz, pw, nw, st, iter, rtol);
    return cudaGetLastError();
}

}  // namespace exact
