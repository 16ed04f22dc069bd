// k_dense.cu -- EXACT with dense measurement vectors (the Gaussian model of
// Sec. 2.2 and the experiment of Sec. 3.2 / Fig. 6): the operator of Eq. (8)
// with an explicit matrix A (rows a_i) instead of the projector, and the
// projected extragradient iteration of Eq. (11) on a box, all in FP64 (the
// experiment follows the error down to machine precision).
//
//   z_i = <a_i, x>              one warp per row, fixed shuffle tree
//   r_i = sum_w (y_{w,i} - I0 sum_k S[w][k] exp(-mu_k max(z_i, 0)))
//   g   = A^T r                 per-chunk column partials, then a fixed-order
//                               sum over the chunks (no atomics)
//   x'  = P_[lo,hi](x_base - eta g / (W n))
//
// Deterministic: every sum has one fixed order.
#include "exact_internal.h"

#include <math.h>
#include <new>
#include <string.h>

namespace exact {
namespace {

constexpr int kDenseRowWarps = 8;    // rows per CTA of the forward kernel (one warp each)
constexpr int kDenseRowsPerChunk = 64;
constexpr int kDenseCols = 128;      // columns per CTA of the adjoint kernels

__global__ void __launch_bounds__(kDenseRowWarps * 32)
    k_dense_fwd_link(const double *__restrict__ A, int n, int d, const double *__restrict__ x, int W, int K,
                     const double *__restrict__ S, const double *__restrict__ mu, double I0,
                     const double *__restrict__ y, double *__restrict__ r)
{
    const int lane = threadIdx.x & 31;
    const long long i = (long long)blockIdx.x * kDenseRowWarps + (threadIdx.x >> 5);
    if (i >= n) return;
    const double *ai = A + i * d;
    double z = 0.0;
    for (int j = lane; j < d; j += 32) z = fma(ai[j], x[j], z);
    for (int o = 16; o > 0; o >>= 1) z += __shfl_down_sync(0xffffffffu, z, o);
    if (lane == 0) {
        const double zp = z > 0.0 ? z : 0.0;
        double res = 0.0;
        for (int w = 0; w < W; ++w) {
            double h = 0.0;
            for (int k = 0; k < K; ++k) h = fma(S[w * K + k], exp(-mu[k] * zp), h);
            res += y[(long long)w * n + i] - I0 * h;
        }
        r[i] = res;
    }
}

// part[c][j] = sum over the rows of chunk c of A[i][j] r[i], in row order.
__global__ void __launch_bounds__(kDenseCols)
    k_dense_adj_partial(const double *__restrict__ A, int n, int d, const double *__restrict__ r,
                        double *__restrict__ part)
{
    const int j = blockIdx.y * kDenseCols + threadIdx.x;
    const int c = blockIdx.x;
    if (j >= d) return;
    const int i0 = c * kDenseRowsPerChunk, i1 = min(n, i0 + kDenseRowsPerChunk);
    double s = 0.0;
    for (int i = i0; i < i1; ++i) s = fma(A[(long long)i * d + j], r[i], s);
    part[(long long)c * d + j] = s;
}

// g_j = sum_c part[c][j] (chunk order); out_j = base ? clamp(base_j + scale g_j)
// : scale g_j.  With x_true, err[slot] = ||out - x_true|| (one CTA, fixed tree).
__global__ void __launch_bounds__(kDenseCols)
    k_dense_step(const double *__restrict__ part, int chunks, int d, double scale, const double *base, double lo,
                 double hi, double *out, const double *__restrict__ x_true, double *err, int slot)
{
    __shared__ double red[kDenseCols];
    double e2 = 0.0;
    for (int j = threadIdx.x; j < d; j += kDenseCols) {
        double g = 0.0;
        for (int c = 0; c < chunks; ++c) g += part[(long long)c * d + j];
        double v = scale * g;
        if (base) {
            v += base[j];
            v = v < lo ? lo : (v > hi ? hi : v);  // keeps a NaN
        }
        out[j] = v;
        if (x_true) {
            const double dv = v - x_true[j];
            e2 = fma(dv, dv, e2);
        }
    }
    if (!x_true) return;
    red[threadIdx.x] = e2;
    __syncthreads();
    for (int h = kDenseCols / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) err[slot] = sqrt(red[0]);
}

}  // namespace
}  // namespace exact

using namespace exact;

struct exact_dense {
    int device = -1;
    int n = 0, d = 0, W = 0, K = 0;
    const double *A = nullptr;
    double *S = nullptr, *mu = nullptr;  // device copies
    double *r = nullptr, *part = nullptr, *xh = nullptr;
    int chunks = 0;
};

namespace {

exact_status dense_status(cudaError_t e)
{
    if (e == cudaSuccess) return EXACT_OK;
    return e == cudaErrorMemoryAllocation ? EXACT_ERR_OOM : EXACT_ERR_CUDA;
}

cudaError_t dense_F(const exact_dense &D, const double *x, const double *y, double I0, double scale,
                    const double *base, double lo, double hi, double *out, const double *x_true, double *err,
                    int slot, cudaStream_t s)
{
    k_dense_fwd_link<<<(D.n + kDenseRowWarps - 1) / kDenseRowWarps, kDenseRowWarps * 32, 0, s>>>(
        D.A, D.n, D.d, x, D.W, D.K, D.S, D.mu, I0, y, D.r);
    const dim3 g2(D.chunks, (D.d + kDenseCols - 1) / kDenseCols);
    k_dense_adj_partial<<<g2, kDenseCols, 0, s>>>(D.A, D.n, D.d, D.r, D.part);
    k_dense_step<<<1, kDenseCols, 0, s>>>(D.part, D.chunks, D.d, scale, base, lo, hi, out, x_true, err, slot);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

exact_status exact_dense_create(int n, int d, const double *A, const exact_spectrum *spectrum,
                                const exact_windows *windows, exact_dense_t *out)
{
    if (!out) return EXACT_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || d < 1 || (long long)n * d > (1LL << 34) || !A || !spectrum || !windows) return EXACT_ERR_INVALID_ARG;
    const int K = spectrum->n_energy, W = windows->n_windows;
    if (K < 1 || K > EXACT_MAX_ENERGY || W < 1 || W > 64 || !spectrum->mu || !windows->S) return EXACT_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k)
        if (!(spectrum->mu[k] > 0.0) || !(spectrum->mu[k] < INFINITY)) return EXACT_ERR_INVALID_ARG;
    for (int q = 0; q < W * K; ++q)
        if (!(windows->S[q] >= 0.0) || !(windows->S[q] < INFINITY)) return EXACT_ERR_INVALID_ARG;
    exact_dense *D = new (std::nothrow) exact_dense;
    if (!D) return EXACT_ERR_OOM;
    if (cudaGetDevice(&D->device) != cudaSuccess) {
        delete D;
        return EXACT_ERR_CUDA;
    }
    D->n = n;
    D->d = d;
    D->W = W;
    D->K = K;
    D->A = A;
    D->chunks = (n + kDenseRowsPerChunk - 1) / kDenseRowsPerChunk;
    cudaError_t e = cudaMalloc(&D->S, sizeof(double) * W * K);
    if (e == cudaSuccess) e = cudaMalloc(&D->mu, sizeof(double) * K);
    if (e == cudaSuccess) e = cudaMalloc(&D->r, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&D->part, sizeof(double) * (size_t)D->chunks * d);
    if (e == cudaSuccess) e = cudaMalloc(&D->xh, sizeof(double) * d);
    if (e == cudaSuccess) e = cudaMemcpy(D->S, windows->S, sizeof(double) * W * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(D->mu, spectrum->mu, sizeof(double) * K, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        exact_dense_destroy(D);
        return dense_status(e);
    }
    *out = D;
    return EXACT_OK;
}

exact_status exact_dense_destroy(exact_dense_t D)
{
    if (!D) return EXACT_OK;
    cudaFree(D->S);
    cudaFree(D->mu);
    cudaFree(D->r);
    cudaFree(D->part);
    cudaFree(D->xh);
    delete D;
    return EXACT_OK;
}

exact_status exact_dense_operator(exact_dense_t D, const double *x, const double *y, double I0, double *F,
                                  exact_stream_t stream)
{
    if (!D || !x || !y || !F || !(I0 > 0.0) || !(I0 < INFINITY)) return EXACT_ERR_INVALID_ARG;
    const double scale = 1.0 / ((double)D->W * (double)D->n);
    return dense_status(dense_F(*D, x, y, I0, scale, nullptr, 0.0, 0.0, F, nullptr, nullptr, 0,
                                reinterpret_cast<cudaStream_t>(stream)));
}

exact_status exact_dense_solve(exact_dense_t D, const double *y, double I0, double eta, int iters, double lo,
                               double hi, double *x, const double *x_true, double *err, exact_stream_t stream)
{
    if (!D || !y || !x || !(I0 > 0.0) || !(I0 < INFINITY) || !(eta > 0.0) || !(eta < INFINITY) || iters < 0)
        return EXACT_ERR_INVALID_ARG;
    if (isnan(lo) || isnan(hi) || lo > hi || lo == INFINITY || hi == -INFINITY) return EXACT_ERR_INVALID_ARG;
    if ((x_true == nullptr) != (err == nullptr)) return EXACT_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const double scale = -eta / ((double)D->W * (double)D->n);
    for (int t = 0; t < iters; ++t) {
        cudaError_t e = dense_F(*D, x, y, I0, scale, x, lo, hi, D->xh, nullptr, nullptr, 0, s);
        if (e == cudaSuccess) e = dense_F(*D, D->xh, y, I0, scale, x, lo, hi, x, x_true, err, t, s);
        if (e != cudaSuccess) return dense_status(e);
    }
    return EXACT_OK;
}

}  // extern "C"
