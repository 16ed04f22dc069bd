// k_adjoint.cu -- adjoint g = A^T r of the Joseph projector of k_forward.cu,
// as a deterministic gather (fixed summation order, no atomics), with the
// fused extragradient epilogue of Eq. (11) and the FP64 partial norms of the
// stopping rule.
//
// FP32 kernel (hot path): one CTA owns a tile of kTW x kTH pixels; its kG warps
// split the views (warp g takes views g, g + kG, ...; interleaving keeps the
// warps' loads even).  For each view a warp walks the rays that cross the tile:
//   - x-driven rays sample every pixel column; lane l owns column tx0 + l and
//     walks, in bin order, the rays whose crossing with that column lies
//     strictly inside (ty0 - 1, ty0 + kTH).  Each ray adds (1 - f) r and f r
//     to the two pixels around its crossing (the two nonzero entries of its
//     row of A in this column);
//   - y-driven rays sample every pixel row; lane l owns a segment of a row
//     (row ty0 + l % kTH, kTH columns starting at tx0 + kTH (l / kTH)) and
//     walks its rays the same way.
// The rays crossing a strip form one contiguous bin range: the two end points
// of the strip projected onto the detector (a ratio of affine forms of the
// pixel coordinates, stored per view) bound it.  Each lane accumulates into
// its own column of a warp-private shared-memory array (bank = lane: no
// conflicts, no races); at the end the CTA adds the kG warps' arrays in warp
// order.  Every output is therefore the same fixed-order sum on every run.
//
// Ray coordinates use the split FP32 form of k_forward.cu: u = t(j) - k_base is
// formed with an exact product split (fmaf) and an exact cancellation of the
// large terms, so the interpolation weights match the FP64 matrix to ~1e-6 and
// the gather is the transpose of the forward walk up to FP32 rounding.
//
// FP64 kernel (power iteration, once per plan): one thread per pixel loops over
// the views and evaluates the few candidate rays of each view directly.
#include "exact_internal.h"

namespace exact {

namespace {

constexpr float kBinEps = 0.01f;

// ---------------------------------------------------------------- FP32 strip walk

constexpr int kTW = 32;        // tile width (pixels) = lanes of a warp
constexpr int kTH = 8;         // tile height = strip length of both walks
constexpr int kG = 6;          // warps per CTA (view subsets)
constexpr int kRows = kTH + 2; // accumulator rows: strip offsets -1 .. kTH
constexpr int kSeg = kTW / kTH; // y-driven lanes: kSeg segments of kTH columns per row
static_assert(kTW % kTH == 0, "y-driven lanes split a tile row into whole segments");

// Bin range of the rays that cross the segment between two points whose
// detector projections are (num1/den1, num2/den2) + c, within [lo_bin, hi_bin).
template <bool FAN>
__device__ __forceinline__ void seg_range(float num1, float den1, float num2, float den2, float c, int lo_bin,
                                          int hi_bin, int &b0, int &b1)
{
    const float u1 = FAN ? __fdividef(num1, den1) : num1;
    const float u2 = FAN ? __fdividef(num2, den2) : num2;
    float lo = fminf(u1, u2) + c - kBinEps;
    float hi = fmaxf(u1, u2) + c + kBinEps;
    lo = fminf(fmaxf(lo, -1.0f), (float)hi_bin);
    hi = fminf(fmaxf(hi, -1.0f), (float)hi_bin);
    b0 = max(lo_bin, (int)ceilf(lo));
    b1 = min(hi_bin - 1, (int)floorf(hi));
}

// Walk rays b0..b1 of one view at driving index jf; deposit into acc rows
// k + 1 and k + 2 (strip offset k = floor(t - kbase) in [-1, kTH - 1]).
template <bool DELTA>
__device__ __forceinline__ void strip_walk(const RayF *__restrict__ vrays, const float *__restrict__ vres,
                                           const float *__restrict__ vdelta, int b0, int b1, float jf, float kbase,
                                           float *__restrict__ acc, int lane)
{
    for (int b = b0; b <= b1; ++b) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(vrays + b));
        const RayF rec = {q.x, q.y, q.z, q.w};
        float rv = __ldg(vres + b);
        if (DELTA) rv *= __ldg(vdelta + b);
        const float p = rec.bh * jf;
        const float e = fmaf(rec.bh, jf, -p);
        const float u = ((rec.A - kbase) + p) + (rec.a + fmaf(rec.bl, jf, e));
        // floor(u) without the conversion pipe (|u| < 2^22)
        const float r = __fadd_rd(u, kFloorMagic);
        const float f = u - (r - kFloorMagic);
        const int k = __float_as_int(r) - kFloorBias;
        if (k >= -1 && k < kTH) {
            const float w1 = f * rv;
            acc[(k + 1) * kTW + lane] += rv - w1;
            acc[(k + 2) * kTW + lane] += w1;
        }
    }
}

template <int MODE, bool FAN, bool DELTA>
__global__ void __launch_bounds__(kG * 32, 8) k_adjoint(AdjArgs a)
{
    if (a.state && a.state->done) return;
    extern __shared__ float smem[];
    __shared__ float stage[kTH][kTW + 1];
    __shared__ float tile[kTH][kTW + 1];
    __shared__ double red0[kG], red1[kG];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    float *accx = smem + g * (2 * kRows * kTW);
    float *accy = accx + kRows * kTW;
    for (int r = 0; r < kRows; ++r) {
        accx[r * kTW + lane] = 0.0f;
        accy[r * kTW + lane] = 0.0f;
    }
    const int tx0 = blockIdx.x * kTW, ty0 = blockIdx.y * kTH;
    // x-driven strip of this lane: column cx, rows ty0 .. ty0 + kTH - 1
    const int cx = tx0 + lane;
    const bool xok = cx < a.nx;
    // strip end points, kept within one pixel of the image so that their
    // fan-beam projections stay well defined (the source is outside the image)
    const float fcx = (float)cx, fy_lo = (float)(ty0 - 1), fy_hi = (float)min(ty0 + kTH, a.ny);
    // y-driven strip of this lane: row ry, columns cy0 .. cy0 + kTH - 1
    const int ry = ty0 + (lane % kTH);
    const int cy0 = tx0 + kTH * (lane / kTH);
    const bool yok = ry < a.ny && cy0 < a.nx;
    const float fry = (float)ry, fx_lo = (float)(cy0 - 1), fx_hi = (float)min(cy0 + kTH, a.nx);

    for (int v = g; v < a.n_views; v += kG) {
        const ViewRec vr = a.views[v];
        const long long vb = (long long)v * a.n_bins;
        const RayF *vrays = a.rays + vb;
        const float *vres = a.r + vb;
        const float *vdel = DELTA ? a.delta + vb : nullptr;
        if (vr.xb1 > vr.xb0 && xok) {
            const float nb = fmaf(vr.n1, fcx, vr.n0), db = fmaf(vr.d1, fcx, vr.d0);
            int b0, b1;
            seg_range<FAN>(fmaf(vr.n2, fy_lo, nb), fmaf(vr.d2, fy_lo, db), fmaf(vr.n2, fy_hi, nb),
                           fmaf(vr.d2, fy_hi, db), vr.c, vr.xb0, vr.xb1, b0, b1);
            strip_walk<DELTA>(vrays, vres, vdel, b0, b1, fcx, (float)ty0, accx, lane);
        }
        if (vr.yb1 > vr.yb0 && yok) {
            const float nb = fmaf(vr.n2, fry, vr.n0), db = fmaf(vr.d2, fry, vr.d0);
            int b0, b1;
            seg_range<FAN>(fmaf(vr.n1, fx_lo, nb), fmaf(vr.d1, fx_lo, db), fmaf(vr.n1, fx_hi, nb),
                           fmaf(vr.d1, fx_hi, db), vr.c, vr.yb0, vr.yb1, b0, b1);
            strip_walk<DELTA>(vrays, vres, vdel, b0, b1, fry, (float)cy0, accy, lane);
        }
    }
    __syncthreads();

    // fixed-order reduction over the warps: the y-driven parts first, staged
    // transposed (row stride kTW + 1), then the x-driven parts
    for (int t = threadIdx.x; t < kTH * kTW; t += kG * 32) {
        const int l = t % kTW, k = t / kTW;  // accy column l, strip offset k
        float s = 0.0f;
        for (int q = 0; q < kG; ++q) s += smem[q * (2 * kRows * kTW) + kRows * kTW + (k + 1) * kTW + l];
        stage[l % kTH][kTH * (l / kTH) + k] = s;
    }
    __syncthreads();
    double s0 = 0.0, s1 = 0.0;
    for (int t = threadIdx.x; t < kTH * kTW; t += kG * 32) {
        const int px = t % kTW, py = t / kTW;
        float gsum = stage[py][px];
        for (int q = 0; q < kG; ++q) gsum += smem[q * (2 * kRows * kTW) + (py + 1) * kTW + px];
        const int kx = tx0 + px, ky = ty0 + py;
        const bool inside = kx < a.nx && ky < a.ny;
        if (MODE == ADJ_PLAIN) {
            if (inside) a.out[(long long)ky * a.nx + kx] = a.scale * gsum;
        } else {
            const long long pr = (long long)ky * a.ldr + kx + kPad;
            const float xb = inside ? a.base_r[pr] : 0.0f;
            // projection onto [lo, hi] that keeps a NaN (so the stopping rule sees it)
            const float step = fmaf(a.scale, gsum, xb);
            const float xn = inside ? (step < a.lo ? a.lo : (step > a.hi ? a.hi : step)) : 0.0f;
            if (inside) a.out_r[pr] = xn;
            tile[py][px] = xn;
            if (MODE == ADJ_EG_FINAL && inside) {
                if (a.avg && a.iter >= a.avg_from) a.avg[(long long)ky * a.nx + kx] += (double)xn;
                const double dd = (double)xn - (double)xb;
                s0 += dd * dd;
                s1 += (double)xb * (double)xb;
            }
        }
    }
    if (MODE == ADJ_PLAIN) return;
    __syncthreads();
    // column-major copy: kTH consecutive ky per kx row
    for (int t = threadIdx.x; t < kTH * kTW; t += kG * 32) {
        const int col = t / kTH, row = t % kTH;
        const int ox = tx0 + col, oy = ty0 + row;
        if (ox < a.nx && oy < a.ny) a.out_c[(long long)ox * a.ldc + oy + kPad] = tile[row][col];
    }
    if (MODE == ADJ_EG_FINAL) {
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_down_sync(0xffffffffu, s0, o);
            s1 += __shfl_down_sync(0xffffffffu, s1, o);
        }
        if (lane == 0) {
            red0[g] = s0;
            red1[g] = s1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t0 = 0.0, t1 = 0.0;
            for (int q = 0; q < kG; ++q) {
                t0 += red0[q];
                t1 += red1[q];
            }
            const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
            a.partials[2 * blk] = t0;
            a.partials[2 * blk + 1] = t1;
        }
    }
}

constexpr size_t kAdjSmem = sizeof(float) * kG * 2 * kRows * kTW;

template <int MODE, bool FAN, bool DELTA>
cudaError_t launch_adj(const AdjArgs &a, cudaStream_t s)
{
    const dim3 grid((a.nx + kTW - 1) / kTW, (a.ny + kTH - 1) / kTH);
    k_adjoint<MODE, FAN, DELTA><<<grid, kG * 32, kAdjSmem, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- FP64 pixel gather

constexpr int DX = 32, DY = 8;

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

// FP64 entry of A: delta (1 - |t - k|)_+ with t = fma(beta, j, alpha).
__device__ __forceinline__ double entry_d(const RayD &rec, double jf, double kc)
{
    const double u = fma(rec.beta, jf, rec.alpha) - kc;
    return fmax(0.0, 1.0 - fabs(u)) * rec.delta;
}

template <bool FAN>
__device__ __forceinline__ double gather_pixel_d(const RayD *__restrict__ rays, const ViewRec *__restrict__ views,
                                                 const double *__restrict__ r, int n_views, int n_bins, int kx,
                                                 int ky)
{
    const float fx = (float)kx, fy = (float)ky;
    const double tx = (double)kx, ty = (double)ky;
    double acc = 0.0;
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
            for (int b = b0; b <= b1; ++b) acc = fma(entry_d(rays[vb + b], tx, ty), r[vb + b], acc);
        }
        if (vr.yb1 > vr.yb0) {  // y-driven rays sample row ky
            int b0, b1;
            bin_range<FAN>(num, den, vr.n1, vr.d1, vr.c, n_bins, b0, b1);
            b0 = max(b0, vr.yb0);
            b1 = min(b1, vr.yb1 - 1);
            for (int b = b0; b <= b1; ++b) acc = fma(entry_d(rays[vb + b], ty, tx), r[vb + b], acc);
        }
    }
    return acc;
}

// FP64 adjoint of the power iteration: w = A^T z into both padded copies,
// plus per-block partial sums of ||w||^2 (fixed order).
template <bool FAN>
__global__ void __launch_bounds__(DX *DY) k_adjoint_d(const RayD *rays, const ViewRec *views, int n_views,
                                                     int n_bins, int nx, int ny, const double *zd, double *xrd,
                                                     double *xcd, long long ldr, long long ldc,
                                                     double *partials, const DevState *st)
{
    if (st->done) return;
    const int kx = blockIdx.x * DX + threadIdx.x;
    const int ky = blockIdx.y * DY + threadIdx.y;
    const bool inside = kx < nx && ky < ny;
    double w = 0.0;
    if (inside) {
        w = gather_pixel_d<FAN>(rays, views, zd, n_views, n_bins, kx, ky);
        xrd[(long long)ky * ldr + kx + kPad] = w;
        xcd[(long long)kx * ldc + ky + kPad] = w;
    }
    double s = w * w;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double sw[DX * DY / 32];
    const int tid = threadIdx.y * DX + threadIdx.x;
    if ((tid & 31) == 0) sw[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int q = 0; q < DX * DY / 32; ++q) t += sw[q];
        partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

}  // namespace

int adjoint_blocks(int nx, int ny) { return ((nx + kTW - 1) / kTW) * ((ny + kTH - 1) / kTH); }

int adjoint_d_blocks(int nx, int ny) { return ((nx + DX - 1) / DX) * ((ny + DY - 1) / DY); }

cudaError_t launch_adjoint(const AdjArgs &a, int mode, bool fan, cudaStream_t s)
{
    const bool delta = a.delta != nullptr;
    if (mode == ADJ_PLAIN) {
        if (fan) return delta ? launch_adj<ADJ_PLAIN, true, true>(a, s) : launch_adj<ADJ_PLAIN, true, false>(a, s);
        return delta ? launch_adj<ADJ_PLAIN, false, true>(a, s) : launch_adj<ADJ_PLAIN, false, false>(a, s);
    }
    if (mode == ADJ_EG) return fan ? launch_adj<ADJ_EG, true, false>(a, s) : launch_adj<ADJ_EG, false, false>(a, s);
    return fan ? launch_adj<ADJ_EG_FINAL, true, false>(a, s) : launch_adj<ADJ_EG_FINAL, false, false>(a, s);
}

cudaError_t launch_adjoint_d(const RayD *rays, const ViewRec *views, int n_views, int n_bins, int nx, int ny,
                             const double *zd, double *xrd, double *xcd, long long ldr, long long ldc,
                             double *partials, DevState *st, bool fan, cudaStream_t s)
{
    const dim3 block(DX, DY);
    const dim3 grid((nx + DX - 1) / DX, (ny + DY - 1) / DY);
    if (fan)
        k_adjoint_d<true><<<grid, block, 0, s>>>(rays, views, n_views, n_bins, nx, ny, zd, xrd, xcd, ldr, ldc,
                                                 partials, st);
    else
        k_adjoint_d<false><<<grid, block, 0, s>>>(rays, views, n_views, n_bins, nx, ny, zd, xrd, xcd, ldr, ldc,
                                                  partials, st);
    return cudaGetLastError();
}

}  // namespace exact
