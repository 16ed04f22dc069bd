// k_adjoint.cu -- adjoint g = A^T r of the Joseph projector of k_forward.cu,
// as a deterministic gather (fixed summation order, no atomics), with the
// fused extragradient epilogue of Eq. (11) and the per-tile FP64 partial norms
// of the stopping rule (FP32 within a thread's few pixels).
//
// FP32 kernel (hot path, body in joseph.cuh): one CTA owns a tile of kTW x kTH
// (32 x 32) pixels and, with a view split, one of its nsplit view subsets.  Its
// kG warps take one view at a time from the plan's view lists, in two phases:
//   - x-driven rays sample every pixel column; lane l owns column tx0 + l and
//     walks, in bin order, the rays whose crossing with that column lies
//     strictly inside (ty0 - 1, ty0 + kTH).  Each ray adds (1 - f) r and f r
//     to the two pixels around its crossing (the two nonzero entries of its
//     row of A in this column);
//   - then the views with y-driven rays: lane l owns row ty0 + l and walks its
//     rays the same way.
// Warp g of split z takes items z kG + g + k kG nsplit of each list, so the
// splits interleave over the views.  Fan beams walk line pairs instead: lane l
// owns lines 2 (l % 16) and the next over half l / 16 of the strip, so one
// step along a ray (its residual, its reciprocal) serves two crossings.
// The rays crossing a strip form one contiguous bin range: the two end points
// of the strip projected onto the detector (a ratio of affine forms of the
// pixel coordinates, stored per view) bound it.  Each lane accumulates into
// its own column of a warp-private [kTH + 2][32] shared-memory array (bank =
// lane: no conflicts, no races); after each phase the CTA adds the warps'
// arrays into the tile in a fixed order (the y phase transposed).  With a view
// split, the last of a tile's CTAs adds the partial tiles in split order.
// Every output is therefore the same fixed-order sum on every run.
//
// Ray coordinates: the crossing of the middle ray of a walk comes from the
// split FP32 record of k_forward.cu (exact product split, exact cancellation
// of the large terms); the other rays of the walk follow from per-ray walk
// coefficients, t_{b+e} = t_b + kappa e / (1 + sg e) (exact for both beams:
// the crossing is a Moebius function of the bin index), so a step reads one
// residual and no ray record, and costs one hardware reciprocal.  The
// interpolation weights match the FP64 matrix to ~1e-6 and the gather is the
// transpose of the forward walk up to FP32 rounding (its crossings agree with
// the forward's per-line anchors to ~1e-6 pixel, not bit for bit).
//
// FP64 kernel (power iteration, once per plan): one thread per pixel loops over
// the views and evaluates the few candidate rays of each view directly.
#include "joseph.cuh"

namespace exact {

namespace {

constexpr int kG = 8;  // warps per CTA of the per-plan kernel (one view at a time each)

template <int MODE, bool FAN, bool DELTA>
__global__ void __launch_bounds__(kG * 32, 5) k_adjoint(AdjArgs a)
{
    if (a.state && a.state->done) return;
    extern __shared__ __align__(16) unsigned char adj_smem[];
    AdjSmem<kG> &sm = *reinterpret_cast<AdjSmem<kG> *>(adj_smem);
    adjoint_tile<MODE, FAN, DELTA, kG, false>(a, blockIdx.x, blockIdx.y,
                                              (long long)blockIdx.y * gridDim.x + blockIdx.x, sm, blockIdx.z);
}

template <int MODE, bool FAN, bool DELTA>
cudaError_t launch_adj(const AdjArgs &a, cudaStream_t s)
{
    const dim3 grid((a.nx + kTW - 1) / kTW, (a.ny + kTH - 1) / kTH, a.nsplit > 1 ? a.nsplit : 1);
    k_adjoint<MODE, FAN, DELTA><<<grid, kG * 32, sizeof(AdjSmem<kG>), s>>>(a);
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
    if (mode == ADJ_STEP)
        return fan ? launch_adj<ADJ_STEP, true, false>(a, s) : launch_adj<ADJ_STEP, false, false>(a, s);
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
