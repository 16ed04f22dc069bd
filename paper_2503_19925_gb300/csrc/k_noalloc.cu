// k_noalloc.cu -- exact_operator_static: the operator F(x) for callers that
// cannot allocate device memory.
//
// exact_operator needs scratch memory (the collapsed counts, the padded row- and
// column-major copies of x and the residual) and takes it from the workspace
// the caller allocated and bound to the plan.  Some callers cannot make that
// allocation at the time they need F: an allocator-free real-time or embedded
// loop that must not stall on cudaMalloc, or a process whose device memory is
// owned by another framework's pool.  This entry point instead uses
// one file-scope device array of kStaticScratchBytes as scratch and allocates
// nothing.  The array exists once per device that loads this library and
// stays until the process exits.
//
// Host code cannot pass the array's name to a kernel (in host code it is a
// stand-in, not a device address), so the first call on each device, with that
// device current, asks the runtime for the array's device address
// (cudaGetSymbolAddress) and keeps it; that first call should therefore come
// before any stream capture.  The kept address belongs to the device's primary
// context: after cudaDeviceReset (or any other teardown of that context) it is
// stale, so the entry point must not be used again in that process.
//
// All calls share the array and it keeps the last call's contents: every
// scratch word a call reads is first written by the same call (the padded
// copies are written whole, pads and alignment tails included), so nothing
// needs clearing, but calls that overlap on the GPU (different streams, or
// different plans at once) race on it.  The adjoint runs one CTA per tile
// (the plan's adj_split is not used: its partial tiles live in the workspace),
// so F equals exact_operator's up to the FP32 summation order of a split.
#include "joseph.cuh"

#include <mutex>
#include <string.h>

namespace exact {
namespace {

constexpr size_t kStaticScratchBytes = size_t(EXACT_STATIC_SCRATCH_MB) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_lock;
void *g_scratch_ptr[kMaxDevices] = {};

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Device address of g_scratch on the current device (set up once per device).
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

exact_status status_of(cudaError_t e)
{
    if (e == cudaSuccess) return EXACT_OK;
    return e == cudaErrorMemoryAllocation ? EXACT_ERR_OOM : EXACT_ERR_CUDA;
}

}  // namespace
}  // namespace exact

using namespace exact;

extern "C" {

exact_status exact_operator_static(exact_plan_t plan, const float *x, const void *y, exact_dtype y_dtype, double I0,
                                   float *F, exact_stream_t stream)
{
    if (!plan || !x || !y || !F) return EXACT_ERR_INVALID_ARG;
    if (y_dtype != EXACT_F32 && y_dtype != EXACT_BF16) return EXACT_ERR_INVALID_ARG;
    if (!(I0 > 0.0) || !(I0 < INFINITY)) return EXACT_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return EXACT_ERR_CUDA;
    if (dev != P.device) return EXACT_ERR_INVALID_ARG;

    // scratch layout: padded row-major copy, padded column-major copy,
    // collapsed counts, residual
    const size_t b_xr = up256(sizeof(float) * (size_t)(P.g.ny * P.ldr()));
    const size_t b_xc = up256(sizeof(float) * (size_t)(P.g.nx * P.ldc()));
    const size_t b_n = up256(sizeof(float) * (size_t)P.n);
    if (b_xr + b_xc + 2 * b_n > kStaticScratchBytes) return EXACT_ERR_UNSUPPORTED;  // plan too large
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return status_of(e);
    char *sp = static_cast<char *>(base);
    float *xr = reinterpret_cast<float *>(sp);
    float *xc = reinterpret_cast<float *>(sp + b_xr);
    float *Y = reinterpret_cast<float *>(sp + b_xr + b_xc);
    float *r = reinterpret_cast<float *>(sp + b_xr + b_xc + b_n);
    CUtensorMap map_r, map_c;
    if (!encode_map(&map_r, xr, P.ldr(), P.g.ny) || !encode_map(&map_c, xc, P.ldc(), P.g.nx))
        return EXACT_ERR_CUDA;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const LinkCoef coef = make_coef(P, I0);
    if ((e = launch_collapse(y, y_dtype, P.W, P.n, Y, s)) != cudaSuccess) return status_of(e);
    if ((e = launch_pack(x, xr, xc, P.g.nx, P.g.ny, P.ldr(), P.ldc(), 0.f, 0.f, false, s)) != cudaSuccess)
        return status_of(e);
    FwdArgs f;
    memset(&f, 0, sizeof(f));
    f.img.xr = xr;
    f.img.xc = xc;
    f.img.nx = P.g.nx;
    f.img.ny = P.g.ny;
    f.img.ldr = P.ldr();
    f.img.ldc = P.ldc();
    f.rays = P.rays_f;
    f.bits = P.ray_bits;
    f.delta = P.ray_delta;
    f.units = P.units;
    f.kstart = P.kstart;
    f.n_units = P.n_units;
    f.n = P.n;
    f.Y = Y;
    f.r = r;
    f.K = P.K;
    f.M = P.bg_M;
    f.bg = P.bg_p;
    if ((e = launch_forward(f, true, &coef, map_r, map_c, s)) != cudaSuccess) return status_of(e);
    AdjArgs a;
    memset(&a, 0, sizeof(a));
    a.rays = P.rays_f;
    a.walk = P.rays_w;
    adj_views(a, P);
    a.n_views = P.g.n_views;
    a.n_bins = P.g.n_bins;
    a.nx = P.g.nx;
    a.ny = P.g.ny;
    a.r = r;
    a.scale = (float)(1.0 / ((double)P.W * (double)P.n));
    a.out = F;
    // nsplit stays 0: one CTA per adjoint tile whatever the plan's adj_split,
    // as the split's partial tiles and arrival counts live in the workspace
    if ((e = launch_adjoint(a, ADJ_PLAIN, P.g.beam == 1, s)) != cudaSuccess) return status_of(e);
    return EXACT_OK;
}

}  // extern "C"
