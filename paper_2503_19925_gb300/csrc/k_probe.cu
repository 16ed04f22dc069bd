// k_probe.cu -- measurement aid (no counterpart in the paper): the rate at which
// this GPU serves 4-byte shared-memory gathers, the ceiling the projector
// kernels are held against.
//
// Both projector kernels are sparse gathers whose operands come from shared
// memory or L1 (forward: staged image bands; adjoint: per-lane accumulators
// and the L1-cached residual), so their bound is the L1/shared data path, one
// 128-byte wavefront (32 words) per SM per clock, not HBM.  k_probe_gather
// issues nothing but conflict-free shared loads (lane l of every warp reads
// bank l of a row that changes every load) with one dependent add each, enough
// warps per SM to cover the load latency, and no global traffic inside the
// timed loop; its words per second measure that ceiling on the device at hand.
#include "exact_internal.h"

namespace exact {
namespace {

constexpr int kProbeRows = 128;   // shared rows of 32 words (16 KB)
constexpr int kProbeUnroll = 16;  // loads per loop trip (immediate offsets)
constexpr int kProbeThreads = 256;

__device__ float g_probe_sink;

__global__ void __launch_bounds__(kProbeThreads) k_probe_gather(int trips)
{
    __shared__ float buf[kProbeRows * 32];
    for (int i = threadIdx.x; i < kProbeRows * 32; i += kProbeThreads) buf[i] = (float)(i & 7) * 0.125f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // base row in [0, 64); the unrolled loads reach at most 63 rows further
    int row = (threadIdx.x >> 5) * 5 & 63;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t = 0; t < trips; ++t) {
        const float *p = buf + row * 32 + lane;
#pragma unroll
        for (int k = 0; k < kProbeUnroll; ++k) acc[k & 3] += p[32 * ((k * 37) & 63)];
        row = (row + 13) & 63;
    }
    const float s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    if (s == -1.0f) g_probe_sink = s;  // never true (the sum is >= 0): keeps the loads
}

}  // namespace
}  // namespace exact

using namespace exact;

extern "C" {

exact_status exact_probe_gather_ceiling(double *words_per_s, int *sm_count, exact_stream_t stream)
{
    if (!words_per_s) return EXACT_ERR_INVALID_ARG;
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EXACT_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return EXACT_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_probe_gather, kProbeThreads, 0) != cudaSuccess ||
        per <= 0)
        return EXACT_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = sms * per;  // one full wave: every SM busy for the whole launch
    const int trips = 4096;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    exact_status st = EXACT_OK;
    float best_ms = 0.0f;
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
        st = EXACT_ERR_CUDA;
    } else {
        k_probe_gather<<<grid, kProbeThreads, 0, s>>>(trips);  // warm-up
        for (int rep = 0; rep < 5 && st == EXACT_OK; ++rep) {
            float ms = 0.0f;
            if (cudaEventRecord(ev[0], s) != cudaSuccess) st = EXACT_ERR_CUDA;
            k_probe_gather<<<grid, kProbeThreads, 0, s>>>(trips);
            if (cudaGetLastError() != cudaSuccess || cudaEventRecord(ev[1], s) != cudaSuccess ||
                cudaEventSynchronize(ev[1]) != cudaSuccess || cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess)
                st = EXACT_ERR_CUDA;
            else if (rep == 0 || ms < best_ms)
                best_ms = ms;
        }
    }
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (st != EXACT_OK) return st;
    if (!(best_ms > 0.0f)) return EXACT_ERR_CUDA;
    const double words = (double)grid * kProbeThreads * (double)trips * kProbeUnroll;
    *words_per_s = words / (best_ms * 1e-3);
    if (sm_count) *sm_count = sms;
    return EXACT_OK;
}

}  // extern "C"
