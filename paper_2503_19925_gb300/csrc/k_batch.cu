// k_batch.cu -- persistent multi-job kernel: many EXACT reconstructions of
// uneven image size, view count and window count advance together in one
// launch.
//
// Work items.  A round of job j is one extragradient iteration (Eq. (11)) in
// five phases: forward+link on x_t (one item per forward work unit), adjoint
// half step (one item per 16x16 tile), forward+link on x_{t+1/2}, adjoint full
// step, and the FP64 stopping reduction (one item).  Items are handed out in a
// fixed global order -- round-major, then phase, then job, then item -- by an
// atomic counter; every CTA loops: take the next item, wait until all items
// of the previous phase of the same job are done, run the item with the shared
// device bodies of joseph.cuh, count it done.
//
// Progress.  An item only waits for items of its own job that come earlier in
// the global order; those were taken earlier by CTAs that are running, so the
// earliest unfinished item never waits and the launch always completes.  Each
// wait is a bounded spin: when it runs out the CTA raises the launch's abort
// flag and the job's EXACT_ERR_TIMEOUT status, and every CTA leaves at its next
// item.
//
// Memory ordering.  A finished item's writes are published by
// __syncthreads + __threadfence + atomicAdd on the job's done counter; the
// waiting thread acquires the counter, fences, and the CTA synchronises before
// use.  Data that other CTAs rewrite during the launch (residuals, iterates,
// partial norms, job state) is read with L2-coherent loads, and tensor-map
// copies are preceded by a proxy fence.
//
// Per item the arithmetic is fixed (same kernels, same warp count, same
// summation order), so a job's result does not depend on what else is in the
// batch.
#include "joseph.cuh"

namespace exact {

namespace {

constexpr int kBG = kBatchThreads / 32;  // adjoint warps per batch CTA
static_assert(kBatchThreads == kFR, "one forward unit per batch CTA");
constexpr long long kDepSpins = 1LL << 26;  // bounded dependency wait (with back-off)

struct __align__(128) BatchSmem {
    union {
        FwdSmem fwd;
        AdjSmem<kBG> adj;
    } u;
    uint64_t bar[kFStages];
    unsigned long long item;
    int ok;
    int go;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *reinterpret_cast<const volatile int *>(p); }

// Fixed-order reduction of a job's partial norms into its state (kBatchThreads
// threads; the same arithmetic as k_solve_reduce with a different block size).
__device__ void batch_reduce(const BatchJob &J, int iter, double *scratch)
{
    const int nparts = J.tiles_x * J.tiles_y;
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kBatchThreads) {
        s0 += __ldcg(J.a.partials + kPartStride * i);
        s1 += __ldcg(J.a.partials + kPartStride * i + 1);
    }
    scratch[threadIdx.x] = s0;
    scratch[kBatchThreads + threadIdx.x] = s1;
    __syncthreads();
    for (int w = kBatchThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            scratch[threadIdx.x] += scratch[threadIdx.x + w];
            scratch[kBatchThreads + threadIdx.x] += scratch[kBatchThreads + threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        DevState *st = J.state;
        const double rel = sqrt(scratch[0]) / fmax(sqrt(scratch[kBatchThreads]), 1e-30);
        st->rel_res = rel;
        st->iters_done = iter + 1;
        if (!isfinite(rel)) {
            st->status = EXACT_ERR_NONFINITE;
            st->done = 1;
        } else if (J.tol > 0.0 && J.check_every > 0 && (iter + 1) % J.check_every == 0 && rel <= J.tol) {
            st->done = 1;
        }
    }
}

__global__ void __launch_bounds__(kBatchThreads, 6) k_batch(const BatchJob *__restrict__ jobs, int n_jobs,
                                                         const int *__restrict__ prefix_g, int rounds,
                                                         unsigned long long *next, unsigned *done_items,
                                                         int *abort_flag, long long dep_polls)
{
    __shared__ BatchSmem sm;
    const int t = threadIdx.x;
    const int nseg = 5 * n_jobs;
    if (t == 0) {
        for (int q = 0; q < kFStages; ++q) mbar_init(&sm.bar[q]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const unsigned long long per_round = (unsigned long long)__ldg(prefix_g + nseg);
    const unsigned long long total = per_round * (unsigned long long)rounds;
    uint32_t fphase = 0u;  // staging-barrier parities of the forward items

    for (;;) {
        if (t == 0) sm.item = atomicAdd(next, 1ULL);
        __syncthreads();
        const unsigned long long item = sm.item;
        if (item >= total) break;
        const int round = (int)(item / per_round);
        const int rem = (int)(item - (unsigned long long)round * per_round);
        // segment s = (phase, job) with prefix[s] <= rem < prefix[s + 1]
        int lo = 0, hi = nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(prefix_g + mid) <= rem) lo = mid;
            else hi = mid - 1;
        }
        const int phase = lo / n_jobs, j = lo - phase * n_jobs;
        const int local = rem - __ldg(prefix_g + lo);
        const BatchJob &J = jobs[j];

        if (t == 0) {
            // (a held job's later phases wait for more completions than it has items)
            const unsigned need = (phase >= 1 && J.hold)
                                      ? J.hold
                                      : (unsigned)round * (unsigned)J.phase_off[5] + (unsigned)J.phase_off[phase];
            int ok = ld_volatile(abort_flag) ? 0 : 1;
            long long spins = 0;
            while (ok && ld_acquire(done_items + j) < need) {
                if (ld_volatile(abort_flag) || ++spins > dep_polls) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
            if (!ok) {
                if (!ld_volatile(abort_flag) && spins > dep_polls) {
                    J.state->status = EXACT_ERR_TIMEOUT;
                    J.state->done = 1;
                    atomicExch(abort_flag, 1);
                }
            }
            __threadfence();
            sm.ok = ok;
            sm.go = ok && round < J.iters && !ld_volatile(&J.state->done);
        }
        __syncthreads();
        if (!sm.ok) break;
        if (sm.go) {
            bool item_ok = true;
            if (phase == 0 || phase == 2) {
                const int q = phase >> 1;
                FwdArgs f = J.f;
                f.img = J.img[q];
                item_ok = forward_unit<true, true>(f, local, J.maps + 2 * q, J.maps + 2 * q + 1, J.coef, sm.u.fwd,
                                                   sm.bar, fphase);
            } else if (phase == 1 || phase == 3) {
                AdjArgs a = J.a;
                a.iter = round;
                // item = (tile, split index): the tile's split CTAs combine
                const int ns = J.nsplit > 1 ? J.nsplit : 1;
                const int tile = local / ns, zsp = local - tile * ns;
                const int bx = tile % J.tiles_x, by = tile / J.tiles_x;
                if (by >= J.tiles_y) {  // a damaged item table: report and touch nothing
                    if (t == 0) {
                        J.state->status = EXACT_ERR_INVALID_ARG;
                        J.state->done = 1;
                    }
                } else if (phase == 1) {
                    a.out_r = J.xr[1];
                    a.out_c = J.xc[1];
                    if (J.fan) adjoint_tile<ADJ_EG, true, false, kBG, true>(a, bx, by, tile, sm.u.adj, zsp);
                    else adjoint_tile<ADJ_EG, false, false, kBG, true>(a, bx, by, tile, sm.u.adj, zsp);
                } else {
                    a.out_r = J.xr[0];
                    a.out_c = J.xc[0];
                    if (J.fan) adjoint_tile<ADJ_EG_FINAL, true, false, kBG, true>(a, bx, by, tile, sm.u.adj, zsp);
                    else adjoint_tile<ADJ_EG_FINAL, false, false, kBG, true>(a, bx, by, tile, sm.u.adj, zsp);
                }
            } else {
                batch_reduce(J, round, reinterpret_cast<double *>(&sm.u));
            }
            if (!item_ok) {
                if (t == 0) atomicExch(abort_flag, 1);
                break;
            }
        }
        __syncthreads();
        if (t == 0) {
            __threadfence();
            atomicAdd(done_items + j, 1u);
        }
    }
}

}  // namespace

int batch_grid_size()
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch, kBatchThreads, 0);
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_batch(const BatchJob *jobs, int n_jobs, const int *prefix, int rounds, unsigned long long *next,
                         unsigned *done_items, int *abort_flag, int grid, long long dep_polls, cudaStream_t s)
{
    if (n_jobs <= 0 || rounds <= 0) return cudaSuccess;
    k_batch<<<grid, kBatchThreads, 0, s>>>(jobs, n_jobs, prefix, rounds, next, done_items, abort_flag,
                                           dep_polls > 0 ? dep_polls : kDepSpins);
    return cudaGetLastError();
}

}  // namespace exact
