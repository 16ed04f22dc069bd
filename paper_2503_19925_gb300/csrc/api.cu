// api.cu -- the C ABI of include/exact.h: plan construction (ray and view
// tables built in FP64 on the host), workspace carve-up, and the entry points
// that enqueue the kernels of k_forward.cu, k_adjoint.cu and k_util.cu.
#include "exact_internal.h"

#include <algorithm>
#include <map>
#include <atomic>
#include <mutex>
#include <thread>

#include <climits>
#include <cudaTypedefs.h>
#include <math.h>
#include <new>
#include <string.h>
#include <vector>

using namespace exact;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool isfin(double v) { return isfinite(v) != 0; }

exact_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return EXACT_OK;
    if (e == cudaErrorMemoryAllocation) return EXACT_ERR_OOM;
    return EXACT_ERR_CUDA;
}

#define EXACT_TRY(expr)                                      \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return cuda_status(_e);       \
    } while (0)

exact_status check_geometry(const exact_geometry *g)
{
    if (!g) return EXACT_ERR_INVALID_ARG;
    if (g->beam != 0 && g->beam != 1) return EXACT_ERR_INVALID_ARG;
    if (g->nx < 1 || g->ny < 1 || g->nx > 16384 || g->ny > 16384) return EXACT_ERR_INVALID_ARG;
    if (g->n_views < 1 || g->n_bins < 1) return EXACT_ERR_INVALID_ARG;
    if ((long long)g->n_views * (long long)g->n_bins > 2147483647LL) return EXACT_ERR_INVALID_ARG;
    if (!isfin(g->pixel) || !(g->pixel > 0.0)) return EXACT_ERR_INVALID_ARG;
    if (!isfin(g->bin_pitch) || !(g->bin_pitch > 0.0)) return EXACT_ERR_INVALID_ARG;
    if (!isfin(g->angle0) || !isfin(g->angle_range) || !isfin(g->det_offset)) return EXACT_ERR_INVALID_ARG;
    if (g->beam == 1) {
        const double half_diag = 0.5 * g->pixel * sqrt((double)g->nx * g->nx + (double)g->ny * g->ny);
        if (!isfin(g->src_to_center) || !isfin(g->src_to_det)) return EXACT_ERR_INVALID_ARG;
        if (!(g->src_to_center > half_diag + 2.0 * g->pixel)) return EXACT_ERR_INVALID_ARG;
        if (!(g->src_to_det > g->src_to_center)) return EXACT_ERR_INVALID_ARG;
    }
    return EXACT_OK;
}

// Ray of view v, bin b: a point (px, py) on it and its unit direction (dx, dy).
void ray_line(const exact_geometry &g, int v, int b, double &px, double &py, double &dx, double &dy)
{
    const double th = g.angle0 + (double)v * g.angle_range / (double)g.n_views;
    const double c = cos(th), s = sin(th);
    const double u = ((double)b - 0.5 * (double)(g.n_bins - 1)) * g.bin_pitch + g.det_offset;
    if (g.beam == 0) {
        px = -s * u;
        py = c * u;
        dx = -c;
        dy = -s;
    } else {
        const double sx = g.src_to_center * c, sy = g.src_to_center * s;
        const double qx = (g.src_to_center - g.src_to_det) * c - s * u;
        const double qy = (g.src_to_center - g.src_to_det) * s + c * u;
        const double ex = qx - sx, ey = qy - sy, len = sqrt(ex * ex + ey * ey);
        px = sx;
        py = sy;
        dx = ex / len;
        dy = ey / len;
    }
}

struct RayHost {
    int axis, jlo, jhi;
    double alpha, beta, delta;
    double ka, kb, sg;  // walk coefficients (RayW)
};

// Walk coefficients of ray (v, b) on driving axis `axis`: d alpha/d b,
// d beta/d b and the Moebius parameter sg (see RayW).  Fan beam, x driving:
// the ray direction from the source is E = (-R_d c - s u, -R_d s + c u);
// beta = E_y / E_x, so d beta/d u = -R_d / E_x^2 and one bin further on
// beta changes by (d beta/d b) e / (1 - s pitch e / E_x); alpha is affine in
// beta.  y driving swaps the roles.  Parallel beam: alpha is affine in u and
// beta constant.
void walk_coefs(const exact_geometry &g, int v, int b, int axis, double &ka, double &kb, double &sg)
{
    const double th = g.angle0 + (double)v * g.angle_range / (double)g.n_views;
    const double c = cos(th), s = sin(th), p = g.pixel, h = g.bin_pitch;
    if (g.beam == 0) {
        ka = axis == 0 ? h / (c * p) : -h / (s * p);
        kb = 0.0;
        sg = 0.0;
        return;
    }
    const double u = ((double)b - 0.5 * (double)(g.n_bins - 1)) * h + g.det_offset;
    const double Rs = g.src_to_center, Rd = g.src_to_det;
    if (axis == 0) {
        const double ex = -Rd * c - s * u, x0 = -0.5 * (double)(g.nx - 1) * p;
        kb = -Rd * h / (ex * ex);
        sg = -s * h / ex;
        ka = (x0 - Rs * c) / p * kb;
    } else {
        const double ey = -Rd * s + c * u, y0 = -0.5 * (double)(g.ny - 1) * p;
        kb = Rd * h / (ey * ey);
        sg = c * h / ey;
        ka = (y0 - Rs * s) / p * kb;
    }
}

RayHost make_ray(const exact_geometry &g, int v, int b)
{
    double px, py, dx, dy;
    ray_line(g, v, b, px, py, dx, dy);
    RayHost r;
    const double x0 = -0.5 * (double)(g.nx - 1) * g.pixel;
    const double y0 = -0.5 * (double)(g.ny - 1) * g.pixel;
    int nd, nc;
    if (fabs(dx) >= fabs(dy)) {
        r.axis = 0;
        r.beta = dy / dx;
        r.alpha = (py + (x0 - px) * r.beta) / g.pixel + 0.5 * (double)(g.ny - 1);
        r.delta = g.pixel / fabs(dx);
        nd = g.nx;
        nc = g.ny;
    } else {
        r.axis = 1;
        r.beta = dx / dy;
        r.alpha = (px + (y0 - py) * r.beta) / g.pixel + 0.5 * (double)(g.nx - 1);
        r.delta = g.pixel / fabs(dy);
        nd = g.ny;
        nc = g.nx;
    }
    walk_coefs(g, v, b, r.axis, r.ka, r.kb, r.sg);
    // driving indices whose crossing lies in (-1.5, nc + 0.5): a superset of
    // the samples that touch the image, half a pixel of margin for FP32 t
    const double tlo = -1.5, thi = (double)nc + 0.5;
    double jl, jh;
    if (r.beta == 0.0) {
        const bool in = r.alpha > tlo && r.alpha < thi;
        jl = in ? 0.0 : 1.0;
        jh = in ? (double)(nd - 1) : 0.0;
    } else {
        double a = (tlo - r.alpha) / r.beta, c = (thi - r.alpha) / r.beta;
        if (a > c) {
            const double t = a;
            a = c;
            c = t;
        }
        jl = fmax(0.0, ceil(a));
        jh = fmin((double)(nd - 1), floor(c));
    }
    if (!(jl <= jh)) {
        r.jlo = 1;
        r.jhi = 0;
    } else {
        r.jlo = (int)jl;
        r.jhi = (int)jh;
    }
    return r;
}

// Cross index k0 = floor(t(j)) of a ray at driving index j, replayed with the
// same FP32 operations as k_forward_tma (anchor at the chunk start j0, then
// fmaf(bh, j - j0, tau0)).  This file is compiled with FP contraction off, so
// the host arithmetic matches the device expression.
long long k0_at(const RayF &r, int j)
{
    const int j0 = (j / kFC) * kFC;
    const float jf = (float)j0;
    const float p = r.bh * jf;
    const float e = fmaf(r.bh, jf, -p);
    const float P = floorf(p);
    const float tau0 = ((p - P) + r.a) + fmaf(r.bl, jf, e);
    const float tau = fmaf(r.bh, (float)(j - j0), tau0);
    return (long long)r.A + (long long)P + (long long)floorf(tau);
}

// Work unit over rays [b, b + cnt) of one view segment: the chunks their
// driving ranges cover and, per chunk, the first staged cross row.  Within a
// view the crossing t_b(j) is monotone in b at every j (rays of a fan or a
// parallel view do not cross inside the image), so the first and last ray
// that sample a chunk bound all others; a row of margin on each side absorbs
// FP32 rounding.  Returns false if a band does not fit in kFHB rows.
bool make_unit(const RayF *rf, const int *bits, long long ray0, int cnt, int axis, FwdUnit &u,
               std::vector<int> &kst)
{
    int jmin = 1 << 30, jmax = -1;
    for (int q = 0; q < cnt; ++q) {
        const int lo = ray_jlo(bits[ray0 + q]), hi = ray_jhi(bits[ray0 + q]);
        if (lo <= hi) {
            jmin = lo < jmin ? lo : jmin;
            jmax = hi > jmax ? hi : jmax;
        }
    }
    u.ray0 = (int)ray0;
    u.count = cnt;
    u.axis = axis;
    u.pad0 = u.pad1 = 0;
    u.koff = (int)kst.size();
    if (jmax < 0) {
        u.jc0 = 0;
        u.nchunks = 0;
        return true;
    }
    u.jc0 = jmin / kFC;
    u.nchunks = jmax / kFC - u.jc0 + 1;
    std::vector<int> local;
    for (int c = 0; c < u.nchunks; ++c) {
        const int j0 = (u.jc0 + c) * kFC, j1 = j0 + kFC - 1;
        int qf = -1, ql = -1;
        for (int q = 0; q < cnt; ++q) {
            const int lo = ray_jlo(bits[ray0 + q]), hi = ray_jhi(bits[ray0 + q]);
            if (lo <= j1 && hi >= j0 && lo <= hi) {
                if (qf < 0) qf = q;
                ql = q;
            }
        }
        if (qf < 0) {  // no ray samples this chunk: stage nothing useful, any aligned start
            local.push_back(-kPad);
            continue;
        }
        long long kmin = LLONG_MAX, kmax = LLONG_MIN;
        for (int q : {qf, ql})
            for (int j : {j0, j1}) {
                const long long k = k0_at(rf[ray0 + q], j);
                kmin = k < kmin ? k : kmin;
                kmax = k > kmax ? k : kmax;
            }
        // rows kmin - 1 .. kmax + 2 (taps k0, k0 + 1 and a row of margin each side)
        long long start = kmin - 1 + kPad;
        start = (start >= 0 ? start / 4 : -((-start + 3) / 4)) * 4 - kPad;
        if (kmax + 2 - start > kFHB - 1) return false;
        if (start < INT_MIN / 2 || start > INT_MAX / 2) return false;
        local.push_back((int)start);
    }
    kst.insert(kst.end(), local.begin(), local.end());
    return true;
}

// Host threads for building a plan's tables: one for small plans, up to 16
// for plans of 64 K rays or more (the per-view work is independent).
int table_threads(long long n_rays)
{
    if (n_rays < (1LL << 16)) return 1;
    const unsigned hw = std::thread::hardware_concurrency();
    return hw < 2 ? 1 : (hw > 16 ? 16 : (int)hw);
}

// body(v) for v in [0, n) on `threads` host threads (views interleaved).
template <class F>
void parallel_views(int n, int threads, const F &body)
{
    if (threads <= 1 || n <= 1) {
        for (int v = 0; v < n; ++v) body(v);
        return;
    }
    const int T = threads < n ? threads : n;
    std::vector<std::thread> pool;
    pool.reserve((size_t)T);
    for (int t = 0; t < T; ++t)
        pool.emplace_back([&body, n, T, t] {
            for (int v = t; v < n; v += T) body(v);
        });
    for (std::thread &th : pool) th.join();
}

// Splits every view segment into work units of at most kFR rays whose bands
// fit.  Views are split independently (on `threads` host threads) and
// concatenated in view order, so the tables do not depend on the threads.
bool build_units(const exact_geometry &g, const std::vector<RayF> &rf, const std::vector<int> &rbits,
                 const std::vector<ViewRec> &vw, std::vector<FwdUnit> &units, std::vector<int> &kst, int threads)
{
    std::vector<std::vector<FwdUnit>> vu((size_t)g.n_views);
    std::vector<std::vector<int>> vk((size_t)g.n_views);
    std::atomic<bool> ok{true};
    parallel_views(g.n_views, threads, [&](int v) {
        const long long vb = (long long)v * g.n_bins;
        const int segs[2][3] = {{vw[v].xb0, vw[v].xb1, 0}, {vw[v].yb0, vw[v].yb1, 1}};
        for (const auto &sg : segs) {
            int b = sg[0];
            while (b < sg[1]) {
                int cnt = sg[1] - b < kFR ? sg[1] - b : kFR;
                FwdUnit u;
                while (!make_unit(rf.data(), rbits.data(), vb + b, cnt, sg[2], u, vk[v])) {
                    if (cnt == 1) {
                        ok = false;
                        return;
                    }
                    cnt = cnt * 3 / 4 > 1 ? cnt * 3 / 4 : 1;
                }
                vu[v].push_back(u);
                b += cnt;
            }
        }
    });
    if (!ok) return false;
    for (int v = 0; v < g.n_views; ++v) {
        const int base = (int)kst.size();  // the view's band starts follow the earlier views'
        for (FwdUnit u : vu[v]) {
            u.koff += base;
            units.push_back(u);
        }
        kst.insert(kst.end(), vk[v].begin(), vk[v].end());
    }
    return true;
}

ViewRec make_view(const exact_geometry &g, int v, int xb0, int xb1, int yb0, int yb1)
{
    const double th = g.angle0 + (double)v * g.angle_range / (double)g.n_views;
    const double c = cos(th), s = sin(th), p = g.pixel;
    const double cx = 0.5 * (double)(g.nx - 1), cy = 0.5 * (double)(g.ny - 1);
    // P.eu = -s p kx + c p ky + (cx s - cy c) p ;  P.es = c p kx + s p ky - (cx c + cy s) p
    ViewRec r;
    const double cc = 0.5 * (double)(g.n_bins - 1) - g.det_offset / g.bin_pitch;
    if (g.beam == 0) {
        const double k = 1.0 / g.bin_pitch;
        r.n0 = (float)(k * (cx * s - cy * c) * p);
        r.n1 = (float)(-k * s * p);
        r.n2 = (float)(k * c * p);
        r.d0 = 1.0f;
        r.d1 = 0.0f;
        r.d2 = 0.0f;
    } else {
        const double k = g.src_to_det / g.bin_pitch;
        r.n0 = (float)(k * (cx * s - cy * c) * p);
        r.n1 = (float)(-k * s * p);
        r.n2 = (float)(k * c * p);
        r.d0 = (float)(g.src_to_center + (cx * c + cy * s) * p);
        r.d1 = (float)(-c * p);
        r.d2 = (float)(-s * p);
    }
    r.c = (float)cc;
    r.pad = 0.0f;
    r.xb0 = xb0;
    r.xb1 = xb1;
    r.yb0 = yb0;
    r.yb1 = yb1;
    return r;
}

// The per-tile arrival counts of the adjoint's view split are zero between
// launches (the last CTA of a tile resets its count); a launch cut short (a
// timed-out batch) could leave some set, so every call that launches the
// adjoint clears them first.
cudaError_t reset_split_counts(const Plan &P, cudaStream_t s)
{
    return cudaMemsetAsync(P.split_count, 0, sizeof(int) * (size_t)adjoint_blocks(P.g.nx, P.g.ny), s);
}

exact_status check_plan(exact_plan_t p, bool need_ws)
{
    if (!p) return EXACT_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return EXACT_ERR_CUDA;
    if (dev != reinterpret_cast<Plan *>(p)->device) return EXACT_ERR_INVALID_ARG;
    if (need_ws && !reinterpret_cast<Plan *>(p)->ws) return EXACT_ERR_NO_WORKSPACE;
    return EXACT_OK;
}

struct Carve {
    size_t off = 0;
    template <typename T>
    T *take(char *base, size_t count)
    {
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off = align_up(off + count * sizeof(T));
        return p;
    }
};

// Lays the workspace out (base == nullptr: only measures).
size_t carve(Plan &P, char *base)
{
    Carve c;
    const long long nx = P.g.nx, ny = P.g.ny;
    for (int q = 0; q < 2; ++q) {
        P.xr[q] = c.take<float>(base, (size_t)(ny * P.ldr()));
        P.xc[q] = c.take<float>(base, (size_t)(nx * P.ldc()));
    }
    P.Y = c.take<float>(base, (size_t)P.n);
    P.r = c.take<float>(base, (size_t)P.n);
    const int nb_adj = adjoint_blocks(P.g.nx, P.g.ny);
    const int nb_fwd = forward_d_blocks(P.n);
    const int nb_adj_d = adjoint_d_blocks(P.g.nx, P.g.ny);
    const int nb_d = nb_adj_d > kSumsqParts ? nb_adj_d : kSumsqParts;
    P.tv_grid = tv_grid(P.d);
    const int nb_eg = nb_adj > P.tv_grid ? nb_adj : P.tv_grid;  // partial-norm producers of a full step
    P.partials = c.take<double>(base, (size_t)(kPartStride * nb_eg + (nb_fwd > kSumsqParts ? nb_fwd : kSumsqParts) + nb_d));
    P.avg = c.take<double>(base, (size_t)P.d);
    P.xrd = c.take<double>(base, (size_t)(ny * P.ldr()));
    P.xcd = c.take<double>(base, (size_t)(nx * P.ldc()));
    P.zd = c.take<double>(base, (size_t)P.n);
    P.w32 = c.take<float>(base, (size_t)P.d);
    P.state = c.take<DevState>(base, 1);
    P.split_part = c.take<float>(base, (size_t)nb_adj * P.max_split * kTH * kTW);
    P.split_count = c.take<int>(base, (size_t)nb_adj);
    P.tv_step = c.take<float>(base, (size_t)P.d);
    P.tv_lam = c.take<double>(base, 2);
    if (P.tv_grid > 0) P.tv_ws = c.take<char>(base, tv_workspace_bytes(nx, ny, P.tv_grid));
    P.stage_y = c.take<float>(base, (size_t)P.W * (size_t)P.n);  // host-buffer solve: counts (FP32 or BF16)
    P.stage_x = c.take<float>(base, (size_t)P.d);                // and the image
    return c.off;
}

// Host-function payload that copies a solve's device state (already copied
// to pinned memory) into the caller's info struct.  A payload enqueued outside
// stream capture runs once and frees itself; one captured in a CUDA graph runs
// on every replay, so it stays alive and is freed with its owner.
struct InfoCopy {
    const DevState *src;
    exact_solve_info *dst;
    bool one_shot;
};

void info_copy_cb(void *data)
{
    InfoCopy *c = static_cast<InfoCopy *>(data);
    c->dst->iters_done = c->src->iters_done;
    c->dst->rel_res = c->src->rel_res;
    c->dst->status = (exact_status)c->src->status;
    c->dst->avg_change = c->src->avg_change;
    if (c->one_shot) delete c;
}

// Enqueue the copy of `st` (device) to `info` (host) on stream s.
exact_status enqueue_info(DevState *st, DevState *host_state, exact_solve_info *info, std::vector<void *> &keep,
                          cudaStream_t s)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    EXACT_TRY(cudaStreamIsCapturing(s, &cap));
    EXACT_TRY(cudaMemcpyAsync(host_state, st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    InfoCopy *c = new (std::nothrow) InfoCopy{host_state, info, cap == cudaStreamCaptureStatusNone};
    if (!c) return EXACT_ERR_OOM;
    cudaError_t e = cudaLaunchHostFunc(s, info_copy_cb, c);
    if (e != cudaSuccess) {
        delete c;
        return cuda_status(e);
    }
    if (!c->one_shot) keep.push_back(c);
    return EXACT_OK;
}

ImgF img_of(const Plan &P, int q)
{
    ImgF im;
    im.xr = P.xr[q];
    im.xc = P.xc[q];
    im.nx = P.g.nx;
    im.ny = P.g.ny;
    im.ldr = P.ldr();
    im.ldc = P.ldc();
    return im;
}

// Event pair around one sampled launch (profiling aid); returns the pair
// index or -1 when this launch is not sampled.
int prof_begin(Plan &P, int kind, int iter, cudaStream_t s)
{
    if (P.prof_every <= 0 || iter % P.prof_every != 0 || P.prof_used >= P.prof_cap) return -1;
    const int u = P.prof_used++;
    P.prof_kind[u] = kind;
    if (cudaEventRecord(P.prof_ev[2 * u], s) != cudaSuccess) return -1;
    return u;
}

void prof_end(Plan &P, int u, cudaStream_t s)
{
    if (u >= 0) cudaEventRecord(P.prof_ev[2 * u + 1], s);
}

constexpr int kSplitCandidates[] = {1, 2, 3, 4, 6, 8, 12, 16};

int device_sms(int device)
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) sms = 1;
    return sms;
}

// Largest view split a plan supports (its workspace holds that many partial
// tiles per tile): up to kMaxSplit while tiles x split stays within about 64
// CTAs per SM; more only adds partial tiles to combine.
int max_split(const Plan &P)
{
    const long long tiles = adjoint_blocks(P.g.nx, P.g.ny), cap = 64LL * device_sms(P.device);
    int best = 1;
    for (int s : kSplitCandidates)
        if (s <= kMaxSplit && tiles * s <= cap) best = s;
    return best;
}

// View split of a new plan's adjoint, before any autotuning: the largest
// candidate that keeps tiles x split within about 14 CTAs per SM (near three
// waves of the 5 adjoint CTAs resident per SM; at 512^2 split 8, the largest
// such, measured faster than 4 and 16).  Small images get more CTAs than they
// have tiles.
int default_split(const Plan &P)
{
    const long long tiles = adjoint_blocks(P.g.nx, P.g.ny), want = 14LL * device_sms(P.device);
    int best = 1;
    for (int s : kSplitCandidates)
        if (s <= P.max_split && tiles * s <= want) best = s;
    return best;
}

void free_solve_graphs(Plan &P)
{
    for (SolveGraph &g : P.graphs) {
        if (g.last) {
            cudaEventSynchronize(g.last);
            cudaEventDestroy(g.last);
        }
        if (g.exec) cudaGraphExecDestroy(g.exec);
    }
    P.graphs.clear();
    if (P.cap_stream) cudaStreamDestroy(P.cap_stream);
    P.cap_stream = nullptr;
}

// Runs a solve's iterations as one CUDA graph launch on s: the graph is a
// single WHILE node whose body holds one iteration's kernels, captured from
// body(cond, stream) on the plan's capture stream; the body's reduction
// kernel sets the loop condition, so the loop stops on the device after the
// stopping test passes or the last iteration.  The instantiated graph is kept
// under `key` (the kernel arguments that the device state does not supply)
// and relaunched when the key recurs; with kSolveGraphs kept, a new one
// replaces the least recently used after that one's last launch has finished.
template <typename Body>
exact_status launch_solve_graph(Plan &P, const void *key, size_t key_bytes, Body &&body, cudaStream_t s)
{
    const unsigned char *kb = static_cast<const unsigned char *>(key);
    SolveGraph *hit = nullptr;
    for (SolveGraph &g : P.graphs)
        if (g.key.size() == key_bytes && memcmp(g.key.data(), kb, key_bytes) == 0) {
            hit = &g;
            break;
        }
    if (!hit) {
        if (!P.cap_stream) EXACT_TRY(cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        EXACT_TRY(cudaGraphCreate(&graph, 0));
        exact_status st = EXACT_OK;
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t last = nullptr;
        do {
            cudaGraphConditionalHandle cond = 0;
            cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault);
            if (e != cudaSuccess) {
                st = cuda_status(e);
                break;
            }
            // zeroed storage: the struct's union has no default constructor
            alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)] = {};
            cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(np_raw);
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = cond;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node = nullptr;
            if ((e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np)) != cudaSuccess) {
                st = cuda_status(e);
                break;
            }
            cudaGraph_t loop = np.conditional.phGraph_out[0];
            if ((e = cudaStreamBeginCaptureToGraph(P.cap_stream, loop, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
                st = cuda_status(e);
                break;
            }
            st = body(cond, P.cap_stream);
            cudaGraph_t captured = nullptr;
            e = cudaStreamEndCapture(P.cap_stream, &captured);
            if (st == EXACT_OK && e != cudaSuccess) st = cuda_status(e);
            if (st != EXACT_OK) break;
            if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
                exec = nullptr;
                st = cuda_status(e);
                break;
            }
            if ((e = cudaEventCreateWithFlags(&last, cudaEventDisableTiming)) != cudaSuccess) {
                st = cuda_status(e);
                break;
            }
        } while (0);
        cudaGraphDestroy(graph);
        if (st != EXACT_OK) {
            if (exec) cudaGraphExecDestroy(exec);
            return st;
        }
        if ((int)P.graphs.size() >= kSolveGraphs) {
            auto lru = std::min_element(P.graphs.begin(), P.graphs.end(),
                                        [](const SolveGraph &u, const SolveGraph &v) { return u.stamp < v.stamp; });
            cudaEventSynchronize(lru->last);
            cudaEventDestroy(lru->last);
            cudaGraphExecDestroy(lru->exec);
            P.graphs.erase(lru);
        }
        SolveGraph g;
        g.exec = exec;
        g.last = last;
        g.key.assign(kb, kb + key_bytes);
        P.graphs.push_back(std::move(g));
        hit = &P.graphs.back();
    }
    hit->stamp = ++P.graph_clock;
    EXACT_TRY(cudaGraphLaunch(hit->exec, s));
    EXACT_TRY(cudaEventRecord(hit->last, s));
    return EXACT_OK;
}

void prof_free(Plan &P)
{
    for (int i = 0; i < 2 * P.prof_cap; ++i) cudaEventDestroy(P.prof_ev[i]);
    delete[] P.prof_ev;
    delete[] P.prof_kind;
    P.prof_ev = nullptr;
    P.prof_kind = nullptr;
    P.prof_cap = P.prof_used = 0;
}

// Nonzero entries of A, counted tap by tap in FP64.
long long count_nnz(const exact_geometry &g)
{
    long long nnz = 0;
    for (int v = 0; v < g.n_views; ++v)
        for (int b = 0; b < g.n_bins; ++b) {
            const RayHost h = make_ray(g, v, b);
            const int nc = h.axis ? g.nx : g.ny;
            for (int j = h.jlo; j <= h.jhi; ++j) {
                const double t = h.alpha + h.beta * (double)j;
                const double k0 = floor(t), f = t - k0;
                if (1.0 - f > 0.0 && k0 >= 0.0 && k0 < (double)nc) ++nnz;
                if (f > 0.0 && k0 + 1.0 >= 0.0 && k0 + 1.0 < (double)nc) ++nnz;
            }
        }
    return nnz;
}

}  // namespace

namespace exact {

// Encodes the 2D tensor map (x = padded cross index, y = driving line) of one
// padded image copy; box kFHB x kFC, zero fill outside.  The driver entry
// point is looked up once per process (thread-safe static initialisation).
bool encode_map(CUtensorMap *map, float *base, long long ld, long long lines)
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        cudaDriverEntryPointQueryResult q;
        void *ptr = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)lines};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kFHB, (cuuint32_t)kFC};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---- fault injection (exact_debug_inject) ----
namespace {
std::atomic<long long> g_wait_polls{0};
std::atomic<int> g_block_batch_job{-1};
std::atomic<int> g_block_tv{0};
}  // namespace

long long debug_wait_polls() { return g_wait_polls.load(); }
int debug_take_batch_block() { return g_block_batch_job.exchange(-1); }
bool debug_take_tv_block() { return g_block_tv.exchange(0) != 0; }

LinkCoef make_coef(const Plan &P, double I0)
{
    LinkCoef c;
    memset(&c, 0, sizeof(c));
    for (int k = 0; k < P.K; ++k) {
        c.mu2[k] = P.mu_log2e[k];
        c.c[k] = (float)(I0 * (double)P.C[k]);
        for (int m = 0; m < P.bg_M; ++m) c.mub[m][k] = P.bg_mu2[m][k];
    }
    return c;
}

}  // namespace exact

extern "C" {

const char *exact_status_string(exact_status s)
{
    switch (s) {
    case EXACT_OK: return "ok";
    case EXACT_ERR_INVALID_ARG: return "invalid argument";
    case EXACT_ERR_CUDA: return "CUDA error";
    case EXACT_ERR_OOM: return "out of memory";
    case EXACT_ERR_TIMEOUT: return "bounded device wait timed out";
    case EXACT_ERR_NONFINITE: return "non-finite residual";
    case EXACT_ERR_UNSUPPORTED: return "unsupported";
    case EXACT_ERR_NO_WORKSPACE: return "no workspace bound";
    }
    return "unknown status";
}

exact_status exact_debug_inject(int kind, long long value)
{
    switch (kind) {
    case EXACT_INJECT_WAIT_POLLS:
        if (value < 0) return EXACT_ERR_INVALID_ARG;
        g_wait_polls.store(value);
        return EXACT_OK;
    case EXACT_INJECT_BLOCK_BATCH_JOB:
        if (value < -1 || value >= kMaxBatch) return EXACT_ERR_INVALID_ARG;
        g_block_batch_job.store((int)value);
        return EXACT_OK;
    case EXACT_INJECT_BLOCK_TV_BARRIER:
        g_block_tv.store(value != 0 ? 1 : 0);
        return EXACT_OK;
    }
    return EXACT_ERR_INVALID_ARG;
}

exact_solve_opts exact_solve_opts_default(void)
{
    exact_solve_opts o;
    o.lo = 0.0;
    o.hi = INFINITY;
    o.tol = 0.0;
    o.check_every = 1;
    o.average_tail = 0;
    o.stop_rule = EXACT_STOP_RESIDUAL;
    o.history_cap = 0;
    o.history = nullptr;
    o.tv_bound = 0.0;
    o.tv = exact_tv_opts_default();
    o.prox_lambda = 0.0;
    o.t0 = 0;
    o.total_iters = 0;
    o.resume = nullptr;
    o.x_last = nullptr;
    o.launch = 0;
    o.pad = 0;
    return o;
}

size_t exact_solve_resume_bytes(exact_plan_t plan)
{
    if (!plan) return 0;
    return sizeof(double) * (size_t)(reinterpret_cast<Plan *>(plan)->d + 2);
}

exact_status exact_plan_create(const exact_geometry *geometry, const exact_spectrum *spectrum,
                               const exact_windows *windows, exact_plan_t *out)
{
    if (!out) return EXACT_ERR_INVALID_ARG;
    *out = nullptr;
    exact_status st = check_geometry(geometry);
    if (st != EXACT_OK) return st;
    if (!spectrum || !windows || !spectrum->mu || !windows->S) return EXACT_ERR_INVALID_ARG;
    const int K = spectrum->n_energy, W = windows->n_windows;
    if (K < 1 || K > kMaxK || W < 1 || W > 64) return EXACT_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k)
        if (!isfin(spectrum->mu[k]) || !(spectrum->mu[k] > 0.0)) return EXACT_ERR_INVALID_ARG;
    for (int w = 0; w < W; ++w) {
        double sw = 0.0;
        for (int k = 0; k < K; ++k) {
            const double v = windows->S[w * K + k];
            if (!isfin(v) || v < 0.0) return EXACT_ERR_INVALID_ARG;
            sw += v;
        }
        if (!(sw > 0.0)) return EXACT_ERR_INVALID_ARG;
    }

    Plan *P = new (std::nothrow) Plan();
    if (!P) return EXACT_ERR_OOM;
    if (cudaGetDevice(&P->device) != cudaSuccess) {
        delete P;
        return EXACT_ERR_CUDA;
    }
    P->g = *geometry;
    P->W = W;
    P->K = K;
    P->n = (long long)geometry->n_views * geometry->n_bins;
    P->d = (long long)geometry->nx * geometry->ny;
    P->Csum_mu = 0.0;
    for (int k = 0; k < K; ++k) {
        double ck = 0.0;
        for (int w = 0; w < W; ++w) ck += windows->S[w * K + k];
        P->C[k] = (float)ck;
        P->mu_log2e[k] = (float)(spectrum->mu[k] * 1.4426950408889634);
        P->Csum_mu += ck * spectrum->mu[k];
    }

    const exact_geometry &g = *geometry;
    std::vector<RayF> rf((size_t)P->n);
    std::vector<RayW> rw((size_t)P->n);
    std::vector<int> rbits((size_t)P->n);
    std::vector<float> rdelta((size_t)P->n);
    std::vector<RayD> rd((size_t)P->n);
    std::vector<ViewRec> vw((size_t)g.n_views);
    const int threads = table_threads(P->n);
    std::atomic<bool> axis_ok{true};
    parallel_views(g.n_views, threads, [&](int v) {
        int switches = 0;
        int prev_axis = -1;
        int first_axis = -1, sw = g.n_bins;
        for (int b = 0; b < g.n_bins; ++b) {
            const RayHost h = make_ray(g, v, b);
            const int bits = (h.jlo & 0x7fff) | ((h.jhi & 0x7fff) << 15) | (h.axis << 30);
            const size_t i = (size_t)v * g.n_bins + b;
            const double A = floor(h.alpha);
            const float bh = (float)h.beta;
            rf[i].A = (float)A;
            rf[i].a = (float)(h.alpha - A);
            rf[i].bh = bh;
            rf[i].bl = (float)(h.beta - (double)bh);
            rw[i].ka = (float)h.ka;
            rw[i].kb = (float)h.kb;
            rw[i].sg = (float)h.sg;
            rw[i].pad = 0.0f;
            rbits[i] = bits;
            rdelta[i] = (float)h.delta;
            rd[i].alpha = h.alpha;
            rd[i].beta = h.beta;
            rd[i].delta = h.delta;
            rd[i].bits = bits;
            rd[i].pad = 0;
            if (b == 0) first_axis = h.axis;
            if (prev_axis >= 0 && h.axis != prev_axis) {
                ++switches;
                sw = b;
            }
            prev_axis = h.axis;
        }
        if (switches > 1) {  // driving axis must switch at most once per view (fan angle below 90 degrees)
            axis_ok = false;
            return;
        }
        // segment [0, sw) has first_axis, [sw, n_bins) the other one
        int xb0 = 0, xb1 = 0, yb0 = 0, yb1 = 0;
        if (first_axis == 0) {
            xb0 = 0; xb1 = sw; yb0 = sw; yb1 = g.n_bins;
        } else {
            yb0 = 0; yb1 = sw; xb0 = sw; xb1 = g.n_bins;
        }
        vw[v] = make_view(g, v, xb0, xb1, yb0, yb1);
    });
    if (!axis_ok) {
        delete P;
        return EXACT_ERR_UNSUPPORTED;
    }
    std::vector<FwdUnit> units;
    std::vector<int> kst;
    if (!build_units(g, rf, rbits, vw, units, kst, threads)) {
        delete P;
        return EXACT_ERR_UNSUPPORTED;
    }
    if (kst.empty()) kst.push_back(0);
    P->n_units = (int)units.size();
    // uploads on a private non-blocking stream: a plan built on one host
    // thread does not wait for (or hold up) work that other threads run on
    // the legacy default stream
    cudaStream_t up = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking);
    auto put = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, up);
    };
    if (e == cudaSuccess) e = cudaMalloc(&P->rays_f, sizeof(RayF) * rf.size());
    if (e == cudaSuccess) e = cudaMalloc(&P->rays_w, sizeof(RayW) * rw.size());
    if (e == cudaSuccess) e = cudaMalloc(&P->units, sizeof(FwdUnit) * units.size());
    if (e == cudaSuccess) e = cudaMalloc(&P->kstart, sizeof(int) * kst.size());
    if (e == cudaSuccess) e = cudaMalloc(&P->ray_bits, sizeof(int) * rbits.size());
    if (e == cudaSuccess) e = cudaMalloc(&P->ray_delta, sizeof(float) * rdelta.size());
    if (e == cudaSuccess) e = cudaMalloc(&P->rays_d, sizeof(RayD) * rd.size());
    if (e == cudaSuccess) e = cudaMalloc(&P->views, sizeof(ViewRec) * vw.size());
    // the adjoint's per-axis view lists: views with x-driven rays, then views
    // with y-driven rays (a fan crossing a diagonal is in both)
    std::vector<int> vit;
    for (int v = 0; v < g.n_views; ++v)
        if (vw[v].xb1 > vw[v].xb0) vit.push_back(v);
    P->nxv = (int)vit.size();
    for (int v = 0; v < g.n_views; ++v)
        if (vw[v].yb1 > vw[v].yb0) vit.push_back(v);
    P->nyv = (int)vit.size() - P->nxv;
    if (vit.empty()) vit.push_back(0);
    if (e == cudaSuccess) e = cudaMalloc(&P->vitems, sizeof(int) * vit.size());
    put(P->vitems, vit.data(), sizeof(int) * vit.size());
    put(P->rays_w, rw.data(), sizeof(RayW) * rw.size());
    put(P->units, units.data(), sizeof(FwdUnit) * units.size());
    put(P->kstart, kst.data(), sizeof(int) * kst.size());
    put(P->rays_f, rf.data(), sizeof(RayF) * rf.size());
    put(P->ray_bits, rbits.data(), sizeof(int) * rbits.size());
    put(P->ray_delta, rdelta.data(), sizeof(float) * rdelta.size());
    put(P->rays_d, rd.data(), sizeof(RayD) * rd.size());
    put(P->views, vw.data(), sizeof(ViewRec) * vw.size());
    if (up) {
        const cudaError_t es = cudaStreamSynchronize(up);  // the host vectors die at return
        if (e == cudaSuccess) e = es;
        cudaStreamDestroy(up);
    }
    if (e == cudaSuccess) e = cudaMallocHost(&P->host_state, sizeof(DevState));
    if (e != cudaSuccess) {
        exact_plan_destroy(reinterpret_cast<exact_plan_t>(P));
        return cuda_status(e);
    }
    P->max_split = max_split(*P);
    P->adj_split = default_split(*P);
    memset(P->host_state, 0, sizeof(DevState));
    *out = reinterpret_cast<exact_plan_t>(P);
    return EXACT_OK;
}

exact_status exact_plan_destroy(exact_plan_t plan)
{
    if (!plan) return EXACT_OK;
    Plan *P = reinterpret_cast<Plan *>(plan);
    int prev = -1;
    cudaGetDevice(&prev);
    if (P->device >= 0 && prev != P->device) cudaSetDevice(P->device);
    if (P->rays_f) cudaFree(P->rays_f);
    if (P->rays_w) cudaFree(P->rays_w);
    if (P->units) cudaFree(P->units);
    if (P->kstart) cudaFree(P->kstart);
    if (P->ray_bits) cudaFree(P->ray_bits);
    if (P->ray_delta) cudaFree(P->ray_delta);
    if (P->rays_d) cudaFree(P->rays_d);
    if (P->views) cudaFree(P->views);
    if (P->vitems) cudaFree(P->vitems);
    free_solve_graphs(*P);
    if (P->host_state) cudaFreeHost(P->host_state);
    if (P->prof_ev) prof_free(*P);
    for (void *c : P->captured_infos) delete static_cast<InfoCopy *>(c);
    if (prev >= 0 && prev != P->device) cudaSetDevice(prev);
    delete P;
    return EXACT_OK;
}

exact_status exact_plan_dims(exact_plan_t plan, long long *n_rays, long long *n_pixels)
{
    if (!plan) return EXACT_ERR_INVALID_ARG;
    const Plan *P = reinterpret_cast<const Plan *>(plan);
    if (n_rays) *n_rays = P->n;
    if (n_pixels) *n_pixels = P->d;
    return EXACT_OK;
}

size_t exact_plan_workspace_bytes(exact_plan_t plan)
{
    if (!plan) return 0;
    Plan tmp = *reinterpret_cast<Plan *>(plan);
    return carve(tmp, nullptr);
}

exact_status exact_plan_bind_workspace(exact_plan_t plan, void *dev_ptr, size_t bytes)
{
    if (!plan) return EXACT_ERR_INVALID_ARG;
    Plan *P = reinterpret_cast<Plan *>(plan);
    free_solve_graphs(*P);  // they hold pointers into the old workspace
    if (!dev_ptr) {
        P->ws = nullptr;
        P->ws_bytes = 0;
        return EXACT_OK;
    }
    if (reinterpret_cast<uintptr_t>(dev_ptr) % kAlign != 0) return EXACT_ERR_INVALID_ARG;
    if (bytes < exact_plan_workspace_bytes(plan)) return EXACT_ERR_INVALID_ARG;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, dev_ptr) != cudaSuccess || attr.type != cudaMemoryTypeDevice ||
        attr.device != P->device) {
        cudaGetLastError();
        return EXACT_ERR_INVALID_ARG;
    }
    carve(*P, static_cast<char *>(dev_ptr));
    for (int q = 0; q < 2; ++q) {
        if (!encode_map(&P->maps_r[q], P->xr[q], P->ldr(), P->g.ny) ||
            !encode_map(&P->maps_c[q], P->xc[q], P->ldc(), P->g.nx)) {
            P->ws = nullptr;
            P->ws_bytes = 0;
            return EXACT_ERR_CUDA;
        }
    }
    if (cudaMemset(P->split_count, 0, sizeof(int) * (size_t)adjoint_blocks(P->g.nx, P->g.ny)) != cudaSuccess) {
        P->ws = nullptr;
        P->ws_bytes = 0;
        return EXACT_ERR_CUDA;
    }
    P->ws = dev_ptr;
    P->ws_bytes = bytes;
    return EXACT_OK;
}

// ---------------------------------------------------------------- tuning

namespace {

struct TuneKey {
    int beam, nx, ny, views, bins;
    bool operator<(const TuneKey &o) const
    {
        if (beam != o.beam) return beam < o.beam;
        if (nx != o.nx) return nx < o.nx;
        if (ny != o.ny) return ny < o.ny;
        if (views != o.views) return views < o.views;
        return bins < o.bins;
    }
};

std::mutex g_tune_lock;
std::map<TuneKey, int> g_tune_cache;  // adj_split chosen per geometry shape, this process

}  // namespace

exact_status exact_plan_get_tuning(exact_plan_t plan, exact_tuning *out)
{
    if (!plan || !out) return EXACT_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->adj_split = reinterpret_cast<Plan *>(plan)->adj_split;
    return EXACT_OK;
}

exact_status exact_plan_set_tuning(exact_plan_t plan, const exact_tuning *t)
{
    if (!plan || !t || t->adj_split < 1 || t->adj_split > kMaxSplit) return EXACT_ERR_INVALID_ARG;
    if (t->adj_split > reinterpret_cast<Plan *>(plan)->max_split) return EXACT_ERR_UNSUPPORTED;
    reinterpret_cast<Plan *>(plan)->adj_split = t->adj_split;
    return EXACT_OK;
}

exact_status exact_plan_autotune(exact_plan_t plan, int force, exact_tuning *out, exact_stream_t stream)
{
    exact_status st = check_plan(plan, true);
    if (st != EXACT_OK) return st;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    const TuneKey key{P.g.beam, P.g.nx, P.g.ny, P.g.n_views, P.g.n_bins};
    if (!force) {
        std::lock_guard<std::mutex> guard(g_tune_lock);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            P.adj_split = it->second;
            return out ? exact_plan_get_tuning(plan, out) : EXACT_OK;
        }
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    EXACT_TRY(cudaMemsetAsync(P.r, 0, sizeof(float) * (size_t)P.n, s));
    EXACT_TRY(reset_split_counts(P, s));
    AdjArgs a;
    memset(&a, 0, sizeof(a));
    a.rays = P.rays_f;
    a.walk = P.rays_w;
    adj_views(a, P);
    a.n_views = P.g.n_views;
    a.n_bins = P.g.n_bins;
    a.nx = P.g.nx;
    a.ny = P.g.ny;
    a.r = P.r;
    a.scale = 1.0f;
    a.out = P.w32;
    a.split_part = P.split_part;
    a.split_count = P.split_count;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return EXACT_ERR_CUDA;
    }
    const bool fan = P.g.beam == 1;
    // candidates are timed round-robin (one launch each per round, after a
    // warm-up round) so that clock drift spreads over all of them
    constexpr int kCands = (int)(sizeof(kSplitCandidates) / sizeof(kSplitCandidates[0]));
    constexpr int kRounds = 9;
    float ms[kCands][kRounds];
    cudaError_t e = cudaSuccess;
    for (int r = -1; r < kRounds && e == cudaSuccess; ++r)
        for (int c = 0; c < kCands && e == cudaSuccess; ++c) {
            if (kSplitCandidates[c] > P.max_split) {  // beyond the plan's partial-tile space
                if (r >= 0) ms[c][r] = INFINITY;
                continue;
            }
            a.nsplit = kSplitCandidates[c];
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = launch_adjoint(a, ADJ_PLAIN, fan, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (r >= 0) ms[c][r] = t;
        }
    int best = 1;
    float best_ms = INFINITY;
    for (int c = 0; c < kCands && e == cudaSuccess; ++c) {
        std::sort(ms[c], ms[c] + kRounds);
        // the fastest median; a larger split must beat a smaller one by 1%
        if (ms[c][kRounds / 2] < 0.99f * best_ms) {
            best_ms = ms[c][kRounds / 2];
            best = kSplitCandidates[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_status(e);
    P.adj_split = best;
    {
        std::lock_guard<std::mutex> guard(g_tune_lock);
        g_tune_cache[key] = best;
    }
    return out ? exact_plan_get_tuning(plan, out) : EXACT_OK;
}

exact_status exact_forward(exact_plan_t plan, const float *x, float *z, exact_stream_t stream)
{
    exact_status st = check_plan(plan, true);
    if (st != EXACT_OK) return st;
    if (!x || !z) return EXACT_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    EXACT_TRY(launch_pack(x, P.xr[0], P.xc[0], P.g.nx, P.g.ny, P.ldr(), P.ldc(), 0.f, 0.f, false, s));
    FwdArgs a;
    memset(&a, 0, sizeof(a));
    a.img = img_of(P, 0);
    a.rays = P.rays_f;
    a.bits = P.ray_bits;
    a.delta = P.ray_delta;
    a.units = P.units;
    a.kstart = P.kstart;
    a.n_units = P.n_units;
    a.n = P.n;
    a.z = z;
    EXACT_TRY(launch_forward(a, false, nullptr, P.maps_r[0], P.maps_c[0], s));
    return EXACT_OK;
}

exact_status exact_adjoint(exact_plan_t plan, const float *r, float *g, exact_stream_t stream)
{
    exact_status st = check_plan(plan, false);
    if (st != EXACT_OK) return st;
    if (!r || !g) return EXACT_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    AdjArgs a;
    memset(&a, 0, sizeof(a));
    a.rays = P.rays_f;
    a.walk = P.rays_w;
    a.nsplit = P.adj_split;
    a.split_part = P.split_part;
    a.split_count = P.split_count;
    adj_views(a, P);
    a.n_views = P.g.n_views;
    a.n_bins = P.g.n_bins;
    a.nx = P.g.nx;
    a.ny = P.g.ny;
    a.r = r;
    a.delta = P.ray_delta;
    a.scale = 1.0f;
    a.out = g;
    EXACT_TRY(reset_split_counts(P, reinterpret_cast<cudaStream_t>(stream)));
    EXACT_TRY(launch_adjoint(a, ADJ_PLAIN, P.g.beam == 1, reinterpret_cast<cudaStream_t>(stream)));
    return EXACT_OK;
}

exact_status exact_operator(exact_plan_t plan, const float *x, const void *y, exact_dtype y_dtype, double I0,
                            float *F, exact_stream_t stream)
{
    exact_status st = check_plan(plan, true);
    if (st != EXACT_OK) return st;
    if (!x || !y || !F) return EXACT_ERR_INVALID_ARG;
    if (y_dtype != EXACT_F32 && y_dtype != EXACT_BF16) return EXACT_ERR_INVALID_ARG;
    if (!isfin(I0) || !(I0 > 0.0)) return EXACT_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const LinkCoef coef = make_coef(P, I0);
    EXACT_TRY(launch_collapse(y, y_dtype, P.W, P.n, P.Y, s));
    EXACT_TRY(launch_pack(x, P.xr[0], P.xc[0], P.g.nx, P.g.ny, P.ldr(), P.ldc(), 0.f, 0.f, false, s));
    FwdArgs f;
    memset(&f, 0, sizeof(f));
    f.img = img_of(P, 0);
    f.rays = P.rays_f;
    f.bits = P.ray_bits;
    f.delta = P.ray_delta;
    f.units = P.units;
    f.kstart = P.kstart;
    f.n_units = P.n_units;
    f.n = P.n;
    f.Y = P.Y;
    f.r = P.r;
    f.K = P.K;
    f.M = P.bg_M;
    f.bg = P.bg_p;
    EXACT_TRY(launch_forward(f, true, &coef, P.maps_r[0], P.maps_c[0], s));
    AdjArgs a;
    memset(&a, 0, sizeof(a));
    a.rays = P.rays_f;
    a.walk = P.rays_w;
    a.nsplit = P.adj_split;
    a.split_part = P.split_part;
    a.split_count = P.split_count;
    adj_views(a, P);
    a.n_views = P.g.n_views;
    a.n_bins = P.g.n_bins;
    a.nx = P.g.nx;
    a.ny = P.g.ny;
    a.r = P.r;
    a.scale = (float)(1.0 / ((double)P.W * (double)P.n));
    a.out = F;
    EXACT_TRY(reset_split_counts(P, s));
    EXACT_TRY(launch_adjoint(a, ADJ_PLAIN, P.g.beam == 1, s));
    return EXACT_OK;
}

exact_status exact_solve(exact_plan_t plan, const void *y, exact_dtype y_dtype, double I0, double eta, int iters,
                         const exact_solve_opts *opts, float *x, exact_solve_info *info, exact_stream_t stream)
{
    exact_status st = check_plan(plan, true);
    if (st != EXACT_OK) return st;
    if (!y || !x) return EXACT_ERR_INVALID_ARG;
    if (y_dtype != EXACT_F32 && y_dtype != EXACT_BF16) return EXACT_ERR_INVALID_ARG;
    if (!isfin(I0) || !(I0 > 0.0) || !isfin(eta) || !(eta > 0.0) || iters < 0) return EXACT_ERR_INVALID_ARG;
    const exact_solve_opts o = opts ? *opts : exact_solve_opts_default();
    if (isnan(o.lo) || isnan(o.hi) || o.lo > o.hi || o.lo == INFINITY || o.hi == -INFINITY)
        return EXACT_ERR_INVALID_ARG;
    if (!isfin(o.tol) || o.tol < 0.0 || o.check_every < 0) return EXACT_ERR_INVALID_ARG;
    if (o.stop_rule != EXACT_STOP_RESIDUAL && o.stop_rule != EXACT_STOP_AVERAGE) return EXACT_ERR_INVALID_ARG;
    if (o.t0 < 0 || o.total_iters < 0 || (long long)o.t0 + iters > INT_MAX / 2) return EXACT_ERR_INVALID_ARG;
    if (o.launch != 0 && o.launch != 1) return EXACT_ERR_INVALID_ARG;
    if (o.resume && (reinterpret_cast<uintptr_t>(o.resume) & 7u)) return EXACT_ERR_INVALID_ARG;
    const int t0 = o.t0, t_end = o.t0 + iters;
    const int T = o.total_iters > 0 ? o.total_iters : t_end;
    if (T < t_end) return EXACT_ERR_INVALID_ARG;
    const bool running = o.stop_rule == EXACT_STOP_AVERAGE;
    if (running && (o.average_tail || !o.history || o.history_cap < (t_end / 2 > 1 ? t_end / 2 : 1)))
        return EXACT_ERR_INVALID_ARG;
    if (isnan(o.tv_bound) || o.tv_bound < 0.0 || o.tv_bound == INFINITY) return EXACT_ERR_INVALID_ARG;
    if (isnan(o.prox_lambda) || o.prox_lambda < 0.0 || o.prox_lambda == INFINITY) return EXACT_ERR_INVALID_ARG;
    const bool proxm = o.prox_lambda > 0.0;
    if (proxm && o.tv_bound > 0.0) return EXACT_ERR_INVALID_ARG;
    const bool tvb = o.tv_bound > 0.0 || proxm;  // both run the TV kernel after an unprojected step
    if (tvb && (o.tv.fgp_iters < 1 || o.tv.max_bisect < 1 || o.tv.max_dykstra < 0 || !(o.tv.tol_tv >= 0.0) ||
                !(o.tv.tol_dykstra >= 0.0) || isnan(o.tv.lam0) || o.tv.lam0 == INFINITY))
        return EXACT_ERR_INVALID_ARG;
    if (tvb && o.average_tail) return EXACT_ERR_UNSUPPORTED;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    if (tvb && !P.tv_ws) return EXACT_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    EXACT_TRY(cudaStreamIsCapturing(s, &cap));
    const float lo = (float)o.lo, hi = (float)o.hi;
    const LinkCoef coef = make_coef(P, I0);
    const int avg_from = T / 2;
    const int nb = adjoint_blocks(P.g.nx, P.g.ny);
    const bool averaging = o.average_tail || running;
    // state continued across calls of one solve: the averaging sums [d] and
    // the lam pair of the TV projections
    double *avg = o.resume ? static_cast<double *>(o.resume) : P.avg;
    double *tv_lam = o.resume ? static_cast<double *>(o.resume) + P.d : P.tv_lam;

    EXACT_TRY(launch_reset_state(P.state, t0, t_end, o.tol, o.check_every, o.stop_rule, avg_from, s));
    EXACT_TRY(reset_split_counts(P, s));
    EXACT_TRY(launch_collapse(y, y_dtype, P.W, P.n, P.Y, s));
    EXACT_TRY(launch_pack(x, P.xr[0], P.xc[0], P.g.nx, P.g.ny, P.ldr(), P.ldc(), lo, hi, true, s));
    EXACT_TRY(cudaMemsetAsync(P.xr[1], 0, sizeof(float) * (size_t)(P.g.ny * P.ldr()), s));
    EXACT_TRY(cudaMemsetAsync(P.xc[1], 0, sizeof(float) * (size_t)(P.g.nx * P.ldc()), s));
    if (averaging && t0 == 0) EXACT_TRY(cudaMemsetAsync(avg, 0, sizeof(double) * (size_t)P.d, s));
    TvLaunch tvl;
    memset(&tvl, 0, sizeof(tvl));
    if (tvb) {
        if (t0 == 0) {
            const double lam2[2] = {proxm ? o.prox_lambda : o.tv.lam0, proxm ? o.prox_lambda : o.tv.lam0};
            EXACT_TRY(cudaMemcpyAsync(tv_lam, lam2, sizeof(lam2), cudaMemcpyHostToDevice, s));
        }
        tvl.nx = P.g.nx;
        tvl.ny = P.g.ny;
        tvl.grid = P.tv_grid;
        tvl.z = P.tv_step;
        tvl.ldr = P.ldr();
        tvl.ldc = P.ldc();
        tvl.ws = P.tv_ws;
        tvl.state = P.state;
        tvl.tau = o.tv_bound;
        tvl.tol_tv = o.tv.tol_tv;
        tvl.tol_dykstra = o.tv.tol_dykstra;
        tvl.fgp_iters = o.tv.fgp_iters;
        tvl.max_bisect = o.tv.max_bisect;
        tvl.max_dykstra = o.tv.max_dykstra;
        tvl.lo = lo;
        tvl.hi = hi;
        tvl.fixed_lam = proxm ? 1 : 0;
    }

    FwdArgs f;
    memset(&f, 0, sizeof(f));
    f.rays = P.rays_f;
    f.bits = P.ray_bits;
    f.delta = P.ray_delta;
    f.units = P.units;
    f.kstart = P.kstart;
    f.n_units = P.n_units;
    f.err = P.state;
    f.n = P.n;
    f.Y = P.Y;
    f.r = P.r;
    f.K = P.K;
    f.M = P.bg_M;
    f.bg = P.bg_p;
    f.state = P.state;
    AdjArgs a;
    memset(&a, 0, sizeof(a));
    a.rays = P.rays_f;
    a.walk = P.rays_w;
    a.nsplit = P.adj_split;
    a.split_part = P.split_part;
    a.split_count = P.split_count;
    adj_views(a, P);
    a.n_views = P.g.n_views;
    a.n_bins = P.g.n_bins;
    a.nx = P.g.nx;
    a.ny = P.g.ny;
    a.r = P.r;
    a.scale = (float)(-eta / ((double)P.W * (double)P.n));
    a.base_r = P.xr[0];
    a.ldr = P.ldr();
    a.ldc = P.ldc();
    a.lo = lo;
    a.hi = hi;
    a.partials = P.partials;
    a.avg = averaging ? avg : nullptr;
    a.avg_from = avg_from;
    a.state = P.state;
    a.hist = running ? o.history : nullptr;
    a.hist_cap = o.history_cap;
    a.hist_drop = -1;
    const bool fan = P.g.beam == 1;

    // One iteration (Eq. (11)): forward+link on x_t, half step into x_{t+1/2},
    // forward+link on x_{t+1/2}, full step from x_t, FP64 stopping reduction.
    // in_graph: captured into a CUDA graph loop, where the iteration index
    // comes from the device state and the reduction sets the loop condition.
    auto iteration = [&](int t, bool in_graph, cudaGraphConditionalHandle cond, cudaStream_t q) -> exact_status {
        int u;
        a.iter_from_state = in_graph ? 1 : 0;
        f.img = img_of(P, 0);
        u = in_graph ? -1 : prof_begin(P, 0, t, q);
        EXACT_TRY(launch_forward(f, true, &coef, P.maps_r[0], P.maps_c[0], q));
        prof_end(P, u, q);
        a.out_r = P.xr[1];
        a.out_c = P.xc[1];
        a.iter = t;
        u = in_graph ? -1 : prof_begin(P, 1, t, q);
        if (tvb) {
            // unprojected half step, then its projection onto the TV ball ∩ box
            a.out = P.tv_step;
            EXACT_TRY(launch_adjoint(a, ADJ_STEP, fan, q));
            tvl.out_r = P.xr[1];
            tvl.out_c = P.xc[1];
            tvl.old_r = nullptr;
            tvl.hist = nullptr;
            tvl.lam_io = tv_lam;
            EXACT_TRY(launch_tv_project(tvl, q));
        } else {
            EXACT_TRY(launch_adjoint(a, ADJ_EG, fan, q));
        }
        prof_end(P, u, q);
        f.img = img_of(P, 1);
        u = in_graph ? -1 : prof_begin(P, 0, t, q);
        EXACT_TRY(launch_forward(f, true, &coef, P.maps_r[1], P.maps_c[1], q));
        prof_end(P, u, q);
        a.out_r = P.xr[0];
        a.out_c = P.xc[0];
        if (running && !in_graph) {
            // iterate number it = t + 1 enters the window of the last
            // m = max(1, floor(it/2)); when m did not grow, x_{it-m} leaves it
            const int it = t + 1, m = it / 2 > 1 ? it / 2 : 1, mp = (it - 1) / 2 > 1 ? (it - 1) / 2 : 1;
            a.hist_put = it % o.history_cap;
            a.hist_drop = (it >= 2 && m == mp) ? (it - m) % o.history_cap : -1;
            a.inv_m = 1.0 / (double)m;
            a.inv_m_prev = it >= 2 ? 1.0 / (double)mp : 0.0;
        }
        u = in_graph ? -1 : prof_begin(P, 2, t, q);
        if (tvb) {
            // unprojected full step from x_t, projected into x_t's padded
            // copies (each pixel's old value is read first for the norms)
            a.out = P.tv_step;
            EXACT_TRY(launch_adjoint(a, ADJ_STEP, fan, q));
            tvl.out_r = P.xr[0];
            tvl.out_c = P.xc[0];
            tvl.old_r = P.xr[0];
            tvl.norm_part = P.partials;
            tvl.lam_io = tv_lam + 1;
            tvl.avg = a.avg;
            tvl.hist = a.hist;
            tvl.hist_put = a.hist_put;
            tvl.hist_drop = a.hist_drop;
            tvl.inv_m = a.inv_m;
            tvl.inv_m_prev = a.inv_m_prev;
            EXACT_TRY(launch_tv_project(tvl, q));
        } else {
            EXACT_TRY(launch_adjoint(a, ADJ_EG_FINAL, fan, q));
        }
        prof_end(P, u, q);
        u = in_graph ? -1 : prof_begin(P, 3, t, q);
        if (in_graph)
            EXACT_TRY(launch_solve_reduce_cond(P.partials, nb, P.state, cond, q));
        else
            EXACT_TRY(launch_solve_reduce(P.partials, tvb ? P.tv_grid : nb, P.state, t, q));
        prof_end(P, u, q);
        return EXACT_OK;
    };

    const bool use_graph =
        iters > 0 && o.launch == 0 && !tvb && P.prof_every <= 0 && cap == cudaStreamCaptureStatusNone;
    if (use_graph) {
        // everything the loop's kernels take as arguments, except what they
        // read from the device state (iteration index, stopping test, bounds)
        struct Key {
            LinkCoef coef;
            float scale, lo, hi;
            int nsplit, fan, running, averaging, hist_cap, bg_M, pad;
            const void *avg, *hist, *bg_p;
        } key;
        memset(&key, 0, sizeof(key));
        key.coef = coef;
        key.scale = a.scale;
        key.lo = lo;
        key.hi = hi;
        key.nsplit = a.nsplit;
        key.fan = fan;
        key.running = running;
        key.averaging = averaging;
        key.hist_cap = o.history_cap;
        key.bg_M = P.bg_M;
        key.avg = a.avg;
        key.hist = a.hist;
        key.bg_p = P.bg_p;
        st = launch_solve_graph(P, &key, sizeof(key),
                                [&](cudaGraphConditionalHandle cond, cudaStream_t q) {
                                    return iteration(t0, true, cond, q);
                                },
                                s);
        if (st != EXACT_OK) return st;
    } else {
        for (int t = t0; t < t_end; ++t) {
            st = iteration(t, false, cudaGraphConditionalHandle{}, s);
            if (st != EXACT_OK) return st;
        }
    }
    EXACT_TRY(launch_unpack(P.xr[0], P.ldr(), P.g.nx, P.g.ny, x, averaging ? avg : nullptr, P.state,
                            running ? -1 : avg_from, s));
    if (o.x_last) EXACT_TRY(launch_unpack(P.xr[0], P.ldr(), P.g.nx, P.g.ny, o.x_last, nullptr, P.state, 0, s));
    if (info) {
        st = enqueue_info(P.state, P.host_state, info, P.captured_infos, s);
        if (st != EXACT_OK) return st;
    }
    return EXACT_OK;
}

exact_status exact_solve_host(exact_plan_t plan, const void *y_host, exact_dtype y_dtype, double I0, double eta,
                              int iters, const exact_solve_opts *opts, float *x_host, exact_solve_info *info,
                              exact_stream_t stream)
{
    exact_status st = check_plan(plan, true);
    if (st != EXACT_OK) return st;
    if (!y_host || !x_host) return EXACT_ERR_INVALID_ARG;
    if (y_dtype != EXACT_F32 && y_dtype != EXACT_BF16) return EXACT_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    EXACT_TRY(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return EXACT_ERR_UNSUPPORTED;  // it synchronises
    const size_t ybytes = (size_t)P.W * (size_t)P.n * (y_dtype == EXACT_BF16 ? 2 : 4);
    const size_t xbytes = sizeof(float) * (size_t)P.d;
    EXACT_TRY(cudaMemcpyAsync(P.stage_y, y_host, ybytes, cudaMemcpyHostToDevice, s));
    EXACT_TRY(cudaMemcpyAsync(P.stage_x, x_host, xbytes, cudaMemcpyHostToDevice, s));
    st = exact_solve(plan, P.stage_y, y_dtype, I0, eta, iters, opts, P.stage_x, info, stream);
    if (st != EXACT_OK) {
        cudaStreamSynchronize(s);
        return st;
    }
    EXACT_TRY(cudaMemcpyAsync(x_host, P.stage_x, xbytes, cudaMemcpyDeviceToHost, s));
    EXACT_TRY(cudaStreamSynchronize(s));
    return EXACT_OK;
}

exact_status exact_norm_estimate(exact_plan_t plan, int max_iters, double rtol, double *normA_sq, int *iters_done,
                                 exact_stream_t stream)
{
    exact_status st = check_plan(plan, true);
    if (st != EXACT_OK) return st;
    if (!normA_sq || max_iters < 1 || !isfin(rtol) || rtol < 0.0) return EXACT_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int nb_adj = adjoint_blocks(P.g.nx, P.g.ny);
    const int nb_fwd = forward_d_blocks(P.n);
    const int nb_adj_d = adjoint_d_blocks(P.g.nx, P.g.ny);
    double *pz = P.partials + kPartStride * (nb_adj > P.tv_grid ? nb_adj : P.tv_grid);
    double *pw = pz + nb_fwd;
    const bool fan = P.g.beam == 1;
    EXACT_TRY(launch_power_init(P.xrd, P.xcd, P.g.nx, P.g.ny, P.ldr(), P.ldc(), P.state, s));
    const int chunk = 8;
    for (int it0 = 0; it0 < max_iters; it0 += chunk) {
        const int it1 = it0 + chunk < max_iters ? it0 + chunk : max_iters;
        for (int it = it0; it < it1; ++it) {
            EXACT_TRY(launch_forward_d(P.rays_d, P.n, P.xrd, P.xcd, P.g.nx, P.g.ny, P.ldr(), P.ldc(), P.zd, pz,
                                       P.state, s));
            EXACT_TRY(launch_adjoint_d(P.rays_d, P.views, P.g.n_views, P.g.n_bins, P.g.nx, P.g.ny, P.zd, P.xrd,
                                       P.xcd, P.ldr(), P.ldc(), pw, P.state, fan, s));
            EXACT_TRY(launch_power_reduce(pz, nb_fwd, pw, nb_adj_d, P.state, it, rtol, s));
        }
        EXACT_TRY(cudaMemcpyAsync(P.host_state, P.state, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        EXACT_TRY(cudaStreamSynchronize(s));
        if (P.host_state->done) break;
    }
    if (P.host_state->status != EXACT_OK) return (exact_status)P.host_state->status;
    *normA_sq = P.host_state->lam;
    if (iters_done) *iters_done = P.host_state->iters_done;
    return EXACT_OK;
}

exact_status exact_norm_estimate_f32(exact_plan_t plan, int max_iters, double rtol, double *normA_sq,
                                     int *iters_done, exact_stream_t stream)
{
    exact_status st = check_plan(plan, true);
    if (st != EXACT_OK) return st;
    if (!normA_sq || max_iters < 1 || !isfin(rtol) || rtol < 0.0) return EXACT_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int nb_adj = adjoint_blocks(P.g.nx, P.g.ny);
    double *pz = P.partials + kPartStride * (nb_adj > P.tv_grid ? nb_adj : P.tv_grid);
    double *pw = pz + (forward_d_blocks(P.n) > kSumsqParts ? forward_d_blocks(P.n) : kSumsqParts);
    EXACT_TRY(launch_power_init_f(P.w32, P.d, P.state, s));
    FwdArgs f;
    memset(&f, 0, sizeof(f));
    f.img = img_of(P, 0);
    f.rays = P.rays_f;
    f.bits = P.ray_bits;
    f.delta = P.ray_delta;
    f.units = P.units;
    f.kstart = P.kstart;
    f.n_units = P.n_units;
    f.err = P.state;
    f.state = P.state;
    f.n = P.n;
    f.z = P.r;
    AdjArgs a;
    memset(&a, 0, sizeof(a));
    a.rays = P.rays_f;
    a.walk = P.rays_w;
    a.nsplit = P.adj_split;
    a.split_part = P.split_part;
    a.split_count = P.split_count;
    adj_views(a, P);
    a.n_views = P.g.n_views;
    a.n_bins = P.g.n_bins;
    a.nx = P.g.nx;
    a.ny = P.g.ny;
    a.r = P.r;
    a.delta = P.ray_delta;
    a.scale = 1.0f;
    a.out = P.w32;
    a.state = P.state;
    EXACT_TRY(reset_split_counts(P, s));
    const int chunk = 8;
    for (int it0 = 0; it0 < max_iters; it0 += chunk) {
        const int it1 = it0 + chunk < max_iters ? it0 + chunk : max_iters;
        for (int it = it0; it < it1; ++it) {
            // v_k = w_k / ||w_k|| into the padded copies, z = A v_k, w_{k+1} = A^T z
            EXACT_TRY(launch_pack(P.w32, P.xr[0], P.xc[0], P.g.nx, P.g.ny, P.ldr(), P.ldc(), 0.f, 0.f, false, s,
                                  &P.state->inv_norm));
            EXACT_TRY(launch_forward(f, false, nullptr, P.maps_r[0], P.maps_c[0], s));
            EXACT_TRY(launch_sumsq(P.r, P.n, pz, kSumsqParts, s));
            EXACT_TRY(launch_adjoint(a, ADJ_PLAIN, P.g.beam == 1, s));
            EXACT_TRY(launch_sumsq(P.w32, P.d, pw, kSumsqParts, s));
            EXACT_TRY(launch_power_reduce(pz, kSumsqParts, pw, kSumsqParts, P.state, it, rtol, s));
        }
        EXACT_TRY(cudaMemcpyAsync(P.host_state, P.state, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        EXACT_TRY(cudaStreamSynchronize(s));
        if (P.host_state->done) break;
    }
    if (P.host_state->status != EXACT_OK) return (exact_status)P.host_state->status;
    *normA_sq = P.host_state->lam;
    if (iters_done) *iters_done = P.host_state->iters_done;
    return EXACT_OK;
}

exact_status exact_recommended_eta(exact_plan_t plan, double I0, double normA_sq, double *eta)
{
    if (!plan || !eta || !isfin(I0) || !(I0 > 0.0) || !isfin(normA_sq) || !(normA_sq > 0.0))
        return EXACT_ERR_INVALID_ARG;
    const Plan *P = reinterpret_cast<const Plan *>(plan);
    const double m = (double)P->W * (double)P->n;
    const double L = I0 * normA_sq / m * P->Csum_mu;
    *eta = 1.0 / (4.0 * L);
    return EXACT_OK;
}

exact_status exact_plan_set_background(exact_plan_t plan, int n_materials, const double *mu_bg, const float *p)
{
    if (!plan || n_materials < 0 || n_materials > kMaxBg) return EXACT_ERR_INVALID_ARG;
    Plan *P = reinterpret_cast<Plan *>(plan);
    if (n_materials == 0) {
        P->bg_M = 0;
        P->bg_p = nullptr;
        return EXACT_OK;
    }
    if (!mu_bg || !p) return EXACT_ERR_INVALID_ARG;
    for (int q = 0; q < n_materials * P->K; ++q)
        if (!isfin(mu_bg[q]) || mu_bg[q] < 0.0) return EXACT_ERR_INVALID_ARG;
    for (int m = 0; m < n_materials; ++m)
        for (int k = 0; k < P->K; ++k) P->bg_mu2[m][k] = (float)(mu_bg[m * P->K + k] * 1.4426950408889634);
    P->bg_M = n_materials;
    P->bg_p = p;
    return EXACT_OK;
}

exact_status exact_plan_nnz(exact_plan_t plan, long long *nnz)
{
    if (!plan || !nnz) return EXACT_ERR_INVALID_ARG;
    Plan *P = reinterpret_cast<Plan *>(plan);
    if (P->nnz == 0) P->nnz = count_nnz(P->g);
    *nnz = P->nnz;
    return EXACT_OK;
}

exact_status exact_profile_enable(exact_plan_t plan, int sample_every)
{
    exact_status st = check_plan(plan, false);
    if (st != EXACT_OK) return st;
    if (sample_every < 0) return EXACT_ERR_INVALID_ARG;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    if (sample_every > 0 && !P.prof_ev) {
        const int cap = 4096;
        P.prof_ev = new (std::nothrow) cudaEvent_t[2 * cap];
        P.prof_kind = new (std::nothrow) int[cap];
        if (!P.prof_ev || !P.prof_kind) {
            delete[] P.prof_ev;
            delete[] P.prof_kind;
            P.prof_ev = nullptr;
            P.prof_kind = nullptr;
            return EXACT_ERR_OOM;
        }
        for (int i = 0; i < 2 * cap; ++i) {
            if (cudaEventCreate(&P.prof_ev[i]) != cudaSuccess) {
                P.prof_cap = i / 2;
                prof_free(P);
                return EXACT_ERR_OOM;
            }
        }
        P.prof_cap = cap;
        P.prof_used = 0;
    }
    P.prof_every = sample_every;
    return EXACT_OK;
}

exact_status exact_profile_read(exact_plan_t plan, double *ms, long long *launches)
{
    exact_status st = check_plan(plan, false);
    if (st != EXACT_OK) return st;
    Plan &P = *reinterpret_cast<Plan *>(plan);
    double acc[EXACT_PROF_KINDS] = {0.0};
    long long cnt[EXACT_PROF_KINDS] = {0};
    for (int u = 0; u < P.prof_used; ++u) {
        float t = 0.0f;
        EXACT_TRY(cudaEventSynchronize(P.prof_ev[2 * u + 1]));
        EXACT_TRY(cudaEventElapsedTime(&t, P.prof_ev[2 * u], P.prof_ev[2 * u + 1]));
        acc[P.prof_kind[u]] += t;
        cnt[P.prof_kind[u]] += 1;
    }
    P.prof_used = 0;
    for (int k = 0; k < EXACT_PROF_KINDS; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = cnt[k];
    }
    return EXACT_OK;
}

}  // extern "C"

// ================================================================ batches

namespace {

// Host staging and its device mirror share this layout (one copy per call).
struct BatchLayout {
    size_t jobs, maps, coefs, prefix, total;
};

BatchLayout batch_layout(int max_jobs)
{
    BatchLayout L;
    size_t off = 0;
    L.jobs = off;
    off = align_up(off + sizeof(BatchJob) * (size_t)max_jobs);
    L.maps = off;
    off = align_up(off + sizeof(CUtensorMap) * 4 * (size_t)max_jobs);
    L.coefs = off;
    off = align_up(off + sizeof(LinkCoef) * (size_t)max_jobs);
    L.prefix = off;
    off = align_up(off + sizeof(int) * (5 * (size_t)max_jobs + 1));
    L.total = off;
    return L;
}

}  // namespace

struct exact_batch {
    int device = -1;
    int max_jobs = 0;
    BatchLayout L;
    char *host = nullptr;   // pinned staging
    char *dev = nullptr;    // device mirror
    unsigned long long *next = nullptr;
    unsigned *done_items = nullptr;
    int *abort_flag = nullptr;
    char *counters = nullptr;
    size_t counter_bytes = 0;
    cudaEvent_t staged = nullptr;
    bool staged_pending = false;
    int grid = 0;
    // 0: persistent kernel, one CTA per adjoint tile; 1: persistent kernel,
    // each plan's adj_split; 2: each job's exact_solve on one of `streams`
    // (exact_batch_autotune / exact_batch_set_policy)
    int split_policy = 0;
    std::vector<void *> captured_infos;  // info payloads of captured graphs
    cudaStream_t streams[kBatchStreams] = {};
    cudaEvent_t fork = nullptr, joins[kBatchStreams] = {};
};

extern "C" {

exact_status exact_batch_create(int max_jobs, exact_batch_t *out)
{
    if (!out) return EXACT_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_jobs < 1 || max_jobs > kMaxBatch) return EXACT_ERR_INVALID_ARG;
    exact_batch *B = new (std::nothrow) exact_batch();
    if (!B) return EXACT_ERR_OOM;
    if (cudaGetDevice(&B->device) != cudaSuccess) {
        delete B;
        return EXACT_ERR_CUDA;
    }
    B->max_jobs = max_jobs;
    B->L = batch_layout(max_jobs);
    B->counter_bytes = align_up(sizeof(unsigned long long)) + align_up(sizeof(unsigned) * (size_t)max_jobs) +
                       align_up(sizeof(int));
    cudaError_t e = cudaMallocHost(&B->host, B->L.total);
    if (e == cudaSuccess) e = cudaMalloc(&B->dev, B->L.total);
    if (e == cudaSuccess) e = cudaMalloc(&B->counters, B->counter_bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->staged, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    for (int k = 0; k < kBatchStreams && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&B->streams[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->joins[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        exact_batch_destroy(B);
        return cuda_status(e);
    }
    memset(B->host, 0, B->L.total);
    B->next = reinterpret_cast<unsigned long long *>(B->counters);
    B->done_items = reinterpret_cast<unsigned *>(B->counters + align_up(sizeof(unsigned long long)));
    B->abort_flag = reinterpret_cast<int *>(B->counters + align_up(sizeof(unsigned long long)) +
                                            align_up(sizeof(unsigned) * (size_t)max_jobs));
    B->grid = batch_grid_size();
    *out = B;
    return EXACT_OK;
}

exact_status exact_batch_destroy(exact_batch_t B)
{
    if (!B) return EXACT_OK;
    if (B->staged) cudaEventDestroy(B->staged);
    if (B->fork) cudaEventDestroy(B->fork);
    for (int k = 0; k < kBatchStreams; ++k) {
        if (B->joins[k]) cudaEventDestroy(B->joins[k]);
        if (B->streams[k]) cudaStreamDestroy(B->streams[k]);
    }
    for (void *c : B->captured_infos) delete static_cast<InfoCopy *>(c);
    if (B->host) cudaFreeHost(B->host);
    if (B->dev) cudaFree(B->dev);
    if (B->counters) cudaFree(B->counters);
    delete B;
    return EXACT_OK;
}

exact_status exact_batch_solve(exact_batch_t B, const exact_job *jobs, int n_jobs, exact_stream_t stream)
{
    if (!B || !jobs || n_jobs < 1 || n_jobs > B->max_jobs) return EXACT_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return EXACT_ERR_CUDA;
    if (dev != B->device) return EXACT_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rounds = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const exact_job &J = jobs[j];
        exact_status st = check_plan(J.plan, true);
        if (st != EXACT_OK) return st;
        if (!J.y || !J.x) return EXACT_ERR_INVALID_ARG;
        if (J.y_dtype != EXACT_F32 && J.y_dtype != EXACT_BF16) return EXACT_ERR_INVALID_ARG;
        if (!isfin(J.I0) || !(J.I0 > 0.0) || !isfin(J.eta) || !(J.eta > 0.0) || J.iters < 0)
            return EXACT_ERR_INVALID_ARG;
        const exact_solve_opts &o = J.opts;
        if (isnan(o.lo) || isnan(o.hi) || o.lo > o.hi || o.lo == INFINITY || o.hi == -INFINITY)
            return EXACT_ERR_INVALID_ARG;
        if (!isfin(o.tol) || o.tol < 0.0 || o.check_every < 0) return EXACT_ERR_INVALID_ARG;
        if (o.average_tail || o.stop_rule != EXACT_STOP_RESIDUAL || o.tv_bound != 0.0 || o.prox_lambda != 0.0 ||
            o.t0 != 0 || o.total_iters != 0 || o.resume || o.x_last)
            return EXACT_ERR_UNSUPPORTED;
        for (int q = 0; q < j; ++q)
            if (jobs[q].plan == J.plan) return EXACT_ERR_INVALID_ARG;
        rounds = J.iters > rounds ? J.iters : rounds;
    }
    if (B->split_policy == 2) {
        // each job's own solve (its graph loop and adj_split) on one of the
        // context's streams, round robin; forked from and joined back into
        // `stream` with events, so the call stays ordered on `stream` (and
        // capturable).  Each job's arithmetic is that of exact_solve.
        const int K = n_jobs < kBatchStreams ? n_jobs : kBatchStreams;
        EXACT_TRY(cudaEventRecord(B->fork, s));
        for (int k = 0; k < K; ++k) EXACT_TRY(cudaStreamWaitEvent(B->streams[k], B->fork, 0));
        exact_status st = EXACT_OK;
        for (int j = 0; j < n_jobs && st == EXACT_OK; ++j) {
            const exact_job &J = jobs[j];
            st = exact_solve(J.plan, J.y, J.y_dtype, J.I0, J.eta, J.iters, &J.opts, J.x, J.info,
                             reinterpret_cast<exact_stream_t>(B->streams[j % K]));
        }
        // join every forked stream, also after a failed call
        for (int k = 0; k < K; ++k) {
            const cudaError_t e = cudaEventRecord(B->joins[k], B->streams[k]);
            const cudaError_t w = e == cudaSuccess ? cudaStreamWaitEvent(s, B->joins[k], 0) : e;
            if (w != cudaSuccess && st == EXACT_OK) st = cuda_status(w);
        }
        return st;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    EXACT_TRY(cudaStreamIsCapturing(s, &cap));
    // the previous call's staging copy must have left the host buffer
    if (B->staged_pending && cap == cudaStreamCaptureStatusNone) {
        EXACT_TRY(cudaEventSynchronize(B->staged));
        B->staged_pending = false;
    }

    BatchJob *hj = reinterpret_cast<BatchJob *>(B->host + B->L.jobs);
    CUtensorMap *hm = reinterpret_cast<CUtensorMap *>(B->host + B->L.maps);
    LinkCoef *hc = reinterpret_cast<LinkCoef *>(B->host + B->L.coefs);
    int *hp = reinterpret_cast<int *>(B->host + B->L.prefix);
    const CUtensorMap *dm = reinterpret_cast<const CUtensorMap *>(B->dev + B->L.maps);
    const LinkCoef *dc = reinterpret_cast<const LinkCoef *>(B->dev + B->L.coefs);
    for (int j = 0; j < n_jobs; ++j) {
        const exact_job &Jb = jobs[j];
        Plan &P = *reinterpret_cast<Plan *>(Jb.plan);
        BatchJob &J = hj[j];
        memset(&J, 0, sizeof(J));
        J.img[0] = img_of(P, 0);
        J.img[1] = img_of(P, 1);
        for (int q = 0; q < 2; ++q) {
            J.xr[q] = P.xr[q];
            J.xc[q] = P.xc[q];
        }
        hm[4 * j + 0] = P.maps_r[0];
        hm[4 * j + 1] = P.maps_c[0];
        hm[4 * j + 2] = P.maps_r[1];
        hm[4 * j + 3] = P.maps_c[1];
        J.maps = dm + 4 * j;
        hc[j] = make_coef(P, Jb.I0);
        J.coef = dc + j;
        J.state = P.state;
        J.f.rays = P.rays_f;
        J.f.bits = P.ray_bits;
        J.f.delta = P.ray_delta;
        J.f.units = P.units;
        J.f.kstart = P.kstart;
        J.f.n_units = P.n_units;
        J.f.err = P.state;
        J.f.n = P.n;
        J.f.Y = P.Y;
        J.f.r = P.r;
        J.f.K = P.K;
        J.f.M = P.bg_M;
        J.f.bg = P.bg_p;
        J.a.rays = P.rays_f;
        J.a.walk = P.rays_w;
        adj_views(J.a, P);
        J.a.n_views = P.g.n_views;
        J.a.n_bins = P.g.n_bins;
        J.a.nx = P.g.nx;
        J.a.ny = P.g.ny;
        J.a.r = P.r;
        J.a.scale = (float)(-Jb.eta / ((double)P.W * (double)P.n));
        J.a.base_r = P.xr[0];
        J.a.ldr = P.ldr();
        J.a.ldc = P.ldc();
        J.a.lo = (float)Jb.opts.lo;
        J.a.hi = (float)Jb.opts.hi;
        J.a.partials = P.partials;
        J.a.state = P.state;
        J.n_units = P.n_units;
        J.tiles_x = (P.g.nx + kTW - 1) / kTW;
        J.tiles_y = (P.g.ny + kTH - 1) / kTH;
        J.fan = P.g.beam == 1;
        J.iters = Jb.iters;
        J.check_every = Jb.opts.check_every;
        J.tol = Jb.opts.tol;
        J.nsplit = B->split_policy == 1 ? P.adj_split : 1;
        J.a.nsplit = J.nsplit;
        J.a.split_part = P.split_part;
        J.a.split_count = P.split_count;
        const int T = J.tiles_x * J.tiles_y * J.nsplit, U = P.n_units;  // adjoint items: (tile, split)
        const int per[5] = {U, T, U, T, 1};
        J.phase_off[0] = 0;
        for (int p = 0; p < 5; ++p) J.phase_off[p + 1] = J.phase_off[p] + per[p];
    }
    long long run = 0;
    for (int p = 0; p < 5; ++p)
        for (int j = 0; j < n_jobs; ++j) {
            hp[p * n_jobs + j] = (int)run;
            run += hj[j].phase_off[p + 1] - hj[j].phase_off[p];
        }
    if (run >= (1LL << 31)) return EXACT_ERR_UNSUPPORTED;
    hp[5 * n_jobs] = (int)run;
    for (int j = 0; j < n_jobs; ++j)
        if ((unsigned long long)hj[j].phase_off[5] * (unsigned long long)(rounds + 1) >= (1ULL << 32))
            return EXACT_ERR_UNSUPPORTED;
    const int held = debug_take_batch_block();
    if (held >= 0 && held < n_jobs) hj[held].hold = (unsigned)hj[held].phase_off[5] * (unsigned)rounds + 1u;

    EXACT_TRY(cudaMemcpyAsync(B->dev, B->host, B->L.total, cudaMemcpyHostToDevice, s));
    if (cap == cudaStreamCaptureStatusNone) {
        EXACT_TRY(cudaEventRecord(B->staged, s));
        B->staged_pending = true;
    }
    EXACT_TRY(cudaMemsetAsync(B->counters, 0, B->counter_bytes, s));
    for (int j = 0; j < n_jobs; ++j) {
        const exact_job &Jb = jobs[j];
        Plan &P = *reinterpret_cast<Plan *>(Jb.plan);
        EXACT_TRY(launch_reset_state(P.state, 0, Jb.iters, Jb.opts.tol, Jb.opts.check_every, EXACT_STOP_RESIDUAL,
                                     Jb.iters / 2, s));
        EXACT_TRY(reset_split_counts(P, s));
        EXACT_TRY(launch_collapse(Jb.y, Jb.y_dtype, P.W, P.n, P.Y, s));
        EXACT_TRY(launch_pack(Jb.x, P.xr[0], P.xc[0], P.g.nx, P.g.ny, P.ldr(), P.ldc(), (float)Jb.opts.lo,
                              (float)Jb.opts.hi, true, s));
        EXACT_TRY(cudaMemsetAsync(P.xr[1], 0, sizeof(float) * (size_t)(P.g.ny * P.ldr()), s));
        EXACT_TRY(cudaMemsetAsync(P.xc[1], 0, sizeof(float) * (size_t)(P.g.nx * P.ldc()), s));
    }
    EXACT_TRY(launch_batch(reinterpret_cast<const BatchJob *>(B->dev + B->L.jobs), n_jobs,
                           reinterpret_cast<const int *>(B->dev + B->L.prefix), rounds, B->next, B->done_items,
                           B->abort_flag, B->grid, debug_wait_polls(), s));
    for (int j = 0; j < n_jobs; ++j) {
        const exact_job &Jb = jobs[j];
        Plan &P = *reinterpret_cast<Plan *>(Jb.plan);
        EXACT_TRY(launch_unpack(P.xr[0], P.ldr(), P.g.nx, P.g.ny, Jb.x, nullptr, P.state, 0, s));
        if (Jb.info) {
            exact_status st = enqueue_info(P.state, P.host_state, Jb.info, B->captured_infos, s);
            if (st != EXACT_OK) return st;
        }
    }
    return EXACT_OK;
}


exact_status exact_batch_set_policy(exact_batch_t B, int policy)
{
    if (!B || policy < 0 || policy > 2) return EXACT_ERR_INVALID_ARG;
    B->split_policy = policy;
    return EXACT_OK;
}

exact_status exact_batch_get_policy(exact_batch_t B, int *policy)
{
    if (!B || !policy) return EXACT_ERR_INVALID_ARG;
    *policy = B->split_policy;
    return EXACT_OK;
}

exact_status exact_batch_autotune(exact_batch_t B, const exact_job *jobs, int n_jobs, int *policy_out,
                                  exact_stream_t stream)
{
    if (!B || !jobs || n_jobs < 1 || n_jobs > B->max_jobs) return EXACT_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<exact_job> trial(jobs, jobs + n_jobs);
    for (exact_job &J : trial) {
        exact_status st = check_plan(J.plan, true);
        if (st != EXACT_OK) return st;
        if (!J.x) return EXACT_ERR_INVALID_ARG;
        J.iters = J.iters < 2 ? J.iters : 2;
        J.info = nullptr;
    }
    // each job's x is saved in its plan's scratch image and put back after
    // every trial, so the trials leave the jobs as they were
    for (const exact_job &J : trial) {
        const Plan &P = *reinterpret_cast<const Plan *>(J.plan);
        EXACT_TRY(cudaMemcpyAsync(P.w32, J.x, sizeof(float) * (size_t)P.d, cudaMemcpyDeviceToDevice, s));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return EXACT_ERR_CUDA;
    }
    const int keep = B->split_policy;
    float best_ms = INFINITY;
    int best = 0;
    exact_status st = EXACT_OK;
    for (int policy = 0; policy < 3 && st == EXACT_OK; ++policy) {
        B->split_policy = policy;
        float ms_min = INFINITY;
        for (int rep = 0; rep < 3 && st == EXACT_OK; ++rep) {
            float ms = 0.0f;
            cudaError_t e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) st = exact_batch_solve(B, trial.data(), n_jobs, stream);
            if (e == cudaSuccess && st == EXACT_OK) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess && st == EXACT_OK) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess && st == EXACT_OK) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) st = cuda_status(e);
            for (const exact_job &J : trial) {
                if (st != EXACT_OK) break;
                const Plan &P = *reinterpret_cast<const Plan *>(J.plan);
                e = cudaMemcpyAsync(J.x, P.w32, sizeof(float) * (size_t)P.d, cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) st = cuda_status(e);
            }
            if (rep > 0 && ms < ms_min) ms_min = ms;  // the first run of a policy warms up
        }
        if (st == EXACT_OK && ms_min < 0.97f * best_ms) {
            best_ms = ms_min;
            best = policy;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == EXACT_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e);
    }
    B->split_policy = st == EXACT_OK ? best : keep;
    if (policy_out) *policy_out = B->split_policy;
    return st;
}

}  // extern "C"
