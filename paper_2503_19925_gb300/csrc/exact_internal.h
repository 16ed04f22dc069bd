// exact_internal.h -- types shared by the host plan code and the kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

#include "../../include/exact.h"

namespace exact {

// Zero columns kept on each side of a padded image row so that a Joseph sample
// at cross index k0 in [-2, n_cross] can read k0 and k0+1 without a bounds test.
constexpr int kPad = 2;

// floor(v) of a float with |v| < 2^22 without the conversion pipe:
// r = v + 1.5 * 2^23 rounded down holds floor(v) in its low mantissa bits,
// floor(v) = r - kFloorMagic exactly and = bits(r) - kFloorBias as an integer.
constexpr float kFloorMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kFloorBias = 0x4B400000;      // bit pattern of kFloorMagic
constexpr int kMaxK = EXACT_MAX_ENERGY;
constexpr int kMaxBg = 4;  // known background materials per plan

// One ray of the Joseph projector, FP32 form.  The cross-axis pixel-index
// coordinate of the crossing at driving index j is t(j) = alpha + beta j
// (alpha, beta from FP64 geometry), stored split so that FP32 arithmetic keeps
// t accurate to ~1e-6 pixel at any image size:
//   alpha = A + a  (A an integer held exactly in a float, a in [0, 1]),
//   beta  = bh + bl (bh = beta rounded to FP32, bl the FP32 remainder).
// The matrix entries are delta * max(0, 1 - |t(j) - k|).
struct __align__(16) RayF {
    float A, a, bh, bl;
};

// Walk coefficients of one ray, for the adjoint's strip walk.  Along the rays
// of one view that share a driving axis, the crossing of driving line j is a
// Moebius function of the bin index: for bins b + e (e a small integer),
//   t_{b+e}(j) = t_b(j) + kappa e / (1 + sg e),   kappa = ka + kb j,
// with ka = d alpha / d b, kb = d beta / d b at bin b and sg the relative change
// of the ray's driving-axis direction component per bin (0 for parallel beams,
// where kb = 0 too).  Computed in FP64 on the host.
struct __align__(16) RayW {
    float ka, kb, sg, pad;
};

// Per-ray driving range and axis: bits 0-14 first driving index j_lo,
// 15-29 last j_hi, 30 driving axis (0: x drives, the image is read through the
// column-major copy; 1: y drives, row-major copy).  An empty range has
// j_lo > j_hi.
__host__ __device__ inline int ray_jlo(int bits) { return bits & 0x7fff; }
__host__ __device__ inline int ray_jhi(int bits) { return (bits >> 15) & 0x7fff; }
__host__ __device__ inline int ray_axis(int bits) { return (bits >> 30) & 1; }

// FP64 form (power iteration): t(j) = alpha + beta j in double.
struct __align__(16) RayD {
    double alpha, beta, delta;
    int bits, pad;
};

// Per-view back-projection table.  The continuous bin coordinate of the point
// at pixel-index position (kx, ky) is (n0 + n1 kx + n2 ky) / (d0 + d1 kx + d2 ky) + c
// (parallel beam: d0 = 1, d1 = d2 = 0).  Bins [xb0, xb1) hold the view's
// x-driven rays and [yb0, yb1) its y-driven rays (each contiguous: one of the
// two ranges is empty unless the fan crosses a diagonal).
struct __align__(16) ViewRec {
    float n0, n1, n2, c;
    float d0, d1, d2, pad;
    int xb0, xb1, yb0, yb1;
};

// Forward-projector work unit: up to kFR adjacent rays of one view with one
// driving axis.  The image band these rays cross in driving lines
// [c kFC, (c + 1) kFC) is staged in shared memory as a kFC x kFHB box whose
// first row is cross index kstart[koff + c - jc0] (a multiple of 4 after
// adding kPad, as the tensor-map x coordinate must be 16-byte aligned).
constexpr int kFR = 128;   // rays per unit (threads per CTA)
constexpr int kFC = 16;    // driving lines per staged chunk
constexpr int kFStages = 2;  // staging buffers (copies kFStages - 1 chunks ahead)
constexpr int kFHB = 192;  // staged cross-axis rows per chunk (tensor-map box height)
// Adjoint tile (pixels): one CTA gathers A^T r over kTW x kTH pixels.
constexpr int kTW = 32;
constexpr int kTH = 32;

struct __align__(16) FwdUnit {
    int ray0, count, axis, jc0;
    int nchunks, koff, pad0, pad1;
};

// Device-side status words of a solve or a norm estimate.
struct DevState {
    int done;         // nonzero: later kernels of this solve return at once
    int iters_done;
    int status;       // exact_status
    int pad;
    double rel_res;
    double lam;       // power iteration: latest ||A v||^2
    double lam_prev;
    double inv_norm;  // power iteration: 1/||w|| for the next forward
    double avg_change;  // running-average rule: ||xbar_t - xbar_{t-1}||
    // solve parameters, set at the start of a solve (k_reset_state): the
    // iteration index one past this call's last, the stopping test and the
    // first iteration index of the tail average (kernels launched from a
    // CUDA graph loop read these instead of per-launch arguments)
    int iter_end;
    int check_every;
    int rule;        // exact_stop_rule
    int avg_from;
    double tol;
};

// FP64 partial sums per adjoint tile of the full step: ||x_out - x_base||^2,
// ||x_base||^2 and ||xbar_t - xbar_{t-1}||^2 (running-average rule).
constexpr int kPartStride = 3;

// One instantiated solve graph (a WHILE node over the iteration's kernels),
// kept by the plan for relaunch while its key -- the kernel arguments that do
// not come from the device state -- stays the same.
struct SolveGraph {
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t last = nullptr;  // recorded after its latest launch
    std::vector<unsigned char> key;
    unsigned long long stamp = 0;  // last use (least recently used is replaced first)
};
constexpr int kSolveGraphs = 4;

struct Plan {
    exact_geometry g;
    int device = -1;
    int W = 0, K = 0;
    long long n = 0, d = 0;
    double Csum_mu = 0.0;          // sum_k mu_k sum_w S[w][k]
    float mu_log2e[kMaxK];         // mu_k * log2(e), FP32
    float C[kMaxK];                // sum_w S[w][k], FP32 (multiplied by I0 per call)
    RayF *rays_f = nullptr;        // [n]
    RayW *rays_w = nullptr;        // [n] walk coefficients (adjoint)
    int *ray_bits = nullptr;       // [n] driving range and axis
    float *ray_delta = nullptr;    // [n] step length delta
    RayD *rays_d = nullptr;        // [n]
    ViewRec *views = nullptr;      // [n_views]
    int *vitems = nullptr;         // [nxv + nyv]: views with x-driven rays, then views with y-driven rays
    int nxv = 0, nyv = 0;
    // workspace carve-up (all device pointers inside the bound workspace)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    float *xr[2] = {nullptr, nullptr};   // padded row-major copies   [ny][nx + 2 kPad]
    float *xc[2] = {nullptr, nullptr};   // padded column-major copies [nx][ny + 2 kPad]
    float *Y = nullptr;                  // collapsed counts [n]
    float *r = nullptr;                  // residual [n]
    double *partials = nullptr;          // per-block FP64 partial sums
    double *avg = nullptr;               // tail-average accumulator [d]
    float *tv_step = nullptr;            // unprojected step [d] (TV-ball solves)
    double *tv_lam = nullptr;            // [2] lam carried by the half- and full-step projections
    void *tv_ws = nullptr;               // workspace of the TV-ball projection
    int tv_grid = 0;                     // its cooperative grid
    float *split_part = nullptr;         // adjoint view split: partial tiles [tiles][max_split][kTH * kTW]
    int *split_count = nullptr;          // [tiles] arrival counts (zeroed when the workspace is bound)
    int adj_split = 1;                   // CTAs per adjoint tile (exact_plan_autotune / set_tuning)
    int max_split = 1;                   // largest adj_split the workspace's partial tiles allow
    float *stage_y = nullptr;            // exact_solve_host: device copy of the host counts [W][n]
    float *stage_x = nullptr;            // exact_solve_host: device copy of the host image [d]
    double *xrd = nullptr, *xcd = nullptr;  // FP64 padded copies (power iteration)
    double *zd = nullptr;                // FP64 projections [n]
    float *w32 = nullptr;                // FP32 power-iteration image [d]
    DevState *state = nullptr;
    // pinned host mirror of the device state (solve info)
    DevState *host_state = nullptr;
    long long nnz = 0;              // nonzero entries of A
    FwdUnit *units = nullptr;       // [n_units] forward work units
    int *kstart = nullptr;          // [n_kstart] staged band start per unit chunk
    int n_units = 0;
    // tensor maps of the padded copies: maps_r[q] over xr[q], maps_c[q] over xc[q]
    CUtensorMap maps_r[2], maps_c[2];
    int bg_M = 0;                    // known background (exact_plan_set_background)
    const float *bg_p = nullptr;     // caller-owned [bg_M][n]
    float bg_mu2[kMaxBg][kMaxK];     // mu_bg log2(e)
    std::vector<void *> captured_infos;  // solve-info payloads owned by captured graphs
    cudaStream_t cap_stream = nullptr;   // stream the solve graphs' loop bodies are captured on
    std::vector<SolveGraph> graphs;      // up to kSolveGraphs instantiated solve graphs
    unsigned long long graph_clock = 0;
    // kernel timing (profiling aid): event pairs recorded around sampled launches
    int prof_every = 0;
    int prof_used = 0;              // event pairs recorded since the last read
    int prof_cap = 0;
    cudaEvent_t *prof_ev = nullptr; // [2 * prof_cap]
    int *prof_kind = nullptr;       // [prof_cap]
    // padded row lengths, rounded up to 4 floats so rows start on 16-byte
    // boundaries (tensor-map strides must be multiples of 16 bytes)
    long long ldr() const { return (g.nx + 2 * kPad + 3) / 4 * 4; }
    long long ldc() const { return (g.ny + 2 * kPad + 3) / 4 * 4; }
};

// ---- launch parameter blocks -------------------------------------------------

struct ImgF {
    const float *xr;  // padded row-major (read by y-driven rays)
    const float *xc;  // padded column-major (read by x-driven rays)
    int nx, ny;
    long long ldr, ldc;
};

struct FwdArgs {
    ImgF img;
    const RayF *rays;
    const int *bits;
    const float *delta;
    const FwdUnit *units;
    const int *kstart;
    int n_units;
    DevState *err;          // where a timed-out staging wait is reported (may be null)
    long long n;
    float *z;             // z output (link == false)
    const float *Y;       // collapsed counts (link == true)
    float *r;             // residual output times delta (link == true)
    int K;
    int M;                  // known background materials (0: none)
    const float *bg;        // [M][n] their projections
    const DevState *state;  // may be null: if set and state->done, return
};

// Link coefficients passed by value (kernel parameter space).
struct LinkCoef {
    float mu2[kMaxK];          // mu_k log2(e)
    float c[kMaxK];            // I0 sum_w S[w][k]
    float mub[kMaxBg][kMaxK];  // known-background attenuation mu_bg[m][k] log2(e)
};

// PLAIN: out = scale A^T r; EG / EG_FINAL: projected extragradient step into
// the padded copies (FINAL adds the partial norms); STEP: out = x_base +
// scale A^T r unprojected (the TV-ball projection follows).
enum AdjMode { ADJ_PLAIN = 0, ADJ_EG = 1, ADJ_EG_FINAL = 2, ADJ_STEP = 3 };

struct AdjArgs {
    const RayF *rays;
    const RayW *walk;
    const ViewRec *views;
    // the views that have x-driven rays (vitems[0 .. nxv)) and those that
    // have y-driven rays (vitems[nxv .. nxv + nyv))
    const int *vitems;
    int nxv, nyv;
    int n_views, n_bins, nx, ny;
    const float *r;        // [n] residual; already times delta unless `delta` is set
    const float *delta;    // [n] or null: multiply r by delta on the fly
    float scale;           // out = scale * A^T r   (PLAIN)  |  x_base + scale * A^T r (EG)
    float *out;            // PLAIN: [ny][nx] output
    const float *base_r;   // EG: padded row-major base iterate x_t
    float *out_r;          // EG: padded row-major output
    float *out_c;          // EG: padded column-major output
    long long ldr, ldc;
    float lo, hi;
    double *partials;      // EG_FINAL: per-block (||x_out - x_base||^2, ||x_base||^2)
    double *avg;           // EG_FINAL: tail-average accumulator or null
    int avg_from;          // EG_FINAL: accumulate when iteration index >= avg_from
    int iter;              // iteration index of this launch
    // EG_FINAL, running-average rule (null hist: off).  avg holds the FP64
    // window sum; hist the ring of window iterates [cap][ny][nx]; this launch
    // stores x_out in slot hist_put and removes slot hist_drop (-1: none)
    // from the sum; the partials get ||sum / m - sum_prev / m_prev||^2.
    float *hist;
    int hist_put, hist_drop;
    double inv_m, inv_m_prev;
    // view split over CTAs (nsplit <= 1: one CTA per tile): partial tiles
    // [tiles][nsplit][kTH * kTW] and per-tile arrival counts (zero between launches)
    int nsplit;
    float *split_part;
    int *split_count;
    const DevState *state;
    // iter_from_state != 0 (launches inside a CUDA graph loop): the iteration
    // index is state->iters_done, avg_from is state->avg_from, and the
    // running-average slots follow from them and hist_cap (the ring length)
    int iter_from_state;
    int hist_cap;
};

constexpr int kMaxSplit = 16;  // view split of the adjoint (autotuned per plan)

// The plan's view tables in the adjoint's arguments.
inline void adj_views(AdjArgs &a, const Plan &P)
{
    a.views = P.views;
    a.vitems = P.vitems;
    a.nxv = P.nxv;
    a.nyv = P.nyv;
}

// One job of the persistent multi-job kernel (k_batch.cu).  A round of a job
// is one extragradient iteration: phase 0 forward+link on x_t (n_units items),
// 1 adjoint half step (n_tiles items), 2 forward+link on x_{t+1/2}, 3 adjoint
// full step, 4 reduction (1 item).
struct BatchJob {
    FwdArgs f;                 // img is set per phase
    AdjArgs a;                 // out_r/out_c/iter set per phase
    ImgF img[2];
    float *xr[2], *xc[2];
    const CUtensorMap *maps;   // [4] in global memory: rows 0, cols 0, rows 1, cols 1
    const LinkCoef *coef;      // global memory
    DevState *state;
    int n_units, tiles_x, tiles_y, fan, nsplit;
    int iters, check_every;
    double tol;
    int phase_off[6];          // items of the job before phase p within a round; [5] = items per round
    unsigned hold;             // fault injection: nonzero, phases >= 1 wait for this many completions
                               // (more than the job has items, so the wait runs out); 0: normal
};

// Fault injection for tests of the bounded device waits (exact_debug_inject):
// the poll limit of the batch dependency waits and the TV grid barriers (0:
// the built-in limits), and one-shot blocks of the next batch job / TV launch.
long long debug_wait_polls();
int debug_take_batch_block();  // job index to block in the next batch launch, or -1
bool debug_take_tv_block();    // block the next TV launch's grid barrier

constexpr int kBatchThreads = 128;  // = kFR, and 4 adjoint warps
constexpr int kMaxBatch = 256;      // jobs per batch launch
constexpr int kBatchStreams = 8;    // streams of a batch context (policy 2: one solve per stream at a time)

// ---- host helpers shared by the plan code (api.cu) and exact_operator_static --
// 2D tensor map of one padded image copy (box kFHB x kFC, zero fill outside).
bool encode_map(CUtensorMap *map, float *base, long long ld, long long lines);
// Link coefficients of a plan at source intensity I0.
LinkCoef make_coef(const Plan &P, double I0);

// ---- launchers (each returns cudaGetLastError()) ------------------------------
cudaError_t launch_forward(const FwdArgs &a, bool link, const LinkCoef *coef, const CUtensorMap &map_r,
                           const CUtensorMap &map_c, cudaStream_t s);
cudaError_t launch_adjoint(const AdjArgs &a, int mode, bool fan, cudaStream_t s);
int adjoint_blocks(int nx, int ny);    // blocks (= partial-norm pairs) of the FP32 adjoint
int adjoint_d_blocks(int nx, int ny);  // blocks (= partial sums) of the FP64 adjoint

cudaError_t launch_pack(const float *x, float *xr, float *xc, int nx, int ny, long long ldr, long long ldc,
                        float lo, float hi, bool project, cudaStream_t s, const double *scale = nullptr);
constexpr int kSumsqParts = 256;  // fixed partial count of the FP32 sums of squares
cudaError_t launch_sumsq(const float *v, long long n, double *partials, int nparts, cudaStream_t s);
cudaError_t launch_power_init_f(float *w, long long d, DevState *st, cudaStream_t s);
cudaError_t launch_unpack(const float *xr, long long ldr, int nx, int ny, float *x, const double *avg,
                          const DevState *state, int avg_from, cudaStream_t s);
cudaError_t launch_collapse(const void *y, int dtype, int W, long long n, float *Y, cudaStream_t s);
// Projection onto {||x||_TV <= tau} ∩ [lo, hi]^d (k_tv.cu).  The workspace
// (tv_workspace_bytes) holds 13 pixel arrays, FP64 partials and a TvTail.
struct TvTail {
    unsigned bar[2];  // grid barrier: arrivals, generation
    int status;       // standalone calls: EXACT_OK or EXACT_ERR_TIMEOUT
    int stats[2];     // Dykstra rounds, regularised solves of the last call
    int pad;
    double lam;       // standalone calls: lam in / out
};
struct TvLaunch {
    int nx, ny, grid;
    const float *z;
    float *out, *out_r, *out_c;  // any may be null
    long long ldr, ldc;
    const float *old_r;          // solve path: previous iterate for the partial norms, or null
    double *norm_part;
    // solve path, running-average rule (see AdjArgs; null hist: off)
    double *avg;
    float *hist;
    int hist_put, hist_drop;
    double inv_m, inv_m_prev;
    void *ws;
    DevState *state;             // solve path: done flag and status, or null
    double *lam_io;              // solve path: lam carried between calls, or null (tail)
    double tau, tol_tv, tol_dykstra;
    int fgp_iters, max_bisect, max_dykstra;
    float lo, hi;
    int fixed_lam;               // proximal mode: argmin ||x - z||^2 + lam TV(x), lam from lam_io
};
size_t tv_workspace_bytes(int nx, int ny, int grid);
int tv_grid(long long d);
TvTail *tv_tail(void *ws, int nx, int ny, int grid);
cudaError_t launch_tv_project(const TvLaunch &L, cudaStream_t s);

// FP64 stopping reduction of iteration `iter` (the stopping test comes from
// the state).  The _cond form runs inside a CUDA graph's WHILE loop: the
// iteration is state->iters_done and it sets the loop condition `cond` to
// "not stopped and state->iters_done < state->iter_end".
cudaError_t launch_solve_reduce(const double *partials, int nparts, DevState *st, int iter, cudaStream_t s);
cudaError_t launch_solve_reduce_cond(const double *partials, int nparts, DevState *st,
                                     cudaGraphConditionalHandle cond, cudaStream_t s);
// Start of a solve call: iterations t0 .. t_end - 1 (0-based), stopping test
// (tol, check_every, rule), tail average from iteration avg_from.
cudaError_t launch_reset_state(DevState *st, int t0, int t_end, double tol, int check_every, int rule, int avg_from,
                               cudaStream_t s);

// FP64 power iteration pieces
cudaError_t launch_power_init(double *xrd, double *xcd, int nx, int ny, long long ldr, long long ldc,
                              DevState *st, cudaStream_t s);
cudaError_t launch_forward_d(const RayD *rays, long long n, const double *xrd, const double *xcd, int nx,
                             int ny, long long ldr, long long ldc, double *zd, double *partials,
                             DevState *st, cudaStream_t s);
int forward_d_blocks(long long n);
cudaError_t launch_adjoint_d(const RayD *rays, const ViewRec *views, int n_views, int n_bins, int nx, int ny,
                             const double *zd, double *xrd, double *xcd, long long ldr, long long ldc,
                             double *partials, DevState *st, bool fan, cudaStream_t s);
// Persistent multi-job kernel: jobs[n_jobs] in device memory, prefix[5 n_jobs + 1]
// = items of the (phase, job) segments before each segment within a round
// (phase-major), rounds = largest iteration count.  next/done_items/abort are
// zeroed by the caller.
cudaError_t launch_batch(const BatchJob *jobs, int n_jobs, const int *prefix, int rounds, unsigned long long *next,
                         unsigned *done_items, int *abort_flag, int grid, long long dep_polls, cudaStream_t s);
int batch_grid_size();

cudaError_t launch_power_reduce(const double *pz, int nz, const double *pw, int nw, DevState *st, int iter,
                                double rtol, cudaStream_t s);

}  // namespace exact
