// joseph.cuh -- device bodies of the Joseph projector work items, shared by
// the per-plan kernels (k_forward.cu, k_adjoint.cu) and the persistent
// multi-job kernel (k_batch.cu).
//
//   forward_unit: Joseph forward walk of one work unit (up to kFR adjacent rays
//     of one view), image bands staged in shared memory by 2D tensor-map
//     copies, optional link/residual epilogue (Eq. (7), Eq. (8));
//   adjoint_tile: deterministic gather of A^T r over one kTW x kTH pixel tile
//     (strip walk), with the extragradient epilogue of Eq. (11) and the FP64
//     partial norms of the stopping rule.
//
// COHERENT selects loads that bypass the non-coherent L1 paths for data that
// other CTAs rewrite during the same launch (the persistent kernel).
#pragma once

#include "exact_internal.h"

namespace exact {

// ------------------------------------------------------------------ helpers

constexpr unsigned kBoxBytes = kFC * kFHB * sizeof(float);
constexpr int kWaitSpins = 1 << 20;  // bounded mbarrier wait (try_wait also suspends briefly)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for the given phase parity; true when the phase completed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t addr = smem_u32(bar);
    for (int it = 0; it < kWaitSpins; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// One kFC x kFHB box of the tensor map at (x = padded cross index, y = line).
__device__ __forceinline__ void tma_box(float *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    const uint32_t b = smem_u32(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(kBoxBytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(b)
        : "memory");
}

// Hardware base-2 exponential (MUFU ex2, a few ulp): the link's 2^(-mu z).
// Results below the smallest normal float flush to zero; they weigh less than
// 1e-30 counts against I0 >= 1.
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <bool COHERENT, typename T>
__device__ __forceinline__ T ld_dyn(const T *p)
{
    return COHERENT ? __ldcg(p) : __ldg(p);
}

// Shared memory of one forward item (the two staging buffers); the two
// mbarriers and the broadcast flag live outside so that a persistent kernel can
// reuse this space for other items.
struct FwdSmem {
    float buf[kFStages][kFC * kFHB];
};

// ------------------------------------------------------------------ forward

// Joseph forward walk of work unit `ui` (see k_forward.cu for the design).
// Thread 0 issues the copies, kFStages - 1 chunks ahead; every thread waits on
// the chunk's mbarrier and keeps in bit b of `phase` the parity of the
// completed phases of barrier b across calls (all 0 after mbar_init).  One
// CTA barrier per chunk.  Returns false (uniformly) if a staging copy timed
// out; the caller must then stop using the shared buffers.  The buffers may
// still be read by other threads when it returns: the caller synchronises the
// CTA before the next unit.
template <bool LINK, bool COHERENT>
__device__ __forceinline__ bool forward_unit(const FwdArgs &a, int ui, const CUtensorMap *map_r,
                                             const CUtensorMap *map_c, const LinkCoef *coef, FwdSmem &sm,
                                             uint64_t *bar, uint32_t &phase)
{
    const FwdUnit u = a.units[ui];
    const int t = threadIdx.x;
    const bool has_ray = t < u.count;
    const long long i = (long long)u.ray0 + t;
    RayF rec = {0.f, 0.f, 0.f, 0.f};
    int bits = 1;  // empty driving range (j_lo = 1 > j_hi = 0)
    if (has_ray) {
        rec = a.rays[i];
        bits = a.bits[i];
    }
    const int jlo = ray_jlo(bits), jhi = ray_jhi(bits);
    // chunks the ray samples: cfirst .. cfirst + cspan (an empty range gets a
    // first chunk no unit reaches, so the unsigned test below always fails)
    const int cfirst = jlo <= jhi ? jlo / kFC : 0x3fffffff;
    const int cspan = jlo <= jhi ? jhi / kFC - jlo / kFC : 0;
    const CUtensorMap *map = u.axis ? map_r : map_c;
    const int A = (int)rec.A;
    const int *kst = a.kstart + u.koff;

    if (t == 0 && u.nchunks > 0) {
        // order earlier generic accesses of the buffers (and of global data
        // synchronised with other CTAs) before the async-proxy copies
        asm volatile("fence.proxy.async;" ::: "memory");
        for (int c = 0; c < kFStages - 1 && c < u.nchunks; ++c)
            tma_box(sm.buf[c], map, kst[c] + kPad, (u.jc0 + c) * kFC, &bar[c]);
    }
    float acc = 0.0f;
    // band start of chunk c, loaded one chunk ahead
    int ks_next = u.nchunks > 0 ? ld_dyn<COHERENT>(kst) : 0;
    // The per-plan kernel unrolls the chunk loop by two, so that the stage
    // b = c % 2 of each copy (and its mbarrier parity bit) folds to a constant
    // (120.5 -> 115.7 us per launch); the persistent kernel keeps one copy of
    // the chunk's code in its large body (two copies cost its multi-job batch
    // 129 -> 110 recon/s).
    static_assert(kFStages == 2, "the stage of chunk c is c % 2");
#pragma unroll(COHERENT ? 1 : 2)
    for (int c = 0; c < u.nchunks; ++c) {
        const int b = c & 1;  // stage of chunk c
        const int ks = ks_next;
        if (c + 1 < u.nchunks) ks_next = ld_dyn<COHERENT>(kst + c + 1);
        // every thread waits for chunk c; the barrier then also tells that all
        // threads are done with chunk c - 1, whose buffer the next copy reuses
        bool ok = mbar_wait(&bar[b], (phase >> b) & 1u);
        ok = __syncthreads_and(ok) != 0;
        if (!ok) {
            // a copy did not complete in time everywhere: report, wait
            // (bounded) for every copy in flight so none lands after the
            // buffers are released
            if (t == 0) {
                for (int q = c; q < u.nchunks && q < c + kFStages - 1; ++q) {
                    const int bq = q % kFStages;
                    mbar_wait(&bar[bq], (phase >> bq) & 1u);
                }
                if (a.err) {
                    a.err->status = EXACT_ERR_TIMEOUT;
                    a.err->done = 1;
                }
            }
            return false;
        }
        phase ^= 1u << b;
        const int cn = c + kFStages - 1;
        if (t == 0 && cn < u.nchunks) {
            // that buffer was last read in chunk c - 1 (before the barrier
            // above); order those reads before the async-proxy write
            const int bn = cn % kFStages;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_box(sm.buf[bn], map, kst[cn] + kPad, (u.jc0 + cn) * kFC, &bar[bn]);
        }
        const int j0 = (u.jc0 + c) * kFC;
        // the ray samples this chunk (an empty range, j_lo > j_hi, never does)
        if ((unsigned)(u.jc0 + c - cfirst) <= (unsigned)cspan) {
            // anchor: t(j0) = K + tau0 with tau0 accurate to FP32 rounding at ~1
            const float jf = (float)j0;
            const float p = rec.bh * jf;
            const float e = fmaf(rec.bh, jf, -p);
            const float P = floorf(p);
            const float tau0 = ((p - P) + rec.a) + fmaf(rec.bl, jf, e);
            // local row = K + floor(tau) - kstart, with the bias of the
            // float-to-int floor folded in
            const int off = A + (int)P - ks - kFloorBias;
            // The walk covers all kFC lines of the chunk, not only the ray's
            // driving range [jlo, jhi]: outside it the crossing lies beyond the
            // image by more than a pixel, so both taps read the zero pads or
            // the copy's zero fill and add exactly +0.  The host sized the band
            // for the whole chunk; the row is monotone in the line (t is
            // linear, the round-down floor monotone), so checking the first and
            // last line keeps every read inside the buffer.  A band that fails
            // the check (a damaged table) poisons the projection with NaN.
            const float tl = fmaf(rec.bh, (float)(kFC - 1), tau0);
            const int rf = off + __float_as_int(__fadd_rd(tau0, kFloorMagic));
            const int rl = off + __float_as_int(__fadd_rd(tl, kFloorMagic));
            // (a crossing that is NaN, infinite or below -2^23 gives a row far
            // outside the band, so the two row tests also cover those)
            const bool inside = (unsigned)rf <= (unsigned)(kFHB - 2) && (unsigned)rl <= (unsigned)(kFHB - 2);
            if (inside) {
                const float *sb = sm.buf[b] + off;  // + bits(r) lands in the buffer
#pragma unroll
                for (int k = 0; k < kFC; ++k) {
                    const float tau = fmaf(rec.bh, (float)k, tau0);
                    // floor(tau) for |tau| < 2^22: a round-down add of 1.5 * 2^23
                    // leaves floor(tau) in the low mantissa bits
                    const float r = __fadd_rd(tau, kFloorMagic);
                    const float f = tau - (r - kFloorMagic);
                    const float *q = sb + __float_as_int(r) + k * kFHB;
                    const float a0 = q[0], a1 = q[1];
                    acc += fmaf(f, a1 - a0, a0);
                }
            } else {
                acc = __int_as_float(0x7fc00000);
            }
        }
    }
    // the caller synchronises the CTA before the buffers are used again
    if (!has_ray) return true;
    const float delta = a.delta[i];
    const float z = delta * acc;
    if (!LINK) {
        a.z[i] = z;
        return true;
    }
    const float zp = fmaxf(z, 0.0f);
    float lam = 0.0f;
    if (a.M == 0) {
        for (int k = 0; k < a.K; ++k) lam = fmaf(coef->c[k], ex2_approx(-coef->mu2[k] * zp), lam);
    } else {
        // known background (Appendix A.1): extra attenuation sum_m mu_bg[m][k] p_m
        float pm[kMaxBg];
#pragma unroll
        for (int m = 0; m < kMaxBg; ++m) pm[m] = m < a.M ? a.bg[(long long)m * a.n + i] : 0.0f;
        for (int k = 0; k < a.K; ++k) {
            float e = coef->mu2[k] * zp;
#pragma unroll
            for (int m = 0; m < kMaxBg; ++m) e = fmaf(coef->mub[m][k], pm[m], e);
            lam = fmaf(coef->c[k], ex2_approx(-e), lam);
        }
    }
    a.r[i] = delta * (a.Y[i] - lam);
    return true;
}

// ------------------------------------------------------------------ adjoint

// Tile kTW x kTH (exact_internal.h).  A warp walks one view at a time: lane l
// owns tile column tx0 + l for the x-driven rays and tile row ty0 + l for the
// y-driven rays, so every strip is kTH = kTW pixels long.  The x-driven parts
// of all views are gathered first, then the y-driven parts, through the same
// per-warp accumulator (rows: strip offsets -1 .. kTH; bank = lane).
//
// Fan beams in the per-plan kernel walk line pairs instead: lane l owns the
// driving lines 2 (l % 16) and 2 (l % 16) + 1 over half h = l / 16 of the cross
// axis (kHalf pixels), so one step along a ray (residual load, reciprocal,
// loop) serves two crossings.  Each half has its own accumulator of kRowsH
// rows (strip offsets -1 .. kHalf) by 32 words; lane l keeps its two lines in
// words (2 (l % 16) + d + h) mod 32, d = 0, 1, so that the 32 lanes of a
// deposit touch 32 different banks.  As at tile edges, a crossing between the
// halves is walked by both, each keeping only its own pixels' weights.
static_assert(kTW == 32 && kTH == 32, "a warp covers one tile side");
constexpr int kRows = kTH + 2;  // accumulator rows: strip offsets -1 .. kTH
constexpr int kAccLd = 32;      // accumulator row stride: word (row, lane)
constexpr int kHalf = kTH / 2;                  // line pairs: strip length
constexpr int kRowsH = kHalf + 2;               // line pairs: rows per half (strip offsets -1 .. kHalf)
constexpr int kHalfWords = kRowsH * kAccLd;     // line pairs: words per half
constexpr int kAccWords = 2 * kHalfWords > kRows * kAccLd ? 2 * kHalfWords : kRows * kAccLd;
constexpr float kBinEps = 0.01f;

template <int G>
struct AdjSmem {
    union {
        float acc[G][kAccWords];       // per warp: its lanes' strips in the current phase
        float tile[kTH][kTW + 1];      // epilogue (the accumulators are dead by then)
    };
    float stage[kTH][kTW + 1];
    double red0[G], red1[G], red2[G];
};

// Hardware reciprocal (MUFU, about 1 ulp); its arguments here are well inside
// the normal range: 1 + sg e (|sg e| < 1/2) and the positive fan-beam depths.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Bin range of the rays that cross the segment between two points whose
// detector projections are (num1/den1, num2/den2) + c, within [lo_bin, hi_bin).
template <bool FAN>
__device__ __forceinline__ void seg_range(float num1, float den1, float num2, float den2, float c, int lo_bin,
                                          int hi_bin, int &b0, int &b1)
{
    const float u1 = FAN ? num1 * rcp_approx(den1) : num1;
    const float u2 = FAN ? num2 * rcp_approx(den2) : num2;
    float lo = fminf(u1, u2) + c - kBinEps;
    float hi = fmaxf(u1, u2) + c + kBinEps;
    lo = fminf(fmaxf(lo, -1.0f), (float)hi_bin);
    hi = fminf(fmaxf(hi, -1.0f), (float)hi_bin);
    b0 = max(lo_bin, (int)ceilf(lo));
    b1 = min(hi_bin - 1, (int)floorf(hi));
}

// Walk rays b0..b1 of one view at driving index jf; deposit into the lane's
// pair slot k + 1 (strip offset k = floor(t - kbase) in [-1, kTH - 1]).  The
// crossing of the middle ray bc is computed from its split record; the others
// follow from the walk coefficients (RayW) as
//   t_{bc+e} = t_bc + (kappa e) / (1 + sg e),
// so a step reads only its residual (and, in a fan, takes one hardware
// reciprocal).  |e| <= 1/2 of the walk keeps the FP32 error of t within a few
// 1e-6 pixel (rms about 1e-6).  al points at the lane's row 0.
template <bool FAN, bool DELTA, bool COHERENT>
__device__ __forceinline__ void strip_walk(const RayF *__restrict__ vrays, const RayW *__restrict__ vwalk,
                                           const float *__restrict__ vres, const float *__restrict__ vdelta,
                                           int b0, int b1, float jf, float kbase, float *__restrict__ al)
{
    if (b0 > b1) return;
    const int bc = (b0 + b1) >> 1;
    const float4 q = __ldg(reinterpret_cast<const float4 *>(vrays + bc));
    const float4 w = __ldg(reinterpret_cast<const float4 *>(vwalk + bc));
    const float p = q.z * jf;
    const float pe = fmaf(q.z, jf, -p);
    const float tc = ((q.x - kbase) + p) + (q.y + fmaf(q.w, jf, pe));
    const float kap = fmaf(w.y, jf, w.x);
    float e = (float)(b0 - bc);
    const float *pr = vres + b0;
    const float *pd = DELTA ? vdelta + b0 : nullptr;
#pragma unroll 2
    for (int n = b1 - b0; n >= 0; --n, e += 1.0f, ++pr) {
        float rv = ld_dyn<COHERENT>(pr);
        if (DELTA) rv *= __ldg(pd++);
        const float u = FAN ? fmaf(kap * e, rcp_approx(fmaf(w.z, e, 1.0f)), tc) : fmaf(kap, e, tc);
        // floor(u) without the conversion pipe (|u| < 2^22)
        const float r = __fadd_rd(u, kFloorMagic);
        const float f = u - (r - kFloorMagic);
        // row k + 1 for the strip offset k = floor(u), with the float-to-int bias folded in
        const unsigned k1 = (unsigned)(__float_as_int(r) - (kFloorBias - 1));
        if (k1 <= (unsigned)kTH) {
            float *p = al + k1 * kAccLd;
            p[0] = fmaf(1.0f - f, rv, p[0]);
            p[kAccLd] = fmaf(f, rv, p[kAccLd]);
        }
    }
}

// Bin range of the rays that cross either of two adjacent lines between cross
// coordinates f_lo and f_hi: the hull of the detector projections
// (num/den + c) of the four corners, within [lo_bin, hi_bin).
template <bool FAN>
__device__ __forceinline__ void seg_range2(float n00, float d00, float n01, float d01, float n10, float d10,
                                           float n11, float d11, float c, int lo_bin, int hi_bin, int &b0, int &b1)
{
    const float u00 = FAN ? n00 * rcp_approx(d00) : n00, u01 = FAN ? n01 * rcp_approx(d01) : n01;
    const float u10 = FAN ? n10 * rcp_approx(d10) : n10, u11 = FAN ? n11 * rcp_approx(d11) : n11;
    float lo = fminf(fminf(u00, u01), fminf(u10, u11)) + c - kBinEps;
    float hi = fmaxf(fmaxf(u00, u01), fmaxf(u10, u11)) + c + kBinEps;
    lo = fminf(fmaxf(lo, -1.0f), (float)hi_bin);
    hi = fminf(fmaxf(hi, -1.0f), (float)hi_bin);
    b0 = max(lo_bin, (int)ceilf(lo));
    b1 = min(hi_bin - 1, (int)floorf(hi));
}

// One crossing of a half strip: t relative to the strip's first pixel, strip
// offset k = floor(t) in [-1, kHalf - 1] deposited into rows k + 1 and k + 2
// (al points at row 0); other crossings belong to other strips.
__device__ __forceinline__ void deposit_half(float *__restrict__ al, float t, float rv)
{
    const float r = __fadd_rd(t, kFloorMagic);
    const float f = t - (r - kFloorMagic);
    const unsigned k1 = (unsigned)(__float_as_int(r) - (kFloorBias - 1));
    if (k1 <= (unsigned)kHalf) {
        float *p = al + k1 * kAccLd;
        p[0] = fmaf(1.0f - f, rv, p[0]);
        p[kAccLd] = fmaf(f, rv, p[kAccLd]);
    }
}

// Line-pair walk (fan beam): rays b0..b1 of one view across driving lines jf
// and jf + 1, into the lane's two half strips (al0: line jf, al1: line jf + 1).
// The crossings of the middle ray bc come from its split record, the others
// from t_{bc+e} = t_bc + kappa (e / (1 + sg e)), where only t_bc and kappa
// depend on the line: one step reads one residual and takes one reciprocal
// for both crossings.
template <bool DELTA, bool COHERENT>
__device__ __forceinline__ void strip_walk2(const RayF *__restrict__ vrays, const RayW *__restrict__ vwalk,
                                            const float *__restrict__ vres, const float *__restrict__ vdelta,
                                            int b0, int b1, float jf, float kbase, float *__restrict__ al0,
                                            float *__restrict__ al1)
{
    if (b0 > b1) return;
    const int bc = (b0 + b1) >> 1;
    const float4 q = __ldg(reinterpret_cast<const float4 *>(vrays + bc));
    const float4 w = __ldg(reinterpret_cast<const float4 *>(vwalk + bc));
    const float jg = jf + 1.0f;
    const float p0 = q.z * jf, p1 = q.z * jg;
    const float pe0 = fmaf(q.z, jf, -p0), pe1 = fmaf(q.z, jg, -p1);
    const float tc0 = ((q.x - kbase) + p0) + (q.y + fmaf(q.w, jf, pe0));
    const float tc1 = ((q.x - kbase) + p1) + (q.y + fmaf(q.w, jg, pe1));
    const float kap0 = fmaf(w.y, jf, w.x), kap1 = fmaf(w.y, jg, w.x);
    float e = (float)(b0 - bc);
    const float *pr = vres + b0;
    const float *pd = DELTA ? vdelta + b0 : nullptr;
#pragma unroll 2
    for (int n = b1 - b0; n >= 0; --n, e += 1.0f, ++pr) {
        float rv = ld_dyn<COHERENT>(pr);
        if (DELTA) rv *= __ldg(pd++);
        const float qe = e * rcp_approx(fmaf(w.z, e, 1.0f));
        deposit_half(al0, fmaf(kap0, qe, tc0), rv);
        deposit_half(al1, fmaf(kap1, qe, tc1), rv);
    }
}

// A^T r over tile (bx, by) with the epilogue of MODE (see k_adjoint.cu).
// blk is the tile's index (partial norms, split bookkeeping).  Phase 0: warp g
// of split z walks the x-driven parts of the views a.vitems[it] for
// it = z G + g + k G nsplit < nxv (lane l: column tx0 + l); phase 1 the
// y-driven parts of a.vitems[nxv + it], it < nyv (lane l: row ty0 + l).  After
// each phase the warps' accumulators are added into sm.stage in a fixed
// order.  With nsplit > 1 each CTA leaves its partial tile in a.split_part;
// the last of the tile's CTAs to finish (counted in a.split_count, which it
// resets) adds the partials in split order and runs the epilogue, so the sum
// is the same on every run.
template <int MODE, bool FAN, bool DELTA, int G, bool COHERENT>
__device__ __forceinline__ void adjoint_tile(const AdjArgs &a, int bx, int by, long long blk, AdjSmem<G> &sm,
                                             int z = 0)
{
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int tx0 = bx * kTW, ty0 = by * kTH;
    const int nsplit = a.nsplit > 1 ? a.nsplit : 1;
    // line pairs for fan beams in the per-plan kernel (see kHalf); the
    // persistent kernel keeps one walk for all its jobs
    constexpr bool PAIR = FAN && !COHERENT;
    for (int phase = 0; phase < 2; ++phase) {
        const bool xd = phase == 0;  // uniform: x-driven rays, else y-driven
        const int nline = xd ? a.nx : a.ny, ncross = xd ? a.ny : a.nx;
        const int *items = a.vitems + (xd ? 0 : a.nxv);
        if constexpr (!PAIR) {
            float *al = sm.acc[g] + lane;
            for (int r = 0; r < kRows; ++r) al[r * kAccLd] = 0.0f;
            // the lane's strip: x-driven rays, column tx0 + lane over rows ty0
            // .. ty0 + kTH - 1; y-driven rays, row ty0 + lane over columns tx0
            // .. tx0 + kTW - 1.  Its end points are kept within one pixel of
            // the image so that their fan-beam projections stay well defined
            // (the source is outside the image).
            const int line = (xd ? tx0 : ty0) + lane;
            const int sb = xd ? ty0 : tx0;
            const float fl = (float)line, f_lo = (float)(sb - 1), f_hi = (float)min(sb + kTH, ncross);
            const int nitems = line < nline ? (xd ? a.nxv : a.nyv) : 0;
            for (int it = z * G + g; it < nitems; it += G * nsplit) {
                const int v = __ldg(items + it);
                const ViewRec vr = a.views[v];
                const long long vb = (long long)v * a.n_bins;
                // detector projections of the strip's end points
                const float nb = xd ? fmaf(vr.n1, fl, vr.n0) : fmaf(vr.n2, fl, vr.n0);
                const float db = xd ? fmaf(vr.d1, fl, vr.d0) : fmaf(vr.d2, fl, vr.d0);
                const float na = xd ? vr.n2 : vr.n1, da = xd ? vr.d2 : vr.d1;
                int b0, b1;
                seg_range<FAN>(fmaf(na, f_lo, nb), fmaf(da, f_lo, db), fmaf(na, f_hi, nb), fmaf(da, f_hi, db), vr.c,
                               xd ? vr.xb0 : vr.yb0, xd ? vr.xb1 : vr.yb1, b0, b1);
                strip_walk<FAN, DELTA, COHERENT>(a.rays + vb, a.walk + vb, a.r + vb, DELTA ? a.delta + vb : nullptr,
                                                 b0, b1, fl, (float)sb, al);
            }
            __syncthreads();
            // fixed-order sum over the warps; pixel j of a lane's strip is its
            // accumulator row j + 1.  The y-driven parts are read transposed
            // (tile row = lane) so that consecutive threads read consecutive
            // banks.
            for (int t = threadIdx.x; t < kTH * kTW; t += G * 32) {
                const int i = t % kTW, k = t / kTW;
                float s = 0.0f;
                for (int q = 0; q < G; ++q) s += sm.acc[q][(k + 1) * kAccLd + i];
                if (xd)
                    sm.stage[k][i] = s;   // column i, row k
                else
                    sm.stage[i][k] += s;  // row i, column k
            }
        } else {
            const int hf = lane >> 4, lp = lane & 15;  // cross-axis half, line pair
            float *al0 = sm.acc[g] + hf * kHalfWords + ((2 * lp + hf) & 31);
            float *al1 = sm.acc[g] + hf * kHalfWords + ((2 * lp + 1 + hf) & 31);
            for (int r = 0; r < kRowsH; ++r) {
                al0[r * kAccLd] = 0.0f;
                al1[r * kAccLd] = 0.0f;
            }
            // the lane's strips: lines `line` and line + 1 over cross pixels
            // sb .. sb + kHalf - 1, end points within one pixel of the image
            const int line = (xd ? tx0 : ty0) + 2 * lp;
            const int sb = (xd ? ty0 : tx0) + hf * kHalf;
            const float fl = (float)line, f_lo = (float)(sb - 1), f_hi = (float)min(sb + kHalf, ncross);
            const int nitems = (line < nline && sb < ncross) ? (xd ? a.nxv : a.nyv) : 0;
            for (int it = z * G + g; it < nitems; it += G * nsplit) {
                const int v = __ldg(items + it);
                const ViewRec vr = a.views[v];
                const long long vb = (long long)v * a.n_bins;
                // detector projections of the four corners of the lane's strips
                const float nl = xd ? vr.n1 : vr.n2, dl = xd ? vr.d1 : vr.d2;
                const float na = xd ? vr.n2 : vr.n1, da = xd ? vr.d2 : vr.d1;
                const float nb0 = fmaf(nl, fl, vr.n0), db0 = fmaf(dl, fl, vr.d0);
                const float nb1 = fmaf(nl, fl + 1.0f, vr.n0), db1 = fmaf(dl, fl + 1.0f, vr.d0);
                int b0, b1;
                seg_range2<FAN>(fmaf(na, f_lo, nb0), fmaf(da, f_lo, db0), fmaf(na, f_hi, nb0), fmaf(da, f_hi, db0),
                                fmaf(na, f_lo, nb1), fmaf(da, f_lo, db1), fmaf(na, f_hi, nb1), fmaf(da, f_hi, db1),
                                vr.c, xd ? vr.xb0 : vr.yb0, xd ? vr.xb1 : vr.yb1, b0, b1);
                strip_walk2<DELTA, COHERENT>(a.rays + vb, a.walk + vb, a.r + vb, DELTA ? a.delta + vb : nullptr, b0,
                                             b1, fl, (float)sb, al0, al1);
            }
            __syncthreads();
            // fixed-order sum over the warps: line i, cross pixel k of the
            // tile is half h = k / kHalf, row k - h kHalf + 1, word (i + h)
            // mod 32; the y-driven parts are written transposed
            for (int t = threadIdx.x; t < kTH * kTW; t += G * 32) {
                const int i = t % kTW, k = t / kTW, h = k / kHalf;
                const int w = h * kHalfWords + (k - h * kHalf + 1) * kAccLd + ((i + h) & 31);
                float s = 0.0f;
                for (int q = 0; q < G; ++q) s += sm.acc[q][w];
                if (xd)
                    sm.stage[k][i] = s;
                else
                    sm.stage[i][k] += s;
            }
        }
        __syncthreads();
    }
    if (nsplit > 1) {
        float *mine = a.split_part + ((long long)blk * nsplit + z) * (kTH * kTW);
        for (int t = threadIdx.x; t < kTH * kTW; t += G * 32) mine[t] = sm.stage[t / kTW][t % kTW];
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            s_last = atomicAdd(a.split_count + blk, 1) == nsplit - 1;
            if (s_last) atomicExch(a.split_count + blk, 0);
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        const float *all = a.split_part + (long long)blk * nsplit * (kTH * kTW);
        for (int t = threadIdx.x; t < kTH * kTW; t += G * 32) {
            float v = 0.0f;
            for (int q = 0; q < nsplit; ++q) v += __ldcg(all + (long long)q * (kTH * kTW) + t);
            sm.stage[t / kTW][t % kTW] = v;
        }
        __syncthreads();
    }
    // partial norms of the stopping rule: each thread sums its few pixels
    // (at most kTH kTW / (32 G) + 1) in FP32, then the warp and tile sums are
    // FP64 (FP64 arithmetic per pixel costs ~6 us per launch on this part; the
    // FP32 stage adds a relative error of ~3e-7 to the norms)
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    float s0f = 0.0f, s1f = 0.0f;
    // iteration index and running-average slots of this launch (from the
    // device state inside a CUDA graph loop, the same values the host passes
    // otherwise)
    int it_idx = a.iter, avg_from = a.avg_from, hist_put = a.hist_put, hist_drop = a.hist_drop;
    double inv_m = a.inv_m, inv_m_prev = a.inv_m_prev;
    if (MODE == ADJ_EG_FINAL && a.iter_from_state) {
        it_idx = a.state->iters_done;
        avg_from = a.state->avg_from;
        if (a.hist) {
            // iterate number it enters the window of the last m = max(1, floor(it/2));
            // when m did not grow, x_{it-m} leaves it
            const int it = it_idx + 1, m = max(1, it / 2), mp = max(1, (it - 1) / 2);
            hist_put = it % a.hist_cap;
            hist_drop = (it >= 2 && m == mp) ? (it - m) % a.hist_cap : -1;
            inv_m = 1.0 / (double)m;
            inv_m_prev = it >= 2 ? 1.0 / (double)mp : 0.0;
        }
    }
    for (int t = threadIdx.x; t < kTH * kTW; t += G * 32) {
        const int px = t % kTW, py = t / kTW;
        const float gsum = sm.stage[py][px];
        const int kx = tx0 + px, ky = ty0 + py;
        const bool inside = kx < a.nx && ky < a.ny;
        if (MODE == ADJ_PLAIN) {
            if (inside) a.out[(long long)ky * a.nx + kx] = a.scale * gsum;
        } else if (MODE == ADJ_STEP) {
            if (inside)
                a.out[(long long)ky * a.nx + kx] =
                    fmaf(a.scale, gsum, ld_dyn<COHERENT>(a.base_r + (long long)ky * a.ldr + kx + kPad));
        } else {
            const long long pr = (long long)ky * a.ldr + kx + kPad;
            const float xb = inside ? ld_dyn<COHERENT>(a.base_r + pr) : 0.0f;
            // projection onto [lo, hi] that keeps a NaN (so the stopping rule sees it)
            const float step = fmaf(a.scale, gsum, xb);
            const float xn = inside ? (step < a.lo ? a.lo : (step > a.hi ? a.hi : step)) : 0.0f;
            if (inside) a.out_r[pr] = xn;
            sm.tile[py][px] = xn;
            if (MODE == ADJ_EG_FINAL && inside) {
                const long long q = (long long)ky * a.nx + kx;
                if (a.hist) {
                    // running average of Sec. 3.1: window sum in FP64 (exact
                    // for FP32 summands), ring of the window's iterates
                    const long long dpix = (long long)a.nx * a.ny;
                    const double sp = a.avg[q];
                    double sn = sp + (double)xn;
                    if (hist_drop >= 0) sn -= (double)a.hist[(long long)hist_drop * dpix + q];
                    a.hist[(long long)hist_put * dpix + q] = xn;
                    a.avg[q] = sn;
                    const double dv = sn * inv_m - sp * inv_m_prev;
                    s2 += dv * dv;
                } else if (a.avg && it_idx >= avg_from) {
                    a.avg[q] += (double)xn;
                }
                const float dd = xn - xb;
                s0f = fmaf(dd, dd, s0f);
                s1f = fmaf(xb, xb, s1f);
            }
        }
    }
    s0 += (double)s0f;
    s1 += (double)s1f;
    if (MODE == ADJ_PLAIN || MODE == ADJ_STEP) return;
    __syncthreads();
    // column-major copy: kTH consecutive ky per kx row
    for (int t = threadIdx.x; t < kTH * kTW; t += G * 32) {
        const int col = t / kTH, row = t % kTH;
        const int ox = tx0 + col, oy = ty0 + row;
        if (ox < a.nx && oy < a.ny) a.out_c[(long long)ox * a.ldc + oy + kPad] = sm.tile[row][col];
    }
    if (MODE == ADJ_EG_FINAL) {
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_down_sync(0xffffffffu, s0, o);
            s1 += __shfl_down_sync(0xffffffffu, s1, o);
            s2 += __shfl_down_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            sm.red0[g] = s0;
            sm.red1[g] = s1;
            sm.red2[g] = s2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t0 = 0.0, t1 = 0.0, t2 = 0.0;
            for (int q = 0; q < G; ++q) {
                t0 += sm.red0[q];
                t1 += sm.red1[q];
                t2 += sm.red2[q];
            }
            a.partials[kPartStride * blk] = t0;
            a.partials[kPartStride * blk + 1] = t1;
            a.partials[kPartStride * blk + 2] = t2;
        }
    }
}

}  // namespace exact
