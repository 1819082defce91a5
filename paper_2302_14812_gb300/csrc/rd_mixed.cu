// Mixed-precision deposit: FP32 Lienard-Wiechert field (Eq. 1) and FP32 accumulation, with the
// arrival time (Eq. 2) kept FP64-accurate.
//
// Work item = (step chunk, block of 256 cells, particle); consecutive CTAs take consecutive
// particles of the same chunk and cell block, so the CTAs resident at one time all reduce into
// the same ~(256 cells x chunk span) slice of the detector, which stays in L2.
//
// Each thread walks two cells through the chunk as one pair: every per-cell quantity is a float2
// (cell A, cell B) and the field arithmetic runs as packed f32x2 add / mul / fma, one instruction
// for both cells; the per-sample constants arrive duplicated and sign-folded (RecM) so no packed
// operation needs a separate negation.  Per cell the walk carries the bin b it is filling and the
// time f already spent in that bin, in units of dt; a step adds the arrival-time increment
//     t'_k - t'_{k-1} = dt [dt g + R_k (g + |n_k - vbar|^2)] / (dt + R_k + R_{k-1})
// (vbar = (x_k - x_{k-1})/dt, g = 1 - |vbar|^2), an exact identity with only positive terms, so
// FP32 keeps its relative precision; the chunk's first and last arrival times are computed in
// FP64 directly from Eq. 2 (anchors), which bounds the drift to one chunk and makes adjacent
// chunks meet exactly.  The field held over the interval is added to the running bin with the
// part of the interval that lies in that bin (integrating deposit, Section 3.2); when the arrival
// time leaves the bin, the bin is added to global memory with two vector reductions.
#include <math.h>

#include <algorithm>

#include "rd_internal.cuh"

namespace rd {

namespace {

#ifndef RD_PIPELINE
#define RD_PIPELINE 0
#endif

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// Two-cell arithmetic: packed f32x2 instructions, or the same operations on each half.
#if RD_PACKED
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
#define RV(r, f) ((r).f)
#else
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c)
{
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
#define RV(r, f) f2((r).f)
#endif

// a*b - c*d per half (scalar form: the negation folds into the fused multiply-add)
__device__ __forceinline__ float2 vfms(float2 a, float2 b, float2 c, float2 d)
{
#if RD_PACKED
    return __ffma2_rn(a, b, __fmul2_rn(__fmul2_rn(c, f2(-1.f)), d));
#else
    return make_float2(fmaf(a.x, b.x, -(c.x * d.x)), fmaf(a.y, b.y, -(c.y * d.y)));
#endif
}

struct Pair {
    float2 Px, Py, Pz;   // cell positions
    float2 f;            // time spent in the current bin, units of dt (0 <= f < W)
    float2 Rpd;          // R_{k-1} + dt
    float2 acc[6];       // E xyz, B xyz of the current bin so far (weights in bins)
    int b[2];            // bin being filled (may lie outside [0, n_bins))
    float* row[2];       // [n_bins][8] accumulators of each cell
    bool live[2];        // some arrival of the chunk falls inside the window
    int below[2];        // intervals whose start lies before the window (clip tracking only)
    int above[2];        // intervals whose end lies after the window (clip tracking only)
};

struct Consts {
    float W;             // bin width / dt
    float invW;
    float2 Q;            // -(charge * dt / dt_det): weights in dt units -> bins, sign of E' folded in
    float2 DT;
    int n_bins;
};

// Packed field of one sample at both cells (E = S E', B = (S/R) d x E').
struct Sample {
    float2 E[3];         // E' = (n - beta)(-c1/kappa) + betadot
    float2 B[3];         // d x E'
    float2 S;            // -q' / (kappa^2 R)
    float2 rinv;         // 1 / R
    float2 du;           // t'_k - t'_{k-1} in units of dt
};

// Add one bin to global memory; bins outside the window are dropped.
__device__ __forceinline__ void flush(float* row, int n_bins, int b, float e0, float e1, float e2,
                                      float b0, float b1, float b2)
{
    if ((unsigned)b < (unsigned)n_bins) {
        float* p = row + (size_t)b * 8;
        red_add_v4(p, e0, e1, e2, b0);
        red_add_v2(p + 4, b1, b2);
    }
}

// Eq. 1 with B = n x E, for both cells:
//   E = q/(kappa^3 R) [ (n - beta)(gamma^-2/R + n.betadot) - betadot kappa ]
//     = S E',  E' = (n - beta)(-c1/kappa) + betadot,  c1 = gamma^-2/R + n.betadot,  S = -q/(kappa^2 R)
//   B = n x E = (S/R) d x E'
// and kappa = (gamma^-2 + |n - beta|^2)/2 avoids the cancellation in 1 - beta.n.
__device__ __forceinline__ void sample_field(Pair& c, const RecM& r, const Consts& C, Sample& o)
{
    const float2 one = f2(1.f), mhalf = f2(-0.5f);
    // geometry: d = x_cell - x_k, R = |d|
    const float2 dx = vadd(c.Px, RV(r, nx)), dy = vadd(c.Py, RV(r, ny)), dz = vadd(c.Pz, RV(r, nz));
    const float2 r2 = vfma(dx, dx, vfma(dy, dy, vmul(dz, dz)));
    float2 rinv;
    rinv.x = fast_rsqrt(r2.x);
    rinv.y = fast_rsqrt(r2.y);
    const float2 bx = vfma(dx, rinv, RV(r, nbx)), by = vfma(dy, rinv, RV(r, nby)),
                 bz = vfma(dz, rinv, RV(r, nbz));                       // n - beta
    const float2 nb2 = vfma(bx, bx, vfma(by, by, vmul(bz, bz)));
    // arrival-time increment in units of dt, numerator and denominator divided by R:
    //   [dt g / R + (g + |n - vbar|^2)] / [1 + (R_{k-1} + dt) / R],
    //   g + |n - vbar|^2 = |n - beta|^2 + 2 (n - beta).(beta - vbar) + (g + |beta - vbar|^2)
    const float2 gg = vfma(bx, RV(r, d2x), vfma(by, RV(r, d2y), vfma(bz, RV(r, d2z), vadd(nb2, RV(r, gd)))));
    const float2 num = vfma(RV(r, dtg), rinv, gg);
    const float2 den = vfma(c.Rpd, rinv, one);
    float2 rden;
    rden.x = fast_rcp(den.x);
    rden.y = fast_rcp(den.y);
    o.du = vmul(num, rden);
    c.Rpd = vfma(r2, rinv, C.DT);
    // Eq. 1
    const float2 kn = vfma(nb2, mhalf, RV(r, nhig2));                  // -kappa
    float2 ikn;
    ikn.x = fast_rcp(kn.x);
    ikn.y = fast_rcp(kn.y);                                            // -1/kappa
    const float2 nrik = vmul(rinv, ikn);                               // -1/(kappa R)
    o.S = vmul(vmul(C.Q, nrik), ikn);                                  // Q/(kappa^2 R) = -q'/(kappa^2 R)
    const float2 dbd = vfma(dx, RV(r, bdx), vfma(dy, RV(r, bdy), vmul(dz, RV(r, bdz))));
    const float2 c1n = vmul(vadd(RV(r, ig2n), dbd), nrik);            // -c1/kappa
    o.E[0] = vfma(bx, c1n, RV(r, bdx));
    o.E[1] = vfma(by, c1n, RV(r, bdy));
    o.E[2] = vfma(bz, c1n, RV(r, bdz));
    o.B[0] = vfms(dy, o.E[2], dz, o.E[1]);
    o.B[1] = vfms(dz, o.E[0], dx, o.E[2]);
    o.B[2] = vfms(dx, o.E[1], dy, o.E[0]);
    o.rinv = rinv;
}

// Interval of cell H (0 = .x, 1 = .y) that passes two or more bin edges (rare): flush the bin
// being filled and the whole bins inside the interval, leaving the state one edge short so that
// the common path below finishes the step (it flushes the last whole bin and starts the next).
template <int H, bool TRACK>
__device__ __forceinline__ void multi_edges(Pair& c, const Sample& o, const Consts& C, float2& fn, int k,
                                         int k_begin, int k_end)
{
    auto h = [](const float2& v) -> float { return H == 0 ? v.x : v.y; };
    auto set = [](float2& v, float x) {
        if (H == 0) v.x = x;
        else v.y = x;
    };
    const float f = h(fn);
    if (!(f >= 2.f * C.W)) return;
    const int b0 = c.b[H];
    const int m = (int)fminf(floorf(f * C.invW), 16777216.f);      // edges passed, >= 2
    flush(c.row[H], C.n_bins, b0, h(c.acc[0]), h(c.acc[1]), h(c.acc[2]), h(c.acc[3]), h(c.acc[4]),
          h(c.acc[5]));
    const float S = h(o.S), rinv = h(o.rinv);
    const float fs = C.W * S, fb = fs * rinv;
    // whole bins b0+1 .. b0+m-2 now; bin b0+m-1 is left in the accumulator for the common path
    const int lo = max(b0 + 1, 0), hi = min(b0 + m - 2, C.n_bins - 1);
    for (int j = lo; j <= hi; ++j)
        flush(c.row[H], C.n_bins, j, h(o.E[0]) * fs, h(o.E[1]) * fs, h(o.E[2]) * fs, h(o.B[0]) * fb,
              h(o.B[1]) * fb, h(o.B[2]) * fb);
    set(c.acc[0], h(o.E[0]) * fs);
    set(c.acc[1], h(o.E[1]) * fs);
    set(c.acc[2], h(o.E[2]) * fs);
    set(c.acc[3], h(o.B[0]) * fb);
    set(c.acc[4], h(o.B[1]) * fb);
    set(c.acc[5], h(o.B[2]) * fb);
    c.b[H] = b0 + m - 1;
    set(fn, fminf(fmaxf(fmaf(-(float)(m - 1), C.W, f), C.W), C.W * 1.99999988f));
    if (TRACK) {
        if (b0 < 0 && b0 + m - 1 >= 0) c.below[H] = k - k_begin + 1;
        if (b0 < C.n_bins && b0 + m - 1 >= C.n_bins) c.above[H] = k_end - k + 1;
    }
}

// Integrating deposit of one interval for both cells: the part of [f, f + du] inside the current
// bin goes to the running bin; a cell whose arrival time passes the bin edge flushes the bin and
// starts the next one with the rest of the interval.  Branch free apart from the rare case of an
// interval spanning several bins.  LAST: the interval ends on the exact FP64 anchors.
// TRACK: bins may lie outside the window (checked, clipped intervals counted).
template <bool LAST, bool TRACK>
__device__ __forceinline__ void deposit(Pair& c, const Sample& o, const Consts& C, const int* b_end,
                                        const float* f_end, int k, int k_begin, int k_end)
{
    float2 fn;
    if (LAST) {
        fn.x = fmaf((float)(b_end[0] - c.b[0]), C.W, f_end[0]);
        fn.y = fmaf((float)(b_end[1] - c.b[1]), C.W, f_end[1]);
    } else {
        fn = vadd(c.f, o.du);
    }
    float2 mn;
    mn.x = fminf(fn.x, C.W);
    mn.y = fminf(fn.y, C.W);
    const float2 ws = vmul(vfma(c.f, f2(-1.f), mn), o.S);
    const float2 wb = vmul(ws, o.rinv);
    c.acc[0] = vfma(o.E[0], ws, c.acc[0]);
    c.acc[1] = vfma(o.E[1], ws, c.acc[1]);
    c.acc[2] = vfma(o.E[2], ws, c.acc[2]);
    c.acc[3] = vfma(o.B[0], wb, c.acc[3]);
    c.acc[4] = vfma(o.B[1], wb, c.acc[4]);
    c.acc[5] = vfma(o.B[2], wb, c.acc[5]);
    if (__any_sync(0xffffffffu, fmaxf(fn.x, fn.y) >= 2.f * C.W)) {
        multi_edges<0, TRACK>(c, o, C, fn, k, k_begin, k_end);
        multi_edges<1, TRACK>(c, o, C, fn, k, k_begin, k_end);
    }
    const bool cx = fn.x >= C.W, cy = fn.y >= C.W;
    // flush the finished bins (predicated, per cell)
    const bool px = TRACK ? (cx && (unsigned)c.b[0] < (unsigned)C.n_bins) : cx;
    const bool py = TRACK ? (cy && (unsigned)c.b[1] < (unsigned)C.n_bins) : cy;
    float* ax = c.row[0] + (ptrdiff_t)c.b[0] * 8;
    float* ay = c.row[1] + (ptrdiff_t)c.b[1] * 8;
    red_add_v4_if(px, ax, c.acc[0].x, c.acc[1].x, c.acc[2].x, c.acc[3].x);
    red_add_v2_if(px, ax + 4, c.acc[4].x, c.acc[5].x);
    red_add_v4_if(py, ay, c.acc[0].y, c.acc[1].y, c.acc[2].y, c.acc[3].y);
    red_add_v2_if(py, ay + 4, c.acc[4].y, c.acc[5].y);
    // start the next bin with the rest of the interval
    const float2 rem = vadd(fn, f2(-C.W));
    const float2 rs = vmul(rem, o.S);
    const float2 rb = vmul(rs, o.rinv);
    const float2 t0 = vmul(o.E[0], rs), t1 = vmul(o.E[1], rs), t2 = vmul(o.E[2], rs);
    const float2 t3 = vmul(o.B[0], rb), t4 = vmul(o.B[1], rb), t5 = vmul(o.B[2], rb);
    c.acc[0] = make_float2(cx ? t0.x : c.acc[0].x, cy ? t0.y : c.acc[0].y);
    c.acc[1] = make_float2(cx ? t1.x : c.acc[1].x, cy ? t1.y : c.acc[1].y);
    c.acc[2] = make_float2(cx ? t2.x : c.acc[2].x, cy ? t2.y : c.acc[2].y);
    c.acc[3] = make_float2(cx ? t3.x : c.acc[3].x, cy ? t3.y : c.acc[3].y);
    c.acc[4] = make_float2(cx ? t4.x : c.acc[4].x, cy ? t4.y : c.acc[4].y);
    c.acc[5] = make_float2(cx ? t5.x : c.acc[5].x, cy ? t5.y : c.acc[5].y);
    c.f = make_float2(cx ? rem.x : fn.x, cy ? rem.y : fn.y);
    if (TRACK) {
        if (cx && c.b[0] == -1) c.below[0] = k - k_begin + 1;
        if (cx && c.b[0] == C.n_bins - 1) c.above[0] = k_end - k + 1;
        if (cy && c.b[1] == -1) c.below[1] = k - k_begin + 1;
        if (cy && c.b[1] == C.n_bins - 1) c.above[1] = k_end - k + 1;
    }
    c.b[0] += cx ? 1 : 0;
    c.b[1] += cy ? 1 : 0;
}

template <bool TRACK>
__device__ __forceinline__ void walk_tile(Pair& c, const RecM* tile, int cnt, bool last_tile,
                                          const Consts& C, const int* b_end, const float* f_end, int k0,
                                          int k_begin, int k_end)
{
    const int n_regular = last_tile ? cnt - 1 : cnt;
#if RD_PIPELINE
    // the field of sample i+1 is evaluated while sample i is deposited (independent work)
    if (n_regular > 0) {
        Sample cur;
        sample_field(c, tile[0], C, cur);
        for (int i = 0; i < n_regular; ++i) {
            Sample nxt;
            const bool more = i + 1 < cnt;
            if (more) sample_field(c, tile[i + 1], C, nxt);
            deposit<false, TRACK>(c, cur, C, b_end, f_end, k0 + i, k_begin, k_end);
            cur = nxt;
        }
        if (last_tile) deposit<true, TRACK>(c, cur, C, b_end, f_end, k_end, k_begin, k_end);
        return;
    }
#else
#pragma unroll 2
    for (int i = 0; i < n_regular; ++i) {
        Sample o;
        sample_field(c, tile[i], C, o);
        deposit<false, TRACK>(c, o, C, b_end, f_end, k0 + i, k_begin, k_end);
    }
#endif
    if (last_tile) {
        Sample o;
        sample_field(c, tile[cnt - 1], C, o);
        deposit<true, TRACK>(c, o, C, b_end, f_end, k_end, k_begin, k_end);
    }
}

}  // namespace

// One work item -- particle p, cell block cb, step chunk ch of one problem -- run by the whole
// CTA.  tile / bar: the CTA's shared staging buffers; g_base counts the tiles the CTA staged
// before this item (it selects buffer and mbarrier phase, so the buffers carry over between items).
// Returns false if a bounded wait ran out (the error is recorded; the CTA must stop).
__device__ __forceinline__ bool deposit_item(const DepositParams& P, int p, int cb, int ch,
                                             RecM (*tile)[kTileSteps], uint64_t* bar, unsigned& g_base)
{
    const int S = P.n_samples - 1;
    const int k_begin = 1 + ch * P.chunk;
    const int k_end = min(S, k_begin + P.chunk - 1);
    const int n_int = k_end - k_begin + 1;
    const int n_tiles = (n_int + kTileSteps - 1) / kTileSteps;
    const RecM* rec = static_cast<const RecM*>(P.rec) + (size_t)p * P.n_samples;
    const int tid = threadIdx.x;

    if (tid == 0) {
        fence_proxy_async();
        for (int t = 0; t < 2 && t < n_tiles; ++t) {
            const int k0 = k_begin + t * kTileSteps;
            const unsigned g = g_base + t;
            const unsigned bytes = (unsigned)min(kTileSteps, k_end - k0 + 1) * sizeof(RecM);
            mbar_arrive_expect_tx(&bar[g & 1], bytes);
            bulk_g2s(tile[g & 1], rec + k0, bytes, &bar[g & 1]);
        }
    }

    Consts C;
    C.W = P.W;
    C.invW = P.invW;
    C.Q = f2(-(P.q ? (float)P.q[p] : 1.f) * P.du_scale);
    C.DT = f2(P.dt_f);
    C.n_bins = P.n_bins;

    // anchors: exact FP64 arrival (bins) at both ends of the chunk, per cell
    Pair c;
    int b_end[2];
    float f_end[2];
    bool partial = false;
    unsigned long long clip = 0, crossed = 0;
    const double* xp = P.x + (size_t)p * P.n_samples * 3;
    float px[2], py[2], pz[2], fa[2], rpd[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int cell = cb * kMixedCellsPerCta + j * kMixedThreads + tid;
        // a cell without arrivals in the window still walks (no per-cell branch in the step) but
        // from a time that never reaches a bin edge: nothing is flushed
        c.live[j] = false;
        c.b[j] = -1073741824;
        c.row[j] = static_cast<float*>(P.fields);
        c.below[j] = c.above[j] = 0;
        fa[j] = -1e30f;
        rpd[j] = 1e6f;
        px[j] = 1e6f;
        py[j] = pz[j] = 0.f;
        b_end[j] = c.b[j];
        f_end[j] = 0.f;
        if (cell < P.n_pix) {
            const D4 cl = P.cells[cell];
            const double* xa = xp + 3 * (size_t)(k_begin - 1);
            const double* xe = xp + 3 * (size_t)k_end;
            double Ra, Re;
            const double ua = arrival_bins(xa[0], xa[1], xa[2], cl, P.t0, k_begin - 1, P.dt, P.inv_dt_det, Ra);
            const double ue = arrival_bins(xe[0], xe[1], xe[2], cl, P.t0, k_end, P.dt, P.inv_dt_det, Re);
            c.live[j] = (ue > 0.0) && (ua < (double)P.n_bins);
            if (!c.live[j]) {
                clip += (unsigned long long)n_int;
            } else {
                const double fla = floor(ua), fle = floor(ue);
                c.b[j] = clamp_bin(fla);
                fa[j] = (float)(ua - fla) * P.W;
                b_end[j] = clamp_bin(fle);
                f_end[j] = (float)(ue - fle) * P.W;
                rpd[j] = (float)Ra + P.dt_f;
                px[j] = (float)cl.x;
                py[j] = (float)cl.y;
                pz[j] = (float)cl.z;
                c.row[j] = static_cast<float*>(P.fields) + (size_t)cell * P.n_bins * 8;
                c.below[j] = (ua < 0.0) ? n_int : 0;
                // unchecked bins need a margin of one bin to each window edge (the FP32 walk may
                // drift by far less than a bin before the end anchor corrects it)
                partial = partial || (ua < 1.0) || (ue > (double)P.n_bins - 1.0);
                crossed += (unsigned long long)max(0, b_end[j] - c.b[j]);
            }
        }
    }
    c.Px = make_float2(px[0], px[1]);
    c.Py = make_float2(py[0], py[1]);
    c.Pz = make_float2(pz[0], pz[1]);
    c.f = make_float2(fa[0], fa[1]);
    c.Rpd = make_float2(rpd[0], rpd[1]);
#pragma unroll
    for (int i = 0; i < 6; ++i) c.acc[i] = f2(0.f);
    // clip tracking costs instructions in the bin-crossing path: only CTAs that need it use it
    const bool track = __syncthreads_or(partial) != 0;

    for (int t = 0; t < n_tiles; ++t) {
        const unsigned g = g_base + t;
        const int buf = g & 1;
        const bool ok = mbar_wait_bounded(&bar[buf], (g >> 1) & 1u);
        if (__syncthreads_or(!ok)) {
            // a bulk copy did not complete: record it, let outstanding copies land, stop.
            if (tid == 0) {
                atomicOr(&P.counters->errors, ERRBIT_TIMEOUT);
                for (int u = t; u < t + 2 && u < n_tiles; ++u)
                    (void)mbar_wait_bounded(&bar[(g_base + u) & 1], ((g_base + u) >> 1) & 1u);
            }
            __syncthreads();
            return false;
        }
        const int k0 = k_begin + t * kTileSteps;
        const int cnt = min(kTileSteps, k_end - k0 + 1);
        const bool last_tile = (t == n_tiles - 1);
        if (track)
            walk_tile<true>(c, tile[buf], cnt, last_tile, C, b_end, f_end, k0, k_begin, k_end);
        else
            walk_tile<false>(c, tile[buf], cnt, last_tile, C, b_end, f_end, k0, k_begin, k_end);
        __syncthreads();
        if (tid == 0 && t + 2 < n_tiles) {
            fence_proxy_async();
            const int k2 = k_begin + (t + 2) * kTileSteps;
            const unsigned bytes = (unsigned)min(kTileSteps, k_end - k2 + 1) * sizeof(RecM);
            mbar_arrive_expect_tx(&bar[buf], bytes);
            bulk_g2s(tile[buf], rec + k2, bytes, &bar[buf]);
        }
    }
    g_base += (unsigned)n_tiles;
    // close the last bin; count clipped intervals and crossed bin edges
    if (c.live[0]) {
        flush(c.row[0], C.n_bins, c.b[0], c.acc[0].x, c.acc[1].x, c.acc[2].x, c.acc[3].x, c.acc[4].x, c.acc[5].x);
        clip += (unsigned long long)min(n_int, c.below[0] + c.above[0]);
    }
    if (c.live[1]) {
        flush(c.row[1], C.n_bins, c.b[1], c.acc[0].y, c.acc[1].y, c.acc[2].y, c.acc[3].y, c.acc[4].y, c.acc[5].y);
        clip += (unsigned long long)min(n_int, c.below[1] + c.above[1]);
    }
    if (clip) atomicAdd(&P.counters->clipped, clip);
    // warp-aggregated count of bin edges crossed (bins touched = intervals + crossings)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) crossed += __shfl_xor_sync(0xffffffffu, crossed, o);
    if ((tid & 31) == 0 && crossed) atomicAdd(&P.counters->crossings, crossed);
    return true;
}

__device__ __forceinline__ void init_staging(uint64_t* bar)
{
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kMixedThreads, RD_MIXED_MINBLOCKS) k_deposit_mixed(const DepositParams P)
{
    __shared__ __align__(128) RecM tile[2][kTileSteps];
    __shared__ __align__(8) uint64_t bar[2];
    init_staging(bar);
    const unsigned bid = blockIdx.x;
    const int p = (int)(bid % (unsigned)P.n_part);
    const unsigned rest = bid / (unsigned)P.n_part;
    const int cb = (int)(rest % (unsigned)P.n_cell_blocks);
    const int ch = (int)(rest / (unsigned)P.n_cell_blocks);
    unsigned g = 0;
    (void)deposit_item(P, p, cb, ch, tile, bar, g);
}

// Persistent form: the resident CTAs draw work items of all problems from one counter.
// Items of problem i are [item_off[i], item_off[i+1]), ordered particle-fastest within a
// (chunk, cell block) like the single-problem grid.  The counter only grows (atomicAdd): no CTA
// ever waits on another.
__global__ void __launch_bounds__(kMixedThreads, RD_MIXED_MINBLOCKS)
    k_deposit_batch(const DepositParams* __restrict__ probs, const long long* __restrict__ item_off, int n_probs,
                    unsigned long long* next_item)
{
    __shared__ __align__(128) RecM tile[2][kTileSteps];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ long long s_item;
    init_staging(bar);
    const long long total = item_off[n_probs];
    unsigned g = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(next_item, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        int lo = 0, hi = n_probs - 1;
        while (lo < hi) {                       // last problem whose first item <= item
            const int mid = (lo + hi + 1) >> 1;
            if (item_off[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const DepositParams P = probs[lo];
        const long long local = item - item_off[lo];
        const int p = (int)(local % P.n_part);
        const long long rest = local / P.n_part;
        const int cb = (int)(rest % P.n_cell_blocks);
        const int ch = (int)(rest / P.n_cell_blocks);
        if (!deposit_item(P, p, cb, ch, tile, bar, g)) break;
    }
}

cudaError_t launch_deposit_batch(const DepositParams* probs, const long long* item_off, int n_probs,
                                 unsigned long long* next_item, int grid, cudaStream_t s)
{
    k_deposit_batch<<<grid, kMixedThreads, 0, s>>>(probs, item_off, n_probs, next_item);
    return cudaGetLastError();
}

int batch_grid()
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deposit_batch, kMixedThreads, 0);
    return std::max(1, sms) * std::max(1, per_sm);
}

cudaError_t launch_deposit_mixed(const DepositParams& p, cudaStream_t s)
{
    const long long blocks = (long long)p.n_cell_blocks * p.n_part * p.n_chunks;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_deposit_mixed<<<(unsigned)blocks, kMixedThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace rd
