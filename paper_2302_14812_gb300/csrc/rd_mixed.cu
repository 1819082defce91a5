// Mixed-precision deposit: FP32 Lienard-Wiechert field (Eq. 1) and FP32 accumulation, with the
// arrival time (Eq. 2) kept FP64-accurate.
//
// Work item = (step chunk, block of CPC cells, particle) with CPC = 64, 128 or 256 (the launch
// shape; 256 by default), ordered by item_coords: consecutive CTAs take one particle to a small
// group of cell blocks, then the next particle (odd groups in reverse particle order), so the CTAs
// resident at one time reduce into the group's slice of the detector, which stays in L2, and each
// particle's staged records come from DRAM about once per group.
//
// Each thread walks NC cells (1 or 2) through the chunk; the per-sample constants (RecS) are read
// once per sample from shared memory and serve all of them.  Per cell the walk carries the bin it
// is filling (as an offset from the CTA's first field row) and the time f already spent in that
// bin, in units of dt; a step adds the arrival-time increment
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

// Bin indices of the walk are clamped to +-2^29 so that offsets (row * n_bins + bin, with
// n_bins <= kMixedMaxBins) and differences of two of them stay inside int32.
constexpr double kWalkClamp = 536870912.0;

__device__ __forceinline__ int walk_bin(double fb) { return (int)fmin(fmax(fb, -kWalkClamp), kWalkClamp); }

// Walk state of the thread's NC cells.
template <int NC>
struct Cells {
    float px[NC], py[NC], pz[NC];   // cell positions
    float f[NC];                    // time spent in the current bin, units of dt (0 <= f < W)
    float rpd[NC];                  // R_{k-1} + dt (far-field limit: 1/R_c)
    float nlx[NC], nly[NC], nlz[NC];  // far-field limit: n_c - (its FP32 rounding in px, py, pz)
    float acc[6][NC];               // E xyz, B xyz of the current bin so far (weights in bins)
    float gp[6][NC];                // linear / quadratic interpolation: scaled field of the previous sample
    float gpp[6][NC];               // quadratic interpolation: scaled field two samples back ...
    float hp[NC];                   // ... and the previous interval's length (units of dt)
    int bo[NC];                     // row * n_bins + bin being filled (bin may lie outside the window)
    int rb[NC];                     // row * n_bins (row = the cell's index inside the CTA's block)
    bool live[NC];                  // some arrival of the chunk falls inside the window
    int below[NC];                  // intervals whose start lies before the window (clip tracking only)
    int above[NC];                  // intervals whose end lies after the window (clip tracking only)
};

#ifndef RD_CHECK
#define RD_CHECK 0   // 1: the walk's unguarded reductions check their bin (a checked build, for tests)
#endif

struct Consts {
    float W;                        // bin width / dt
    float invW;
    float DT;
    int n_bins;
    float* base;                    // field row 0 of the CTA's cell block
    int kq;                         // quadratic interpolation: first interval (this call's index) with
                                    // three fields behind it (the trajectory's third interval)
#if RD_CHECK
    unsigned* errors;               // the detector's latched error bits
#endif
};

// Checked build: a reduction the window margin should keep inside the detector row is verified,
// and one that would leave it latches RD_ERR_BOUNDS and is dropped.
__device__ __forceinline__ bool bin_ok(const Consts& C, int b)
{
#if RD_CHECK
    if ((unsigned)b < (unsigned)C.n_bins) return true;
    atomicOr(C.errors, ERRBIT_BOUNDS);
    return false;
#else
    (void)C;
    (void)b;
    return true;
#endif
}

// Field of one sample at one cell, scaled to the bin weights (E = S E', B = (S/R) d x E').
struct Field {
    float E[3];                     // E' = Q [(n - beta)(-c1/kappa) + betadot],  Q = -q dt/dt_det
    float B[3];                     // d x E'
    float S;                        // 1 / (kappa^2 R)
    float rinv;                     // 1 / R
    float num, rden;                // t'_k - t'_{k-1} = num * rden in units of dt
};

__device__ __forceinline__ float* bin_addr(const Consts& C, int bo)
{
    return reinterpret_cast<float*>(reinterpret_cast<char*>(C.base) + (size_t)(unsigned)bo * 32u);
}

// Add one bin (b = bin index, bo = its offset) to global memory; bins outside the window are dropped.
__device__ __forceinline__ void flush(const Consts& C, int b, int bo, float e0, float e1, float e2, float b0,
                                      float b1, float b2)
{
    if ((unsigned)b < (unsigned)C.n_bins) {
        float* p = bin_addr(C, bo);
        red_add_v4(p, e0, e1, e2, b0);
        red_add_v2(p + 4, b1, b2);
    }
}

// B of a bin.  Far-field limit: every sample of a cell has the same n_c and scale (1/R_c folded
// into S, 1/R = 1), so B = n_c x E holds for each sample's weighted field and hence for the bin
// sums: the walk carries E only and forms B when the bin is written.  Otherwise B is carried.
template <int NC, bool FF>
__device__ __forceinline__ void bin_b(const Cells<NC>& c, int j, const float* e, const float* carried, float* b)
{
    if (FF) {
        b[0] = fmaf(c.py[j], e[2], -(c.pz[j] * e[1]));
        b[1] = fmaf(c.pz[j], e[0], -(c.px[j] * e[2]));
        b[2] = fmaf(c.px[j], e[1], -(c.py[j] * e[0]));
    } else {
        b[0] = carried[0];
        b[1] = carried[1];
        b[2] = carried[2];
    }
}

// Add bin b of cell j from its accumulator.
template <int NC, bool FF>
__device__ __forceinline__ void flush_acc(const Consts& C, const Cells<NC>& c, int j, int b, int bo)
{
    const float e[3] = {c.acc[0][j], c.acc[1][j], c.acc[2][j]};
    const float cb[3] = {c.acc[3][j], c.acc[4][j], c.acc[5][j]};
    float bb[3];
    bin_b<NC, FF>(c, j, e, cb, bb);
    flush(C, b, bo, e[0], e[1], e[2], bb[0], bb[1], bb[2]);
}

// Eq. 1 with B = n x E at one cell:
//   E = q/(kappa^3 R) [ (n - beta)(gamma^-2/R + n.betadot) - betadot kappa ]
//     = S E',  S = 1/(kappa^2 R),  E' = -q [(n - beta)(-c1/kappa) + betadot],  c1 = gamma^-2/R + n.betadot
//   B = n x E = (S/R) d x E'
// E' also carries the bin weight per unit dt (the records hold Q = -q dt/dt_det times betadot and
// gamma^-2), and kappa = (gamma^-2 + |n - beta|^2)/2 avoids the cancellation in 1 - beta.n.
__device__ __forceinline__ void field_at(const RecS& r, float px, float py, float pz, float& rpd, const Consts& C,
                                         Field& o)
{
    // geometry: d = x_cell - x_k, R = |d|
    const float dx = px + r.nx, dy = py + r.ny, dz = pz + r.nz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float rinv = fast_rsqrt(r2);
    const float bx = fmaf(dx, rinv, r.nbx), by = fmaf(dy, rinv, r.nby), bz = fmaf(dz, rinv, r.nbz);   // n - beta
    const float nb2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
    // arrival-time increment in units of dt, numerator and denominator divided by R:
    //   [dt g / R + (g + |n - vbar|^2)] / [1 + (R_{k-1} + dt) / R],
    //   g + |n - vbar|^2 = |n - beta|^2 + 2 (n - beta).(beta - vbar) + (g + |beta - vbar|^2)
    const float gg = fmaf(bx, r.d2x, fmaf(by, r.d2y, fmaf(bz, r.d2z, nb2 + r.gd)));
    const float num = fmaf(r.dtg, rinv, gg);
    const float den = fmaf(rpd, rinv, 1.f);
    o.num = num;
    o.rden = fast_rcp(den);
    rpd = fmaf(r2, rinv, C.DT);
    // Eq. 1
    const float kn = fmaf(nb2, -0.5f, r.nhig2);                         // -kappa
    const float ikn = fast_rcp(kn);                                     // -1/kappa
    const float nrik = rinv * ikn;                                      // -1/(kappa R)
    o.S = nrik * ikn;                                                   // 1/(kappa^2 R)
    // with the record's charge factor Q: Q (gamma^-2 + d.betadot) (-1/(kappa R)) = -Q c1/kappa
    const float c1n = fmaf(dx, r.bdx, fmaf(dy, r.bdy, fmaf(dz, r.bdz, r.ig2n))) * nrik;
    o.E[0] = fmaf(bx, c1n, r.bdx);
    o.E[1] = fmaf(by, c1n, r.bdy);
    o.E[2] = fmaf(bz, c1n, r.bdz);
    o.B[0] = fmaf(dy, o.E[2], -(dz * o.E[1]));
    o.B[1] = fmaf(dz, o.E[0], -(dx * o.E[2]));
    o.B[2] = fmaf(dx, o.E[1], -(dy * o.E[0]));
    o.rinv = rinv;
}

// Far-field limit (RD_FARFIELD) at one cell, seen from the origin along n_c at R_c (n_c and
// 1/R_c fixed per cell):
//   t'_k - t'_{k-1} = dt (1 - n_c.vbar) = dt [g + |n_c - vbar|^2] / 2   (Eq. 3, |n_c| = 1)
//   E = S E',  S = 1/(kappa^2 R_c),  E' = Q [(n_c - beta)(-n_c.betadot/kappa) + betadot],  B = S n_c x E'
// with kappa = 1 - beta.n_c = (gamma^-2 + |n_c - beta|^2)/2.  n_c is held as its FP32 rounding
// (nx, ny, nz) plus the rest (lx, ly, lz): the rounding is fixed per cell, and along the beam, where
// n_c - beta is ~1e-3, it would bias kappa by ~5e-5 (the field by ~1.5e-4, as kappa^-3) on every
// sample of the cell.  nx - beta_x is exact there (the two are within a factor of two), and adding
// the rest restores n_c - beta to FP32 precision.
__device__ __forceinline__ void field_at_ff(const RecS& r, float nx, float ny, float nz, float invR, float lx,
                                            float ly, float lz, Field& o)
{
    const float bx = (nx + r.nbx) + lx, by = (ny + r.nby) + ly, bz = (nz + r.nbz) + lz;   // n_c - beta
    const float nb2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
    o.num = fmaf(bx, r.d2x, fmaf(by, r.d2y, fmaf(bz, r.d2z, nb2 + r.gd)));
    o.rden = 0.5f;
    const float kn = fmaf(nb2, -0.5f, r.nhig2);                         // -kappa
    const float ikn = fast_rcp(kn);
    o.S = (ikn * ikn) * invR;
    const float c1n = fmaf(nx, r.bdx, fmaf(ny, r.bdy, nz * r.bdz)) * ikn; // -Q n_c.betadot / kappa
    o.E[0] = fmaf(bx, c1n, r.bdx);
    o.E[1] = fmaf(by, c1n, r.bdy);
    o.E[2] = fmaf(bz, c1n, r.bdz);
    o.B[0] = fmaf(ny, o.E[2], -(nz * o.E[1]));
    o.B[1] = fmaf(nz, o.E[0], -(nx * o.E[2]));
    o.B[2] = fmaf(nx, o.E[1], -(ny * o.E[0]));
    o.rinv = 1.f;
}

// Interval of cell j that passes two or more bin edges (rare): flush the bin being filled and the
// whole bins inside the interval, leaving the state one edge short so that the common path below
// finishes the step (it flushes the last whole bin and starts the next).
template <int NC, bool TRACK, bool FF>
__device__ __forceinline__ void multi_edges(Cells<NC>& c, int j, const Field& o, const Consts& C, float& fn, int k,
                                            int k_begin, int k_end)
{
    const float f = fn;
    if (!(f >= 2.f * C.W)) return;
    const int b0 = c.bo[j] - c.rb[j];
    const int m = (int)fminf(floorf(f * C.invW), 16777216.f);      // edges passed, >= 2
    flush_acc<NC, FF>(C, c, j, b0, c.bo[j]);
    const float fs = C.W * o.S, fb = fs * o.rinv;
    // whole bins b0+1 .. b0+m-2 now; bin b0+m-1 is left in the accumulator for the common path
    const int lo = max(b0 + 1, 0), hi = min(b0 + m - 2, C.n_bins - 1);
    for (int b = lo; b <= hi; ++b)
        flush(C, b, c.rb[j] + b, o.E[0] * fs, o.E[1] * fs, o.E[2] * fs, o.B[0] * fb, o.B[1] * fb, o.B[2] * fb);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        c.acc[i][j] = o.E[i] * fs;
        if (!FF) c.acc[3 + i][j] = o.B[i] * fb;
    }
    c.bo[j] += m - 1;
    fn = fminf(fmaxf(fmaf(-(float)(m - 1), C.W, f), C.W), C.W * 1.99999988f);
    if (TRACK) {
        if (b0 < 0 && b0 + m - 1 >= 0) c.below[j] = k - k_begin + 1;
        if (b0 < C.n_bins && b0 + m - 1 >= C.n_bins) c.above[j] = k_end - k + 1;
    }
}

// Field of the sample in bin-weight units per unit dt: G = (S E', (S/R) d x E').
__device__ __forceinline__ void scaled_field(const Field& o, float* G)
{
    const float sb = o.S * o.rinv;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        G[i] = o.E[i] * o.S;
        G[3 + i] = o.B[i] * sb;
    }
}

// Linear interpolation (RD_LINEAR; with the ramp terms scaled to zero, ramp = 0, the previous field
// held over the interval, RD_HOLD_PREV): over the interval the field goes linearly from G0 = gp (previous
// sample) to G (this sample); the part [s0, s1] of the interval (dt units from its start, length L)
// weighs G0 (s1 - s0) + (G - G0) (s1^2 - s0^2) / (2 L) = G0 (s1 - s0 - ramp) + G ramp with
// ramp = (s1^2 - s0^2) / (2 L).  Quadratic interpolation (RD_QUADRATIC) adds D2 cu, D2 the second
// divided difference of the scaled fields of samples k-2, k-1, k over their arrival times and
// cu = int_{s0}^{s1} s (s - L) ds (qcube below).  Interval of cell j passing two or more bin
// edges (exact walk only): flush the bin being filled, every whole bin, and leave the last, partial
// bin in the accumulator with the time already in it; fn comes back below W (no edge left for the
// common path).
// s^2 (s/3 - L/2): int_0^s t (t - L) dt
__device__ __forceinline__ float qcube(float s, float L) { return (s * s) * fmaf(s, 1.f / 3.f, -0.5f * L); }

template <int NC, bool TRACK, bool FF, bool QUAD>
__device__ __forceinline__ void multi_edges_lin(Cells<NC>& c, int j, const float* G, const float* D2, float L,
                                                float inv2L, const Consts& C, float& fn, int k, int k_begin, int k_end)
{
    constexpr int NF = FF ? 3 : 6;                                  // carried field components
    const float f = fn;
    if (!(f >= 2.f * C.W)) return;
    const float f0 = c.f[j];
    const int b0 = c.bo[j] - c.rb[j];
    const int m = (int)fminf(floorf(f * C.invW), 16777216.f);      // edges passed, >= 2
    flush_acc<NC, FF>(C, c, j, b0, c.bo[j]);
    // whole bins b0+i, i = 1..m-1, cover [i W, (i+1) W] from the start of bin b0
    const int lo = max(1, -b0), hi = min(m - 1, C.n_bins - 1 - b0);
    for (int i = lo; i <= hi; ++i) {
        const float s0 = fmaf((float)i, C.W, -f0), s1 = s0 + C.W;
        const float ramp = (s1 * s1 - s0 * s0) * inv2L;
        float v[6];
#pragma unroll
        for (int q = 0; q < NF; ++q) v[q] = fmaf(c.gp[q][j], C.W - ramp, G[q] * ramp);
        if (QUAD) {
            const float cu = qcube(s1, L) - qcube(s0, L);
#pragma unroll
            for (int q = 0; q < NF; ++q) v[q] = fmaf(D2[q], cu, v[q]);
        }
        bin_b<NC, FF>(c, j, v, v + 3, v + 3);
        flush(C, b0 + i, c.bo[j] + i, v[0], v[1], v[2], v[3], v[4], v[5]);
    }
    // bin b0+m holds [m W, f]
    const float s0 = fmaf((float)m, C.W, -f0);
    const float len = fmaf(-(float)m, C.W, f);
    const float ramp = (L * L - s0 * s0) * inv2L;
#pragma unroll
    for (int q = 0; q < NF; ++q) c.acc[q][j] = fmaf(c.gp[q][j], len - ramp, G[q] * ramp);
    if (QUAD) {
        const float cu = qcube(L, L) - qcube(s0, L);
#pragma unroll
        for (int q = 0; q < NF; ++q) c.acc[q][j] = fmaf(D2[q], cu, c.acc[q][j]);
    }
    c.bo[j] += m;
    fn = fminf(fmaxf(len, 0.f), C.W * 0.99999994f);
    if (TRACK) {
        if (b0 < 0 && b0 + m >= 0) c.below[j] = k - k_begin + 1;
        if (b0 < C.n_bins && b0 + m >= C.n_bins) c.above[j] = k_end - k + 1;
    }
}

// Walk modes.  kFast: the common step, with no code for an interval that passes two or more bin
// edges; such an interval sets the cell's time to -inf, after which the cell crosses no edge and
// flushes nothing for the rest of the tile.  kExact: the same arithmetic plus the multi-edge case;
// used to walk a tile again (from its saved start) for a warp in which some cell stopped, flushing
// only from the interval that stopped it onwards (earlier bins were flushed by the fast walk).
// Both walks evaluate every value with the same operations in the same order (no implicit
// contraction), so they agree bit for bit up to that interval.
enum { kFast = 0, kExact = 1 };

// One interval for all cells of the thread: field of the sample (Eq. 1), the part of [f, f + du]
// inside the current bin added to the running bin; a cell whose arrival time passes the bin edge
// flushes the bin and starts the next one with the rest of the interval.  LAST: the interval ends
// on the exact FP64 anchors.  TRACK: bins may lie outside the window (checked, clipped intervals
// counted).  ok: kExact only, false from the interval that stopped the fast walk onwards.
template <int NC, int MODE, bool LAST, bool TRACK, bool FF, int LIN>
__device__ __forceinline__ void step(Cells<NC>& c, const RecS& r, const Consts& C, const int* bo_end,
                                     const float* f_end, int k, int k_begin, int k_end, bool* ok, float ramp)
{
    constexpr int NF = FF ? 3 : 6;                  // carried field components (far field: E only)
    constexpr bool QUAD = LIN == 2;                 // quadratic interpolation (RD_QUADRATIC)
    Field o[NC];
    float fn[NC];
    float G[NC][6], L[NC], inv2L[NC], ramp1[NC];               // linear / quadratic interpolation only
    float D2[NC][6], cu1[NC];                                  // quadratic interpolation only
    // the trajectory's first two intervals have fewer than three fields behind them: no curvature
    const float qon = (QUAD && k >= C.kq) ? 1.f : 0.f;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (FF)
            field_at_ff(r, c.px[j], c.py[j], c.pz[j], c.rpd[j], c.nlx[j], c.nly[j], c.nlz[j], o[j]);
        else
            field_at(r, c.px[j], c.py[j], c.pz[j], c.rpd[j], C, o[j]);
        float t;
        if (LAST) {
            t = fmaf((float)(bo_end[j] - c.bo[j]), C.W, f_end[j]);
            if (MODE == kFast) t = c.f[j] == -INFINITY ? -INFINITY : t;
        } else {
            t = fmaf(o[j].num, o[j].rden, c.f[j]);
        }
        if (LIN) {
            scaled_field(o[j], G[j]);
            L[j] = t - c.f[j];
            inv2L[j] = (0.5f * ramp) * fast_rcp(fmaxf(L[j], 1e-30f));
            const float len1 = fminf(t, C.W) - c.f[j];
            ramp1[j] = (len1 * len1) * inv2L[j];
            // G0 (s1 - s0) + (G - G0) ramp = G0 (s1 - s0 - ramp) + G ramp
            const float a1 = len1 - ramp1[j];
#pragma unroll
            for (int i = 0; i < NF; ++i) c.acc[i][j] = fmaf(c.gp[i][j], a1, fmaf(G[j][i], ramp1[j], c.acc[i][j]));
            if (QUAD) {
                // D2 = ((G - G0) / L - (G0 - Gpp) / h) / (L + h), h the previous interval (ramp = 1 here,
                // so 2 inv2L = 1/L); the part [0, len1] adds D2 int_0^len1 s (s - L) ds
                const float iL = 2.f * inv2L[j];
                const float ih = fast_rcp(c.hp[j]);
                const float iLh = qon * fast_rcp(L[j] + c.hp[j]);
                cu1[j] = qcube(len1, L[j]);
#pragma unroll
                for (int i = 0; i < NF; ++i) {
                    D2[j][i] = fmaf(G[j][i] - c.gp[i][j], iL, -((c.gp[i][j] - c.gpp[i][j]) * ih)) * iLh;
                    c.acc[i][j] = fmaf(D2[j][i], cu1[j], c.acc[i][j]);
                }
            }
        } else {
            const float ws = (fminf(t, C.W) - c.f[j]) * o[j].S;
            const float wb = ws * o[j].rinv;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                c.acc[i][j] = fmaf(o[j].E[i], ws, c.acc[i][j]);
                if (!FF) c.acc[3 + i][j] = fmaf(o[j].B[i], wb, c.acc[3 + i][j]);
            }
        }
        if (MODE == kFast)
            t = t < 2.f * C.W ? t : -INFINITY;
        else
            ok[j] = ok[j] && (t < 2.f * C.W);
        fn[j] = t;
    }
    if (MODE == kExact) {
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            if (LIN)
                multi_edges_lin<NC, TRACK, FF, QUAD>(c, j, G[j], D2[j], L[j], inv2L[j], C, fn[j], k, k_begin, k_end);
            else
                multi_edges<NC, TRACK, FF>(c, j, o[j], C, fn[j], k, k_begin, k_end);
        }
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        // the arrival time passed the bin edge (a time exactly on the edge belongs to the upper bin)
        const bool cr = fn[j] >= C.W;
        if (MODE == kFast && !TRACK) {
            if (cr) {
                float* a = bin_addr(C, c.bo[j]);
                const float e[3] = {c.acc[0][j], c.acc[1][j], c.acc[2][j]};
                const float cb[3] = {c.acc[3][j], c.acc[4][j], c.acc[5][j]};
                float bb[3];
                bin_b<NC, FF>(c, j, e, cb, bb);
                if (bin_ok(C, c.bo[j] - c.rb[j])) {
                    red_add_v4(a, e[0], e[1], e[2], bb[0]);
                    red_add_v2(a + 4, bb[1], bb[2]);
                }
                const float rem = fn[j] - C.W;
                if (LIN) {
                    const float ramp2 = fmaf(0.5f * ramp, L[j], -ramp1[j]);
#pragma unroll
                    for (int i = 0; i < NF; ++i) c.acc[i][j] = fmaf(c.gp[i][j], rem - ramp2, G[j][i] * ramp2);
                    if (QUAD) {
                        const float cu2 = qcube(L[j], L[j]) - cu1[j];       // the part [len1, L]
#pragma unroll
                        for (int i = 0; i < NF; ++i) c.acc[i][j] = fmaf(D2[j][i], cu2, c.acc[i][j]);
                    }
                } else {
                    const float rs = rem * o[j].S;
                    const float rbw = rs * o[j].rinv;
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        c.acc[i][j] = o[j].E[i] * rs;
                        if (!FF) c.acc[3 + i][j] = o[j].B[i] * rbw;
                    }
                }
                c.f[j] = rem;
                c.bo[j] += 1;
            } else {
                c.f[j] = fn[j];
            }
        } else {
            const int b = c.bo[j] - c.rb[j];
            const bool go = MODE == kFast || !ok[j];
            const bool pr = cr && go && (TRACK ? (unsigned)b < (unsigned)C.n_bins : (!RD_CHECK || bin_ok(C, b)));
            float* a = bin_addr(C, c.bo[j]);
            const float e[3] = {c.acc[0][j], c.acc[1][j], c.acc[2][j]};
            const float cb[3] = {c.acc[3][j], c.acc[4][j], c.acc[5][j]};
            float bb[3];
            bin_b<NC, FF>(c, j, e, cb, bb);
            red_add_v4_if(pr, a, e[0], e[1], e[2], bb[0]);
            red_add_v2_if(pr, a + 4, bb[1], bb[2]);
            const float rem = fn[j] - C.W;
            if (LIN) {
                const float ramp2 = fmaf(0.5f * ramp, L[j], -ramp1[j]);
                const float cu2 = QUAD ? qcube(L[j], L[j]) - cu1[j] : 0.f;
#pragma unroll
                for (int i = 0; i < NF; ++i) {
                    float v = fmaf(c.gp[i][j], rem - ramp2, G[j][i] * ramp2);
                    if (QUAD) v = fmaf(D2[j][i], cu2, v);
                    c.acc[i][j] = cr ? v : c.acc[i][j];
                }
            } else {
                const float rs = rem * o[j].S;
                const float rbw = rs * o[j].rinv;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    c.acc[i][j] = cr ? o[j].E[i] * rs : c.acc[i][j];
                    if (!FF) c.acc[3 + i][j] = cr ? o[j].B[i] * rbw : c.acc[3 + i][j];
                }
            }
            c.f[j] = cr ? rem : fn[j];
            if (TRACK) {
                if (cr && b == -1) c.below[j] = k - k_begin + 1;
                if (cr && b == C.n_bins - 1) c.above[j] = k_end - k + 1;
            }
            c.bo[j] += cr ? 1 : 0;
        }
        if (LIN) {
#pragma unroll
            for (int i = 0; i < NF; ++i) {
                if (QUAD) c.gpp[i][j] = c.gp[i][j];
                c.gp[i][j] = G[j][i];
            }
            if (QUAD) c.hp[j] = L[j];
        }
    }
}

#ifndef RD_UNROLL
#define RD_UNROLL 0
#endif
constexpr int kUnroll = RD_UNROLL > 0 ? RD_UNROLL : 1;   // samples per loop iteration

// Per-thread copy of the walk state at the start of a tile, in shared memory ([word][thread]):
// f, rpd, bo, below, above, acc[6], gp[6], and for the quadratic interpolation gpp[6], hp.
constexpr int save_cell(int lin) { return lin == 2 ? 24 : 17; }

template <int NC, int NT, bool FF, int LIN>
__device__ __forceinline__ void save_state(const Cells<NC>& c, float (*sv)[NT], int tid)
{
    constexpr int NF = FF ? 3 : 6;
    constexpr int kSaveCell = save_cell(LIN);
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        sv[j * kSaveCell + 0][tid] = c.f[j];
        sv[j * kSaveCell + 1][tid] = c.rpd[j];
        sv[j * kSaveCell + 2][tid] = __int_as_float(c.bo[j]);
        sv[j * kSaveCell + 3][tid] = __int_as_float(c.below[j]);
        sv[j * kSaveCell + 4][tid] = __int_as_float(c.above[j]);
#pragma unroll
        for (int i = 0; i < NF; ++i) sv[j * kSaveCell + 5 + i][tid] = c.acc[i][j];
        if (LIN) {
#pragma unroll
            for (int i = 0; i < NF; ++i) sv[j * kSaveCell + 11 + i][tid] = c.gp[i][j];
        }
        if (LIN == 2) {
#pragma unroll
            for (int i = 0; i < NF; ++i) sv[j * kSaveCell + 17 + i][tid] = c.gpp[i][j];
            sv[j * kSaveCell + 23][tid] = c.hp[j];
        }
    }
}

template <int NC, int NT, bool FF, int LIN>
__device__ __forceinline__ void restore_state(Cells<NC>& c, float (*sv)[NT], int tid)
{
    constexpr int NF = FF ? 3 : 6;
    constexpr int kSaveCell = save_cell(LIN);
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        c.f[j] = sv[j * kSaveCell + 0][tid];
        c.rpd[j] = sv[j * kSaveCell + 1][tid];
        c.bo[j] = __float_as_int(sv[j * kSaveCell + 2][tid]);
        c.below[j] = __float_as_int(sv[j * kSaveCell + 3][tid]);
        c.above[j] = __float_as_int(sv[j * kSaveCell + 4][tid]);
#pragma unroll
        for (int i = 0; i < NF; ++i) c.acc[i][j] = sv[j * kSaveCell + 5 + i][tid];
        if (LIN) {
#pragma unroll
            for (int i = 0; i < NF; ++i) c.gp[i][j] = sv[j * kSaveCell + 11 + i][tid];
        }
        if (LIN == 2) {
#pragma unroll
            for (int i = 0; i < NF; ++i) c.gpp[i][j] = sv[j * kSaveCell + 17 + i][tid];
            c.hp[j] = sv[j * kSaveCell + 23][tid];
        }
    }
}

template <int NC, int NT, bool TRACK, bool FF, int LIN>
__device__ __forceinline__ void walk_tile(Cells<NC>& c, const RecS* tile, int cnt, bool last_tile, const Consts& C,
                                          float ramp, const int* bo_end, const float* f_end, int k0, int k_begin,
                                          int k_end, float (*sv)[NT])
{
    const int tid = threadIdx.x;
    const int n_regular = last_tile ? cnt - 1 : cnt;
    save_state<NC, NT, FF, LIN>(c, sv, tid);
    bool ok[NC];
#pragma unroll kUnroll
    for (int i = 0; i < n_regular; ++i)
        step<NC, kFast, false, TRACK, FF, LIN>(c, tile[i], C, bo_end, f_end, k0 + i, k_begin, k_end, ok, ramp);
    if (last_tile)
        step<NC, kFast, true, TRACK, FF, LIN>(c, tile[cnt - 1], C, bo_end, f_end, k_end, k_begin, k_end, ok, ramp);
    bool stopped = false;
#pragma unroll
    for (int j = 0; j < NC; ++j) stopped = stopped || c.f[j] == -INFINITY;
    if (__any_sync(0xffffffffu, stopped)) {
        // some interval of a cell of this warp passed two or more bin edges: walk the tile again
        restore_state<NC, NT, FF, LIN>(c, sv, tid);
#pragma unroll
        for (int j = 0; j < NC; ++j) ok[j] = true;
#pragma unroll 1
        for (int i = 0; i < n_regular; ++i)
            step<NC, kExact, false, TRACK, FF, LIN>(c, tile[i], C, bo_end, f_end, k0 + i, k_begin, k_end, ok, ramp);
        if (last_tile)
            step<NC, kExact, true, TRACK, FF, LIN>(c, tile[cnt - 1], C, bo_end, f_end, k_end, k_begin, k_end, ok, ramp);
    }
}

}  // namespace

// One work item -- particle p, cell block cb, step chunk ch of one problem -- run by the whole
// CTA.  tile / bar: the CTA's shared staging buffers; g_base counts the tiles the CTA staged
// before this item (it selects buffer and mbarrier phase, so the buffers carry over between items).
// Returns false if a bounded wait ran out (the error is recorded; the CTA must stop).
template <bool FF, int LIN, int NC, int CPC>
__device__ __forceinline__ bool deposit_item(const DepositParams& P, int p, int cb, int ch,
                                             RecS (*tile)[kTileSteps], uint64_t* bar, float (*sv)[CPC / NC],
                                             unsigned& g_base)
{
    constexpr int NT = CPC / NC;                // threads of the CTA
    const int S = P.n_samples - 1;
    const int k_begin = P.k_first + ch * P.chunk;
    const int k_end = min(S, k_begin + P.chunk - 1);
    const int n_int = k_end - k_begin + 1;
    const int n_tiles = (n_int + kTileSteps - 1) / kTileSteps;
    const RecS* rec = static_cast<const RecS*>(P.rec) + (size_t)p * P.n_samples;
    const int tid = threadIdx.x;

    if (tid == 0) {
        fence_proxy_async();
        for (int t = 0; t < 2 && t < n_tiles; ++t) {
            const int k0 = k_begin + t * kTileSteps;
            const unsigned g = g_base + t;
            const unsigned bytes = (unsigned)min(kTileSteps, k_end - k0 + 1) * sizeof(RecS);
            mbar_arrive_expect_tx(&bar[g & 1], bytes);
            bulk_g2s(tile[g & 1], rec + k0, bytes, &bar[g & 1]);
        }
    }

    Consts C;
    C.W = P.W;
    C.invW = P.invW;
    C.DT = P.dt_f;
    C.n_bins = P.n_bins;
    C.base = static_cast<float*>(P.fields) + (size_t)cb * CPC * P.n_bins * 8;
    C.kq = 3 - P.k_real0;
#if RD_CHECK
    C.errors = &P.counters->errors;
#endif
    constexpr bool QUAD = LIN == 2;
    const bool q_prev = QUAD && k_begin >= 3;     // the chunk starts with three fields behind it

    // anchors: exact FP64 arrival (bins) at both ends of the chunk, per cell
    Cells<NC> c;
    int bo_end[NC];
    float f_end[NC];
    float hp0[NC];                              // quadratic: length of interval k_begin - 1 (dt units)
    bool partial = false;
    unsigned long long clip = 0, crossed = 0;
    const double* xp = P.x + (size_t)p * P.n_samples * 3;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const int row = j * NT + tid;
        const int cell = cb * CPC + row;
        // a cell without arrivals in the window still walks (no per-cell branch in the step) but
        // from a time that never reaches a bin edge: nothing is flushed
        c.rb[j] = row * P.n_bins;
        c.bo[j] = c.rb[j];
        c.live[j] = false;
        c.below[j] = c.above[j] = 0;
        c.f[j] = -1e30f;
        c.rpd[j] = 1e6f;
        c.px[j] = 1e6f;
        c.py[j] = c.pz[j] = 0.f;
        c.nlx[j] = c.nly[j] = c.nlz[j] = 0.f;
        bo_end[j] = c.bo[j];
        f_end[j] = 0.f;
#pragma unroll
        for (int i = 0; i < 6; ++i) c.acc[i][j] = 0.f;
        if (cell < P.n_pix) {
            const D4 cl = P.cells[cell];
            const double* xa = xp + 3 * (size_t)(k_begin - 1);
            const double* xe = xp + 3 * (size_t)k_end;
            double Ra = 0.0, Re, ua, ue, ncx = 0.0, ncy = 0.0, ncz = 0.0, Rc = 1.0;
            if (FF) {
                farfield_cell(cl, ncx, ncy, ncz, Rc);
                ua = arrival_bins_ff(xa[0], xa[1], xa[2], ncx, ncy, ncz, Rc, cl.w, P.t0, k_begin - 1, P.dt, P.inv_dt_det);
                ue = arrival_bins_ff(xe[0], xe[1], xe[2], ncx, ncy, ncz, Rc, cl.w, P.t0, k_end, P.dt, P.inv_dt_det);
            } else {
                ua = arrival_bins(xa[0], xa[1], xa[2], cl, P.t0, k_begin - 1, P.dt, P.inv_dt_det, Ra);
                ue = arrival_bins(xe[0], xe[1], xe[2], cl, P.t0, k_end, P.dt, P.inv_dt_det, Re);
            }
            c.live[j] = (ue > 0.0) && (ua < (double)P.n_bins);
            hp0[j] = 1.f;
            if (q_prev && c.live[j]) {
                const double* xq = xp + 3 * (size_t)(k_begin - 2);
                double Rq;
                const double uq =
                    FF ? arrival_bins_ff(xq[0], xq[1], xq[2], ncx, ncy, ncz, Rc, cl.w, P.t0, k_begin - 2, P.dt,
                                         P.inv_dt_det)
                       : arrival_bins(xq[0], xq[1], xq[2], cl, P.t0, k_begin - 2, P.dt, P.inv_dt_det, Rq);
                hp0[j] = (float)((ua - uq) * P.W);
            }
            if (!c.live[j]) {
                clip += (unsigned long long)n_int;
            } else {
                const double fla = floor(ua), fle = floor(ue);
                c.bo[j] = c.rb[j] + walk_bin(fla);
                c.f[j] = (float)(ua - fla) * P.W;
                bo_end[j] = c.rb[j] + walk_bin(fle);
                f_end[j] = (float)(ue - fle) * P.W;
                if (FF) {
                    c.px[j] = (float)ncx;
                    c.py[j] = (float)ncy;
                    c.pz[j] = (float)ncz;
                    c.rpd[j] = (float)(1.0 / Rc);
                    c.nlx[j] = (float)(ncx - (double)c.px[j]);
                    c.nly[j] = (float)(ncy - (double)c.py[j]);
                    c.nlz[j] = (float)(ncz - (double)c.pz[j]);
                } else {
                    c.rpd[j] = (float)Ra + P.dt_f;
                    c.px[j] = (float)cl.x;
                    c.py[j] = (float)cl.y;
                    c.pz[j] = (float)cl.z;
                }
                c.below[j] = (ua < 0.0) ? n_int : 0;
                // unchecked bins need a margin of one bin to each window edge (the FP32 walk may
                // drift by far less than a bin before the end anchor corrects it)
                partial = partial || (ua < 1.0) || (ue > (double)P.n_bins - 1.0);
                crossed += (unsigned long long)max(0, bo_end[j] - c.bo[j]);
            }
        }
    }
    // clip tracking costs instructions in the bin-crossing path: only CTAs that need it use it
    if (LIN) {
        // field of the sample before the chunk; a trajectory's first interval holds F_1 (sample 0
        // has no field), so the first chunk starts from the field of sample 1 itself
        const RecS r0 = rec[k_begin > 1 ? k_begin - 1 : 1];
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            Field o;
            float rtmp = c.rpd[j];
            if (FF)
                field_at_ff(r0, c.px[j], c.py[j], c.pz[j], c.rpd[j], c.nlx[j], c.nly[j], c.nlz[j], o);
            else
                field_at(r0, c.px[j], c.py[j], c.pz[j], rtmp, C, o);
            float G[6];
            scaled_field(o, G);
#pragma unroll
            for (int i = 0; i < 6; ++i) c.gp[i][j] = G[i];      // far field: only E is read
            if (QUAD) {
                // the field two samples before the chunk and the interval before it (used from the
                // trajectory's third interval on)
                c.hp[j] = hp0[j];
                if (q_prev) {
                    const RecS r1 = rec[k_begin - 2];
                    float rtmp1 = c.rpd[j];
                    if (FF)
                        field_at_ff(r1, c.px[j], c.py[j], c.pz[j], c.rpd[j], c.nlx[j], c.nly[j], c.nlz[j], o);
                    else
                        field_at(r1, c.px[j], c.py[j], c.pz[j], rtmp1, C, o);
                    scaled_field(o, G);
                }
#pragma unroll
                for (int i = 0; i < 6; ++i) c.gpp[i][j] = G[i];
            }
        }
    }
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
            walk_tile<NC, NT, true, FF, LIN>(c, tile[buf], cnt, last_tile, C, P.lin == 2 ? 0.f : 1.f, bo_end, f_end, k0,
                                     k_begin, k_end, sv);
        else
            walk_tile<NC, NT, false, FF, LIN>(c, tile[buf], cnt, last_tile, C, P.lin == 2 ? 0.f : 1.f, bo_end, f_end, k0,
                                      k_begin, k_end, sv);
        __syncthreads();
        if (tid == 0 && t + 2 < n_tiles) {
            fence_proxy_async();
            const int k2 = k_begin + (t + 2) * kTileSteps;
            const unsigned bytes = (unsigned)min(kTileSteps, k_end - k2 + 1) * sizeof(RecS);
            mbar_arrive_expect_tx(&bar[buf], bytes);
            bulk_g2s(tile[buf], rec + k2, bytes, &bar[buf]);
        }
    }
    g_base += (unsigned)n_tiles;
    // close the last bin; count clipped intervals and crossed bin edges
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (c.live[j]) {
            flush_acc<NC, FF>(C, c, j, c.bo[j] - c.rb[j], c.bo[j]);
            clip += (unsigned long long)min(n_int, c.below[j] + c.above[j]);
        }
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

// Resident CTAs per SM the register allotment must allow: about 640 threads, as for the default
// shape (2 cells per thread, 256 cells per CTA: 128 threads, 5 CTAs).
#ifndef RD_QUAD_MINBLOCKS
#define RD_QUAD_MINBLOCKS 4      // the quadratic walk's CTAs per SM (its state needs more than 96 registers)
#endif
constexpr int mixed_min_blocks(int nt, int lin = 0)
{
    return nt >= 128 ? (nt == 128 ? (lin == 2 ? RD_QUAD_MINBLOCKS : RD_MIXED_MINBLOCKS) : 640 / nt) : 640 / nt;
}

template <bool FF, int LIN, int NC, int CPC>
__global__ void __launch_bounds__(CPC / NC, mixed_min_blocks(CPC / NC, LIN)) k_deposit_mixed(const DepositParams P)
{
    constexpr int NT = CPC / NC;
    __shared__ __align__(128) RecS tile[2][kTileSteps];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float sv[NC * save_cell(LIN)][NT];
    init_staging(bar);
    int p, cb, ch;
    item_coords(blockIdx.x, P, p, cb, ch);
    unsigned g = 0;
    (void)deposit_item<FF, LIN, NC, CPC>(P, p, cb, ch, tile, bar, sv, g);
}

// Persistent form: the resident CTAs draw work items of all problems from one counter.
// Items of problem i are [item_off[i], item_off[i+1]), ordered by item_coords like the
// single-problem grid.  The counter only grows (atomicAdd): no CTA ever waits on another.  One
// instantiation per walk family (far field or not x held / linear family / quadratic): a launch
// holds problems of one family, so the kernel carries only that walk's registers and shared
// state.  (Drawing the next item while walking the current one measured 8 % slower: the drawing
// thread then waits on the atomic before it issues the current item's record copies.)
template <bool FF, int LIN>
__global__ void __launch_bounds__(kMixedThreads, mixed_min_blocks(kMixedThreads, LIN))
    k_deposit_batch(const DepositParams* __restrict__ probs, const long long* __restrict__ item_off, int n_probs,
                    unsigned long long* next_item)
{
    __shared__ __align__(128) RecS tile[2][kTileSteps];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ long long s_next;
    __shared__ float sv[kMixedCells * save_cell(LIN)][kMixedThreads];
    init_staging(bar);
    const long long total = item_off[n_probs];
    unsigned g = 0;
    for (;;) {
        if (threadIdx.x == 0) s_next = (long long)atomicAdd(next_item, 1ull);
        __syncthreads();
        const long long item = s_next;
        if (item >= total) break;
        int lo = 0, hi = n_probs - 1;
        while (lo < hi) {                       // last problem whose first item <= item
            const int mid = (lo + hi + 1) >> 1;
            if (item_off[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const DepositParams P = probs[lo];
        int p, cb, ch;
        item_coords((unsigned)(item - item_off[lo]), P, p, cb, ch);
        if (!deposit_item<FF, LIN, kMixedCells, kMixedCellsPerCta>(P, p, cb, ch, tile, bar, sv, g)) break;
    }
}

cudaError_t launch_deposit_batch(int family, const DepositParams* probs, const long long* item_off, int n_probs,
                                 unsigned long long* next_item, cudaStream_t s)
{
    const int grid = batch_grid(family);
    switch (family) {
    case 0: k_deposit_batch<false, 0><<<grid, kMixedThreads, 0, s>>>(probs, item_off, n_probs, next_item); break;
    case 1: k_deposit_batch<false, 1><<<grid, kMixedThreads, 0, s>>>(probs, item_off, n_probs, next_item); break;
    case 2: k_deposit_batch<false, 2><<<grid, kMixedThreads, 0, s>>>(probs, item_off, n_probs, next_item); break;
    case 4: k_deposit_batch<true, 0><<<grid, kMixedThreads, 0, s>>>(probs, item_off, n_probs, next_item); break;
    case 5: k_deposit_batch<true, 1><<<grid, kMixedThreads, 0, s>>>(probs, item_off, n_probs, next_item); break;
    case 6: k_deposit_batch<true, 2><<<grid, kMixedThreads, 0, s>>>(probs, item_off, n_probs, next_item); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <bool FF, int LIN>
static int resident_batch_ctas()
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deposit_batch<FF, LIN>, kMixedThreads, 0);
    return std::max(1, per_sm);
}

int batch_grid(int family)
{
    int per_sm = 1;
    switch (family) {
    case 0: per_sm = resident_batch_ctas<false, 0>(); break;
    case 1: per_sm = resident_batch_ctas<false, 1>(); break;
    case 2: per_sm = resident_batch_ctas<false, 2>(); break;
    case 4: per_sm = resident_batch_ctas<true, 0>(); break;
    case 5: per_sm = resident_batch_ctas<true, 1>(); break;
    case 6: per_sm = resident_batch_ctas<true, 2>(); break;
    default: break;
    }
    return sm_count() * per_sm;
}

#ifndef RD_CARVEOUT
#define RD_CARVEOUT 0
#endif

template <bool FF, int LIN, int NC, int CPC>
static void launch_mixed(const DepositParams& p, unsigned blocks, cudaStream_t s)
{
    if (RD_CARVEOUT) {
        // the largest shared-memory carveout, so that shared memory does not cap the resident CTAs
        static bool done = false;
        if (!done) {
            cudaFuncSetAttribute(k_deposit_mixed<FF, LIN, NC, CPC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
            done = true;
        }
    }
    k_deposit_mixed<FF, LIN, NC, CPC><<<blocks, CPC / NC, 0, s>>>(p);
}

bool mixed_shape_supported(int cells_per_cta, int cells_per_thread)
{
    return (cells_per_cta == 64 || cells_per_cta == 128 || cells_per_cta == 256) &&
           (cells_per_thread == 1 || cells_per_thread == 2);
}

cudaError_t launch_deposit_mixed(const DepositParams& p, cudaStream_t s)
{
    const long long blocks = (long long)p.n_cell_blocks * p.n_part * p.n_chunks;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const unsigned b = (unsigned)blocks;
    if (p.ff || p.lin) {
        // the far-field and interpolation variants run in the default shape only
        if (p.cpc != kMixedCellsPerCta || p.nc != kMixedCells) return cudaErrorInvalidValue;
        const int lm = p.lin == 3 ? 2 : p.lin ? 1 : 0;       // walk: held, linear family, quadratic
        if (p.ff) {
            if (lm == 2) launch_mixed<true, 2, kMixedCells, kMixedCellsPerCta>(p, b, s);
            else if (lm == 1) launch_mixed<true, 1, kMixedCells, kMixedCellsPerCta>(p, b, s);
            else launch_mixed<true, 0, kMixedCells, kMixedCellsPerCta>(p, b, s);
        } else {
            if (lm == 2) launch_mixed<false, 2, kMixedCells, kMixedCellsPerCta>(p, b, s);
            else launch_mixed<false, 1, kMixedCells, kMixedCellsPerCta>(p, b, s);
        }
        return cudaGetLastError();
    }
    switch (p.cpc * 8 + p.nc) {
    case 256 * 8 + 2: launch_mixed<false, 0, 2, 256>(p, b, s); break;
    case 128 * 8 + 2: launch_mixed<false, 0, 2, 128>(p, b, s); break;
    case 64 * 8 + 2: launch_mixed<false, 0, 2, 64>(p, b, s); break;
    case 256 * 8 + 1: launch_mixed<false, 0, 1, 256>(p, b, s); break;
    case 128 * 8 + 1: launch_mixed<false, 0, 1, 128>(p, b, s); break;
    case 64 * 8 + 1: launch_mixed<false, 0, 1, 64>(p, b, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rd
