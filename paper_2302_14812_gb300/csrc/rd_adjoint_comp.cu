// Compensated adjoint of the mixed-precision deposit (RD_ADJ_COMPENSATED): the gradient the FP32
// adjoint computes, carried in double-float wherever a later difference of neighbouring samples
// would magnify FP32 rounding.
//
// Why the FP32 adjoint stops near 1e-5.  Sample j's gradient holds two differences of terms that
// nearly cancel:
//   d L / d x_j  ~  n_j (F_{j+1} - F_j) . g(bin(t'_j)) / dt_det     (its arrival time ends interval
//                                                                    j and starts interval j+1)
//   d L / d beta_j  ~  (d L / d betadot_j - d L / d betadot_{j+1}) / dt   (betadot_k =
//                                                                    (beta_k - beta_{k-1}) / dt)
// F and d L / d betadot change by a few per cent from one sample to the next, so an FP32 evaluation
// of each (a few units of 2^-24) loses that factor in the difference; d L / d u = (I - beta beta^T)
// d L / d beta / gamma then removes the large component along beta and loses another factor gamma.
//
// Here, per (cell, interval k), the field F_k of Eq. 1, the gathered seed G_k = sum_b w_b g_b with
// the bin weights of Section 3.2, the vector-Jacobian product of Eq. 1 up to d L / d beta and
// d L / d betadot, and the projection to d L / d u are evaluated in double-float (rd_df.cuh); the
// arrival-time walk advances by the same all-positive-term increment as the forward path, in
// double-float, from an FP64 arrival time (Eq. 2) at the start of every chunk.  Each difference
// is formed in one thread: a CTA that owns intervals k_begin..k_end outputs samples
// k_begin-1..k_end-1 (and the last sample S), walking interval k_begin-1 once more first, so that
// sample j's two terms meet in the thread that walks interval j+1.  Only the small position
// derivative through the field (n and R at distance R, 1/R times the others) stays in FP32.  Per
// step the 6 outputs of a CTA's cells are summed in double-float (warp butterfly, then shared
// memory), converted to FP64 and added to the gradients once per 64-sample tile.
//
// CTA = (chunk of intervals, block of 128 cells, particle), one cell per thread; records staged in
// shared memory by bulk asynchronous copies (bounded waits, as in the other kernels).
#include <math.h>

#include "rd_df.cuh"
#include "rd_internal.cuh"

#ifndef RD_COMP_MINBLOCKS
#define RD_COMP_MINBLOCKS 2      // resident CTAs per SM the register allotment must allow
#endif

namespace rd {

namespace {

struct V3 {
    df2 x, y, z;
};

__device__ __forceinline__ V3 v_add(const V3& a, const V3& b) { return {df_add(a.x, b.x), df_add(a.y, b.y), df_add(a.z, b.z)}; }
__device__ __forceinline__ V3 v_sub(const V3& a, const V3& b) { return {df_sub(a.x, b.x), df_sub(a.y, b.y), df_sub(a.z, b.z)}; }
__device__ __forceinline__ V3 v_scale(const V3& a, df2 s) { return {df_mul(a.x, s), df_mul(a.y, s), df_mul(a.z, s)}; }
__device__ __forceinline__ df2 v_dot(const V3& a, const V3& b)
{
    return df_fma(a.x, b.x, df_fma(a.y, b.y, df_mul(a.z, b.z)));
}
__device__ __forceinline__ V3 v_cross(const V3& a, const V3& b)
{
    return {df_sub(df_mul(a.y, b.z), df_mul(a.z, b.y)), df_sub(df_mul(a.z, b.x), df_mul(a.x, b.z)),
            df_sub(df_mul(a.x, b.y), df_mul(a.y, b.x))};
}
__device__ __forceinline__ V3 v_neg(const V3& a) { return {df_neg(a.x), df_neg(a.y), df_neg(a.z)}; }
// (I - beta beta^T) v / gamma: d L / d u from d L / d beta (beta = u / sqrt(1 + u^2))
__device__ __forceinline__ V3 project_u(const V3& beta, df2 ig, const V3& v)
{
    const df2 bv = v_dot(beta, v);
    return v_scale(v_sub(v, v_scale(beta, bv)), ig);
}

// Seed rows in double-float: [n_bins][16] floats per cell, (hi of E xyz, B xyz, 2 unused, lo of the
// same, 2 unused); an FP64 upstream gradient keeps ~48 of its bits (FP32 would act on the gradient as
// a noise seed of relative size 2^-24, which the cancellation of neighbouring samples does not damp).
__device__ __forceinline__ void load_seed(const float* row, int n_bins, int b, df2* g)
{
    if ((unsigned)b < (unsigned)n_bins) {
        const float4* q = reinterpret_cast<const float4*>(row + (size_t)b * 16);
        const float4 h0 = __ldg(q), h1 = __ldg(q + 1), l0 = __ldg(q + 2), l1 = __ldg(q + 3);
        g[0] = {h0.x, l0.x};
        g[1] = {h0.y, l0.y};
        g[2] = {h0.z, l0.z};
        g[3] = {h0.w, l0.w};
        g[4] = {h1.x, l1.x};
        g[5] = {h1.y, l1.y};
    } else {
#pragma unroll
        for (int i = 0; i < 6; ++i) g[i] = {0.f, 0.f};
    }
}

// warp sum of a double-float value (butterfly; every lane ends with the sum)
__device__ __forceinline__ df2 warp_sum_df(df2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        df2 w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return v;
}

struct CCell {
    V3 P;           // cell position
    df2 f;          // arrival time of the previous sample within bin b (bin units, [0, 1))
    int b;          // bin of the walk
    int bx;         // bin of the previous sample's arrival for its end-point terms
    df2 Rpd;        // R_{k-1} + dt
    df2 g[6];       // seed of bin b (zero outside the window)
    const float* row;
    // previous sample k-1
    df2 Fp[6];      // field of interval k-1 (E, B); zero for sample 0
    V3 gbdp;        // d L / d betadot_{k-1} from interval k-1
    V3 gbetp;       // d L / d beta_{k-1} through interval k-1's field, betadot term excluded
    V3 bp;          // beta_{k-1}
    df2 igp;        // 1 / gamma_{k-1}
    float np[3];    // n_{k-1}
    float gxf[3];   // d L / d x_{k-1} through interval k-1's field (n and R), arrival terms excluded
};

struct CompConsts {
    df2 du_scale;   // dt / dt_det
    df2 dt;
    df2 inv_dt;
    float inv_dt_det;
    bool near, far;
    float edge_tol; // bins from an edge below which an arrival's bin is taken from Eq. 2 in FP64
};

// Sample j's outputs from its two intervals' terms (j = k-1 when interval k has just been walked,
// or the last sample S with Fk = 0 and gbdk = 0): position, momentum.
// The momentum outputs stay double-float: the sum over cells can cancel far below its terms.
__device__ __forceinline__ void sample_out(const CCell& c, const df2* Fk, const V3& gbdk, const df2* gx_seed,
                                           const CompConsts& K, df2* out)
{
    float dF[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) dF[i] = df_round(df_sub(Fk[i], c.Fp[i]));
    float da = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) da = fmaf(dF[i], df_round(gx_seed[i]), da);
    const float a = da * K.inv_dt_det;
#pragma unroll
    for (int i = 0; i < 3; ++i) out[i] = df_make(fmaf(c.np[i], a, c.gxf[i]));
    const V3 gb = v_add(c.gbetp, v_scale(v_sub(c.gbdp, gbdk), K.inv_dt));
    const V3 gu = project_u(c.bp, c.igp, gb);
    out[3] = gu.x;
    out[4] = gu.y;
    out[5] = gu.z;
}

}  // namespace

// Per-sample records of the compensated adjoint, double-float split of FP64 values:
//   x_k, beta_k, far * betadot_k, gamma_k^-2, 1/gamma_k, dt g_k, 2 (beta_k - vbar_k), g_k + |beta_k - vbar_k|^2
// (vbar_k = (x_k - x_{k-1}) / dt, g_k = 1 - |vbar_k|^2).
struct __align__(16) RecC {
    df2 x[3];
    df2 b[3];
    df2 bd[3];
    df2 ig2;
    df2 ig;
    df2 dtg;
    df2 d2[3];
    df2 gd;
};
static_assert(sizeof(RecC) == 128, "RecC must be 128 bytes");

__global__ void k_precompute_comp(const double* __restrict__ x, const double* __restrict__ u, int n_part,
                                  int n_samples, double dt, int flags, RecC* __restrict__ rec, DevCounters* counters)
{
    const long long total = (long long)n_part * n_samples;
    const bool far_on = (flags & RD_FAR) != 0;
    const double inv_dt = 1.0 / dt;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % n_samples);
        const double* xk = x + 3 * i;
        const double* uk = u + 3 * i;
        bool bad = !(isfinite(xk[0]) && isfinite(xk[1]) && isfinite(xk[2]) && isfinite(uk[0]) && isfinite(uk[1]) &&
                     isfinite(uk[2]));
        const double uu = uk[0] * uk[0] + uk[1] * uk[1] + uk[2] * uk[2];
        const double gam = sqrt(1.0 + uu);
        const double b[3] = {uk[0] / gam, uk[1] / gam, uk[2] / gam};
        double a[3] = {0.0, 0.0, 0.0}, v[3] = {0.0, 0.0, 0.0}, g = 1.0;
        if (k > 0) {
            const double* up = uk - 3;
            const double gp = sqrt(1.0 + (up[0] * up[0] + up[1] * up[1] + up[2] * up[2]));
            for (int c = 0; c < 3; ++c) {
                a[c] = (b[c] - up[c] / gp) * inv_dt;
                v[c] = (xk[c] - xk[c - 3]) * inv_dt;
            }
            g = 1.0 - (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            bad = bad || !(g > 0.0);
        }
        if (bad) atomicOr(&counters->errors, ERRBIT_INPUT);
        RecC r;
        double e2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double e = b[c] - v[c];
            e2 += e * e;
            r.x[c] = df_from_double(xk[c]);
            r.b[c] = df_from_double(b[c]);
            r.bd[c] = df_from_double(far_on ? a[c] : 0.0);
            r.d2[c] = df_from_double(2.0 * e);
        }
        r.ig2 = df_from_double(1.0 / (1.0 + uu));
        r.ig = df_from_double(1.0 / gam);
        r.dtg = df_from_double(dt * g);
        r.gd = df_from_double(g + e2);
        rec[i] = r;
    }
}

namespace {

// One interval k of one cell: field, walk and gather, vector-Jacobian product in double-float.
// out_on: write sample k-1's finished gradient into out (false on the halo interval, whose sample
// belongs to the previous chunk).  LAST: the interval ends on the chunk's FP64 end anchor.
template <bool LAST>
__device__ __forceinline__ void comp_step(CCell& c, const RecC& r, const AdjointParams& P, const CompConsts& K,
                                          df2 q, int b_end, df2 f_end, bool out_on, df2* out, const double* xp,
                                          int cell, int k)
{
    // ---- geometry, arrival increment ----
    const V3 X = {r.x[0], r.x[1], r.x[2]};
    const V3 beta = {r.b[0], r.b[1], r.b[2]};
    const V3 bd = {r.bd[0], r.bd[1], r.bd[2]};
    const V3 d = v_sub(c.P, X);
    const df2 r2 = v_dot(d, d);
    const df2 rinv = df_rsqrt(r2);
    const df2 R = df_mul(r2, rinv);
    const V3 n = v_scale(d, rinv);
    const V3 nb = v_sub(n, beta);
    const df2 nb2 = v_dot(nb, nb);
    // t'_k - t'_{k-1} = dt [dt g + R_k (g + |n_k - vbar|^2)] / (dt + R_k + R_{k-1}), in bins, with
    // g + |n - vbar|^2 = |n - beta|^2 + 2 (n - beta).(beta - vbar) + (g + |beta - vbar|^2)
    const V3 d2 = {r.d2[0], r.d2[1], r.d2[2]};
    const int b_start = c.b;
    df2 fn;
    if (LAST) {
        fn = df_add(df_make((float)(b_end - c.b)), f_end);
    } else {
        const df2 num = df_add(df_fma(r.dtg, rinv, nb2), df_add(v_dot(nb, d2), r.gd));
        const df2 den = df_add_f(df_mul(c.Rpd, rinv), 1.0f);
        fn = df_add(c.f, df_mul(df_mul(num, df_rcp(den)), K.du_scale));
    }
    c.Rpd = df_add(R, K.dt);

    // ---- Eq. 1: E = s V, s = q / (kappa^3 R), V = (n - beta) c1 - kappa betadot, B = n x E ----
    const df2 kap = df_scale2(df_add(r.ig2, nb2), 0.5f);       // 1 - beta.n
    const df2 ik = df_rcp(kap);
    const df2 s = df_mul(df_mul(q, rinv), df_mul(df_mul(ik, ik), ik));
    const df2 ig2n = K.near ? r.ig2 : df_make(0.f);
    const df2 c1 = df_fma(ig2n, rinv, v_dot(n, bd));          // gamma^-2 / R + n.betadot
    const V3 V = v_sub(v_scale(nb, c1), v_scale(bd, kap));
    const V3 E = v_scale(V, s);
    const V3 B = v_cross(n, E);
    const df2 F[6] = {E.x, E.y, E.z, B.x, B.y, B.z};

    // ---- transpose of the integrating deposit: G = sum_b w_b g_b over [u_{k-1}, u_k] ----
    df2 g0[6];                                                // seed of the bin the interval starts in
#pragma unroll
    for (int i = 0; i < 6; ++i) g0[i] = c.g[i];
    df2 G[6];
    if (!df_ge(fn, 1.0f)) {
        const df2 w = df_sub(fn, c.f);
#pragma unroll
        for (int i = 0; i < 6; ++i) G[i] = df_mul(w, c.g[i]);
        c.f = fn;
    } else {
        const df2 w0 = df_sub(df_make(1.0f), c.f);
#pragma unroll
        for (int i = 0; i < 6; ++i) G[i] = df_mul(w0, c.g[i]);
        const int m = min(df_floor(fn), 1 << 24);             // bin edges passed (>= 1)
        // whole bins b+1 .. b+m-1, bounded by the window
        const int lo = max(c.b + 1, 0), hi = min(c.b + m - 1, P.n_bins - 1);
        for (int bb = lo; bb <= hi; ++bb) {
            df2 t[6];
            load_seed(c.row, P.n_bins, bb, t);
#pragma unroll
            for (int i = 0; i < 6; ++i) G[i] = df_add(G[i], t[i]);
        }
        c.b += m;
        load_seed(c.row, P.n_bins, c.b, c.g);
        const df2 rem = df_sub(fn, df_make((float)m));
#pragma unroll
        for (int i = 0; i < 6; ++i) G[i] = df_add(G[i], df_mul(rem, c.g[i]));
        c.f = rem;
    }
    // bin of this arrival for its end-point terms: the walk's, or Eq. 2 in FP64 where the walk ends
    // within edge_tol of a bin edge (the FP64 value decides there, as in the oracle); the end anchor
    // is itself Eq. 2 in FP64
    int barr = c.b;
    if (!LAST && (c.f.hi < K.edge_tol || c.f.hi > 1.0f - K.edge_tol)) {
        const D4 cl = P.cells[cell];
        const double* xk = xp + 3 * (size_t)k;
        double Rk;
        barr = clamp_bin(floor(arrival_bins(xk[0], xk[1], xk[2], cl, P.t0, k, P.dt, P.inv_dt_det, Rk)));
    }

    // ---- vector-Jacobian product of Eq. 1 with seed (GE, GB) = G ----
    const V3 GE = {G[0], G[1], G[2]}, GB = {G[3], G[4], G[5]};
    const V3 H = v_add(GE, v_cross(GB, n));                    // E.GE + (n x E).GB = E.H
    const df2 gsv = v_dot(V, H);                               // d/ds
    const V3 gV = v_scale(H, s);                               // d/dV
    const df2 gc1 = v_dot(nb, gV);                             // d/dc1
    const df2 gss = df_mul(gsv, s);
    // d/dkappa = -(betadot . gV) - 3 s gsv / kappa
    const df2 gk = df_neg(df_fma(df_scale2(gss, 2.0f), ik, df_fma(gss, ik, v_dot(bd, gV))));
    const df2 gig2 = K.near ? df_mul(gc1, rinv) : df_make(0.f);  // d/d(gamma^-2)
    // d/dbeta through V ((n - beta) c1), kappa = 1 - n.beta and gamma^-2 = 1 - beta^2; betadot's part
    // (+-1/dt) is added when the sample's output is formed
    const V3 gbet = v_neg(v_add(v_add(v_scale(gV, c1), v_scale(n, gk)), v_scale(beta, df_scale2(gig2, 2.0f))));
    // d/dbetadot: c1 = ... + n.betadot, V = ... - kappa betadot
    V3 gbd = v_sub(v_scale(n, gc1), v_scale(gV, kap));
    if (!K.far) gbd = {df_make(0.f), df_make(0.f), df_make(0.f)};

    // ---- sample k-1: its two intervals' terms meet here ----
    if (out_on) {
        df2 gs[6];
        if (c.bx == b_start) {
#pragma unroll
            for (int i = 0; i < 6; ++i) gs[i] = g0[i];
        } else {
            load_seed(c.row, P.n_bins, c.bx, gs);
        }
        sample_out(c, F, gbd, gs, K, out);
    }

    // ---- position derivative through the field (n, R): small (1/R), FP32 ----
    const float nx = df_round(n.x), ny = df_round(n.y), nz = df_round(n.z);
    const float fE[3] = {df_round(E.x), df_round(E.y), df_round(E.z)};
    const float fGB[3] = {df_round(GB.x), df_round(GB.y), df_round(GB.z)};
    const float fgV[3] = {df_round(gV.x), df_round(gV.y), df_round(gV.z)};
    const float fc1 = df_round(c1), fgc1 = df_round(gc1), fgk = df_round(gk), frinv = df_round(rinv);
    const float fbd[3] = {df_round(bd.x), df_round(bd.y), df_round(bd.z)};
    const float fb[3] = {df_round(beta.x), df_round(beta.y), df_round(beta.z)};
    float gn[3];
    gn[0] = fE[1] * fGB[2] - fE[2] * fGB[1];                  // d/dn of (n x E).GB = E x GB
    gn[1] = fE[2] * fGB[0] - fE[0] * fGB[2];
    gn[2] = fE[0] * fGB[1] - fE[1] * fGB[0];
#pragma unroll
    for (int i = 0; i < 3; ++i) gn[i] += fc1 * fgV[i] + fgc1 * fbd[i] - fgk * fb[i];
    // R: s = q / (kappa^3 R), c1 holds gamma^-2 / R
    const float gR = -(df_round(gss) + fgc1 * df_round(ig2n) * frinv) * frinv;
    // d = x_cell - x_k: d/dd = gn / R + n (gR - n.gn / R); d/dx_k = -d/dd
    const float ndg = nx * gn[0] + ny * gn[1] + nz * gn[2];
    const float tn = gR - ndg * frinv;
    c.gxf[0] = -(gn[0] * frinv + nx * tn);
    c.gxf[1] = -(gn[1] * frinv + ny * tn);
    c.gxf[2] = -(gn[2] * frinv + nz * tn);

    // ---- this sample becomes the previous one ----
#pragma unroll
    for (int i = 0; i < 6; ++i) c.Fp[i] = F[i];
    c.gbdp = gbd;
    c.gbetp = gbet;
    c.bp = beta;
    c.igp = r.ig;
    c.np[0] = nx;
    c.np[1] = ny;
    c.np[2] = nz;
    c.bx = barr;
}

}  // namespace

// One CTA = (chunk of intervals, block of 128 cells, particle); thread tid owns cell
// cb * 128 + tid.  Outputs samples k_begin-1 .. k_end-1 (and S in the last chunk).
__global__ void __launch_bounds__(kAdjointCompThreads, RD_COMP_MINBLOCKS) k_adjoint_comp(const AdjointParams P)
{
    constexpr int NT = kAdjointCompThreads, NW = NT / 32;
    __shared__ __align__(128) RecC tile[2][kTileSteps];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ df2 red[NW][kTileSteps + 1][6];

    const unsigned bid = blockIdx.x;
    const int p = (int)(bid % (unsigned)P.n_part);
    const unsigned rest = bid / (unsigned)P.n_part;
    const int cb = (int)(rest % (unsigned)P.n_cell_blocks);
    const int ch = (int)(rest / (unsigned)P.n_cell_blocks);
    const int S = P.n_samples - 1;
    const int k_begin = 1 + ch * P.chunk;
    const int k_end = min(S, k_begin + P.chunk - 1);
    const int k_walk = k_begin > 1 ? k_begin - 1 : 1;       // first interval walked (halo before k_begin)
    const int n_walk = k_end - k_walk + 1;
    const int n_tiles = (n_walk + kTileSteps - 1) / kTileSteps;
    const RecC* rec = static_cast<const RecC*>(P.recc) + (size_t)p * P.n_samples;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cell = cb * NT + tid;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int t = 0; t < 2 && t < n_tiles; ++t) {
            const int k0 = k_walk + t * kTileSteps;
            const unsigned bytes = (unsigned)min(kTileSteps, k_end - k0 + 1) * sizeof(RecC);
            mbar_arrive_expect_tx(&bar[t], bytes);
            bulk_g2s(tile[t], rec + k0, bytes, &bar[t]);
        }
    }

    CompConsts K;
    K.du_scale = df_from_double(P.dt * P.inv_dt_det);
    K.dt = df_from_double(P.dt);
    K.inv_dt = df_from_double(1.0 / P.dt);
    K.inv_dt_det = (float)P.inv_dt_det;
    K.near = (P.flags & RD_NEAR) != 0;
    K.far = (P.flags & RD_FAR) != 0;
    K.edge_tol = 1e-6f;
    const df2 q = df_from_double(P.q ? P.q[p] : 1.0);
    const double* xp = P.x + (size_t)p * P.n_samples * 3;

    // state at the arrival of sample k_walk - 1 (FP64 anchor), the end anchor at sample k_end
    CCell c;
    const df2 z = df_make(0.f);
    c.P = {z, z, z};
    c.f = z;
    c.b = 0;
    c.bx = 0;
    c.Rpd = df_make(1.f);
    c.row = P.seed;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        c.g[i] = z;
        c.Fp[i] = z;
    }
    c.gbdp = c.gbetp = c.bp = {z, z, z};
    c.igp = df_make(1.f);
#pragma unroll
    for (int i = 0; i < 3; ++i) c.np[i] = c.gxf[i] = 0.f;
    int b_end = 0;
    df2 f_end = z;
    bool live = false;
    if (cell < P.n_pix) {
        const D4 cl = P.cells[cell];
        const double* xa = xp + 3 * (size_t)(k_walk - 1);
        const double* xe = xp + 3 * (size_t)k_end;
        double Ra, Re;
        const double ua = arrival_bins(xa[0], xa[1], xa[2], cl, P.t0, k_walk - 1, P.dt, P.inv_dt_det, Ra);
        const double ue = arrival_bins(xe[0], xe[1], xe[2], cl, P.t0, k_end, P.dt, P.inv_dt_det, Re);
        live = (ue > 0.0) && (ua < (double)P.n_bins);
        if (live) {
            const double fa = floor(ua), fe = floor(ue);
            c.b = clamp_bin(fa);
            c.bx = c.b;
            c.f = df_from_double(ua - fa);
            b_end = clamp_bin(fe);
            f_end = df_from_double(ue - fe);
            c.Rpd = df_from_double(Ra + P.dt);
            c.P = {df_from_double(cl.x), df_from_double(cl.y), df_from_double(cl.z)};
            c.row = P.seed + (size_t)cell * P.n_bins * 16;
            load_seed(c.row, P.n_bins, c.b, c.g);
            // sample 0 (no halo): its arrival starts interval 1; it has no field of its own
            c.np[0] = (float)((cl.x - xa[0]) / Ra);
            c.np[1] = (float)((cl.y - xa[1]) / Ra);
            c.np[2] = (float)((cl.z - xa[2]) / Ra);
            const RecC r0 = rec[k_walk - 1];
            c.bp = {r0.b[0], r0.b[1], r0.b[2]};
            c.igp = r0.ig;
        }
    }

    for (int t = 0; t < n_tiles; ++t) {
        const int buf = t & 1;
        const bool ok = mbar_wait_bounded(&bar[buf], (unsigned)(t >> 1) & 1u);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(&P.counters->errors, ERRBIT_TIMEOUT);
                for (int u = t; u < t + 2 && u < n_tiles; ++u)
                    (void)mbar_wait_bounded(&bar[u & 1], (unsigned)(u >> 1) & 1u);
            }
            __syncthreads();
            return;
        }
        const int k0 = k_walk + t * kTileSteps;
        const int cnt = min(kTileSteps, k_end - k0 + 1);
        const bool last_tile = (t == n_tiles - 1);
        for (int i = 0; i < cnt; ++i) {
            const int k = k0 + i;
            df2 out[6] = {z, z, z, z, z, z};
            const bool out_on = k >= k_begin;
            if (live) {
                if (last_tile && i == cnt - 1)
                    comp_step<true>(c, tile[buf][i], P, K, q, b_end, f_end, out_on, out, xp, cell, k);
                else
                    comp_step<false>(c, tile[buf][i], P, K, q, 0, z, out_on, out, xp, cell, k);
            }
            if (out_on) {
#pragma unroll
                for (int e = 0; e < 6; ++e) {
                    const df2 v = warp_sum_df(out[e]);
                    if (lane == 0) red[warp][i][e] = v;
                }
            }
        }
        // the last sample of the trajectory: interval S's terms only
        const bool tail = last_tile && k_end == S;
        if (tail) {
            df2 out[6] = {z, z, z, z, z, z};
            if (live) {
                df2 gs[6];
                load_seed(c.row, P.n_bins, c.bx, gs);
                const df2 Fz[6] = {z, z, z, z, z, z};
                const V3 gz = {z, z, z};
                sample_out(c, Fz, gz, gs, K, out);
            }
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                const df2 v = warp_sum_df(out[e]);
                if (lane == 0) red[warp][cnt][e] = v;
            }
        }
        __syncthreads();
        // sample k - 1 of row i (k = k0 + i >= k_begin) and, in the tail row, sample S
        const int rows = cnt + (tail ? 1 : 0);
        for (int e = tid; e < rows * 6; e += NT) {
            const int i = e / 6, j = e - 6 * (e / 6);
            const int sample = i < cnt ? k0 + i - 1 : S;
            if (i < cnt && k0 + i < k_begin) continue;
            df2 v = red[0][i][j];
#pragma unroll
            for (int w = 1; w < NW; ++w) v = df_add(v, red[w][i][j]);
            const double dv = (double)v.hi + (double)v.lo;
            if (dv != 0.0) {
                const size_t o = ((size_t)p * P.n_samples + (size_t)sample) * 3;
                if (j < 3) atomicAdd(P.gx + o + j, dv);
                else atomicAdd(P.gu + o + (j - 3), dv);
            }
        }
        __syncthreads();
        if (tid == 0 && t + 2 < n_tiles) {
            fence_proxy_async();
            const int k2 = k_walk + (t + 2) * kTileSteps;
            const unsigned bytes = (unsigned)min(kTileSteps, k_end - k2 + 1) * sizeof(RecC);
            mbar_arrive_expect_tx(&bar[buf], bytes);
            bulk_g2s(tile[buf], rec + k2, bytes, &bar[buf]);
        }
    }
}

// upstream gradient (E, B) [n_pix][n_bins][3] of any type -> double-float seed rows [n_pix][n_bins][16]
template <typename T>
__global__ void k_pack_seed_df(const T* __restrict__ gE, const T* __restrict__ gB, long long n, float* __restrict__ seed)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float h[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, l[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int c = 0; c < 3; ++c) {
            const df2 e = df_from_double(gE ? (double)gE[3 * i + c] : 0.0);
            const df2 b = df_from_double(gB ? (double)gB[3 * i + c] : 0.0);
            h[c] = e.hi;
            l[c] = e.lo;
            h[3 + c] = b.hi;
            l[3 + c] = b.lo;
        }
        float4* o = reinterpret_cast<float4*>(seed + 16 * i);
        o[0] = make_float4(h[0], h[1], h[2], h[3]);
        o[1] = make_float4(h[4], h[5], 0.f, 0.f);
        o[2] = make_float4(l[0], l[1], l[2], l[3]);
        o[3] = make_float4(l[4], l[5], 0.f, 0.f);
    }
}

size_t comp_record_bytes() { return sizeof(RecC); }

cudaError_t launch_pack_seed_df(const void* gE, const void* gB, int dtype, int n_pix, int n_bins, float* seed,
                                cudaStream_t s)
{
    const long long n = (long long)n_pix * n_bins;
    const int g = grid_stride_blocks(n, 256, 16);
    if (dtype == RD_F32)
        k_pack_seed_df<float><<<g, 256, 0, s>>>(static_cast<const float*>(gE), static_cast<const float*>(gB), n, seed);
    else
        k_pack_seed_df<double><<<g, 256, 0, s>>>(static_cast<const double*>(gE), static_cast<const double*>(gB), n,
                                                 seed);
    return cudaGetLastError();
}

cudaError_t launch_precompute_comp(const double* x, const double* u, int n_part, int n_samples, double dt, int flags,
                                   void* rec, DevCounters* counters, cudaStream_t s)
{
    const long long n = (long long)n_part * n_samples;
    k_precompute_comp<<<grid_stride_blocks(n, 256, 16), 256, 0, s>>>(x, u, n_part, n_samples, dt, flags,
                                                                     static_cast<RecC*>(rec), counters);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_comp(const AdjointParams& p, cudaStream_t s)
{
    const long long blocks = (long long)p.n_cell_blocks * p.n_part * p.n_chunks;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_adjoint_comp<<<(unsigned)blocks, kAdjointCompThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace rd
