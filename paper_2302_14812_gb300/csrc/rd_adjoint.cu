// Adjoint (gather) of the mixed-precision deposit: d loss / d x and d loss / d beta for every
// trajectory sample, given the upstream gradient g = d loss / d (E_det, B_det).
//
// The deposit adds F_k * w_b(u_{k-1}, u_k) to bin b, with F_k = (E, B) of Eq. 1 at sample k and
// w_b = |[u_{k-1}, u_k] ∩ [b, b+1)| in bin units (Section 3.2).  Its transpose, per (cell, interval):
//   G_k = sum_b w_b g_b                      gathered seed, drives the VJP of Eq. 1
//   d loss / d u_k     += F_k . g(bin(u_k))       (end point of interval k)
//   d loss / d u_{k-1} -= F_k . g(bin(u_{k-1}))   (start point), with du/dR = 1/dt_det
// and beta_k, betadot_k = (beta_k - beta_{k-1})/dt, n_k, R_k carry the chain to x_k and beta.
// The walk over bins, arrival times and anchors is the forward walk (same records, same FP32
// increments anchored in FP64), so the gradient is that of the computed deposit.  Field math in
// FP32; per step the cells of a CTA (one per thread) are summed (a reduce-scatter over each warp,
// then shared memory) and the sums are added to FP64 buffers once per 64-step tile.
#include <math.h>

#include "rd_internal.cuh"

namespace rd {

namespace {

// Bin of a stopped cell: far below any window (and far enough from int32 limits for b_end - b).
constexpr int kParkedBin = -(1 << 29);

struct ACell {
    float Px, Py, Pz;
    float f;            // time spent in bin b, units of dt
    float Rpd;          // R_{k-1} + dt
    int b;              // current bin
    int bx;             // bin of the previous arrival time for its end-point term (b unless corrected)
    float g[6];         // seed of bin b (zero outside the window)
    float np[3];        // n of the previous sample
    float pend[6];      // partial gradient of the previous sample: d/dx (3), d/dbeta (3)
    const float* row;   // seed row [n_bins][8]
};

__device__ __forceinline__ void load_seed(const float* row, int n_bins, int b, float* g)
{
    if ((unsigned)b < (unsigned)n_bins) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(row + (size_t)b * 8));
        const float4 c = __ldg(reinterpret_cast<const float4*>(row + (size_t)b * 8 + 4));
        g[0] = a.x;
        g[1] = a.y;
        g[2] = a.z;
        g[3] = a.w;
        g[4] = c.x;
        g[5] = c.y;
    } else {
#pragma unroll
        for (int i = 0; i < 6; ++i) g[i] = 0.f;
    }
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums of six per-lane values over the warp by reduce-scatter (values padded to eight): at each
// of the first three butterfly stages a lane keeps half of its values and sends the other half,
// so 7 + 2 shuffles replace 6 x 5.  Returns, on every lane, the warp sum of value (lane >> 2) & 7
// (values 6 and 7 are zero).
__device__ __forceinline__ float warp_sum6(const float* v, int lane)
{
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
    float a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float lo = v[i], hi = i + 4 < 6 ? v[i + 4] : 0.f;
        const float keep = h4 ? hi : lo, send = h4 ? lo : hi;
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float b[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float keep = h3 ? a[i + 2] : a[i], send = h3 ? a[i] : a[i + 2];
        b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float c = (h2 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, h2 ? b[0] : b[1], 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// Sums over the warp's lanes of the outputs of ns <= kSub steps, staged as [step][value][lane]:
// lane r < 6 ns sums row r (step r / 6, value r % 6; `row` points at it) into dst[r]
// (= red[warp][first step][0] + r).  Each lane reads its row as eight 16-byte chunks starting at a
// lane-dependent chunk, so that the lanes of one load spread over all banks.
constexpr int kSub = 4;

__device__ __forceinline__ void sum_rows(const float4* row, int ns, int lane, float* dst)
{
    if (lane < 6 * ns) {
        float4 a = row[lane & 7];
#pragma unroll
        for (int q = 1; q < 8; ++q) {
            const float4 b = row[(q + lane) & 7];
            a.x += b.x;
            a.y += b.y;
            a.z += b.z;
            a.w += b.w;
        }
        dst[lane] = (a.x + a.y) + (a.z + a.w);
    }
}

// One interval k of one cell: forward field, gathered seed, VJP.  Returns in `out` the finished
// gradient of sample k-1 (d/dx, d/dbeta) and keeps sample k's partial in c.pend.
// EXACT = false (fast walk): an interval that passes two or more bin edges is not handled; the cell
// is stopped instead (stop = true; it outputs zeros until the tile is walked again with EXACT = true
// from its saved start).
// Bin of sample k's arrival time at cell `cell`, from Eq. 2 in FP64 (the walk's FP32 position can
// be off by ~1e-5 bin; near a bin edge that decides the bin of the end-point terms).
__device__ __forceinline__ int exact_bin(const AdjointParams& P, const double* xp, int cell, int k)
{
    const D4 cl = P.cells[cell];
    const double* xk = xp + 3 * (size_t)k;
    double R;
    return clamp_bin(floor(arrival_bins(xk[0], xk[1], xk[2], cl, P.t0, k, P.dt, P.inv_dt_det, R)));
}

__device__ __forceinline__ float dot6(float Ex, float Ey, float Ez, float Bx, float By, float Bz, const float* g)
{
    return Ex * g[0] + Ey * g[1] + Ez * g[2] + Bx * g[3] + By * g[4] + Bz * g[5];
}

template <bool LAST, bool EXACT>
__device__ __forceinline__ void adj_step(ACell& c, const RecS& r, const AdjointParams& P, float q,
                                         float near, float far, int b_end, float f_end, float* out, bool& stop,
                                         const double* xp, int cell, int k)
{
    const float W = P.W;
    // ---- forward: geometry, arrival increment, Eq. 1 ----
    const float dx = c.Px + r.nx, dy = c.Py + r.ny, dz = c.Pz + r.nz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float rinv = fast_rsqrt(r2);
    const float nx = dx * rinv, ny = dy * rinv, nz = dz * rinv;
    const float bx = nx + r.nbx, by = ny + r.nby, bz = nz + r.nbz;          // n - beta
    const float nb2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
    const float gg = fmaf(bx, r.d2x, fmaf(by, r.d2y, fmaf(bz, r.d2z, nb2 + r.gd)));
    const float num = fmaf(r.dtg, rinv, gg);
    const float rden = fast_rcp(fmaf(c.Rpd, rinv, 1.f));
    c.Rpd = fmaf(r2, rinv, P.dt_f);
    const float kap = fmaf(nb2, 0.5f, -r.nhig2);
    const float ik = fast_rcp(kap);
    const float s = q * rinv * (ik * ik * ik);
    const float bdx = r.bdx, bdy = r.bdy, bdz = r.bdz;
    const float dbd = fmaf(nx, bdx, fmaf(ny, bdy, nz * bdz));
    const float c1 = fmaf(r.ig2n, rinv, dbd);                               // gamma^-2/R + n.betadot
    const float Vx = fmaf(bx, c1, -kap * bdx), Vy = fmaf(by, c1, -kap * bdy), Vz = fmaf(bz, c1, -kap * bdz);
    const float Ex = s * Vx, Ey = s * Vy, Ez = s * Vz;
    const float Bx = fmaf(ny, Ez, -nz * Ey), By = fmaf(nz, Ex, -nx * Ez), Bz = fmaf(nx, Ey, -ny * Ex);

    // ---- transpose of the integrating deposit: gathered seed and end-point seeds ----
    // F_k . g(bin(u_{k-1})): the seed of the bin the interval starts in
    const float a_walk = dot6(Ex, Ey, Ez, Bx, By, Bz, c.g);
    float a_beg = a_walk;
    if (c.bx != c.b) {
        float t[6];
        load_seed(c.row, P.n_bins, c.bx, t);
        a_beg = dot6(Ex, Ey, Ez, Bx, By, Bz, t);
    }
    float a_end = a_walk;
    const float fn = LAST ? fmaf((float)(b_end - c.b), W, f_end) : fmaf(num, rden, c.f);
    // the part of the interval inside bin b, then (on a crossing) the rest in the next bin(s)
    const float w1 = (fminf(fn, W) - c.f) * P.du_scale;
    float G[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) G[i] = c.g[i] * w1;
    if (fn < W) {
        c.f = fn;
    } else {
        float rem = fn - W;
        c.b += 1;
        if (!EXACT && rem >= W) {
            // stop the cell for the rest of the tile: with its seeds and pending partials zero and its
            // bin parked far below the window (seed loads there return zero), every output it makes
            // from this step on is exactly zero
            stop = true;
            c.b = kParkedBin;
            rem = 0.f;
            a_beg = 0.f;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                G[i] = 0.f;
                c.pend[i] = 0.f;
            }
        }
        if (EXACT && rem >= W) {
            // whole bins inside the interval (bounded by the window)
            const float nf = floorf(rem * P.invW);
            const int nfull = (int)fminf(nf, 16777216.f);
            const int lo = max(c.b, 0), hi = min(c.b + nfull - 1, P.n_bins - 1);
            const float wf = W * P.du_scale;
            float tmp[6];
            for (int j = lo; j <= hi; ++j) {
                load_seed(c.row, P.n_bins, j, tmp);
#pragma unroll
                for (int i = 0; i < 6; ++i) G[i] = fmaf(tmp[i], wf, G[i]);
            }
            c.b += nfull;
            rem = fminf(fmaxf(fmaf(-nf, W, rem), 0.f), W * 0.99999994f);
        }
        load_seed(c.row, P.n_bins, c.b, c.g);
        const float w2 = rem * P.du_scale;
#pragma unroll
        for (int i = 0; i < 6; ++i) G[i] = fmaf(c.g[i], w2, G[i]);
        c.f = rem;
        // F_k . g(bin(u_k))
        a_end = dot6(Ex, Ey, Ez, Bx, By, Bz, c.g);
    }
    // the end-point terms take the bin of the exact arrival time: rarely another one than the walk's,
    // and only where the walk ends within P.edge_tol of a bin edge (not for stopped or inert cells)
    int b_arr = c.b;
    if (!LAST && c.b > kParkedBin / 2 && ((c.f >= 0.f && c.f < P.edge_tol) || c.f > W - P.edge_tol)) {
        b_arr = exact_bin(P, xp, cell, k);
        if (b_arr != c.b) {
            float t[6];
            load_seed(c.row, P.n_bins, b_arr, t);
            a_end = dot6(Ex, Ey, Ez, Bx, By, Bz, t);
        }
    }
    c.bx = b_arr;

    // ---- VJP of Eq. 1 with B = n x E, seed (GE, GB) = G ----
    const float GEx = G[0], GEy = G[1], GEz = G[2], GBx = G[3], GBy = G[4], GBz = G[5];
    // L = E.H + n.(E x GB),  H = GE + GB x n
    const float Hx = fmaf(GBy, nz, fmaf(-GBz, ny, GEx));
    const float Hy = fmaf(GBz, nx, fmaf(-GBx, nz, GEy));
    const float Hz = fmaf(GBx, ny, fmaf(-GBy, nx, GEz));
    float gnx = fmaf(Ey, GBz, -Ez * GBy), gny = fmaf(Ez, GBx, -Ex * GBz), gnz = fmaf(Ex, GBy, -Ey * GBx);
    const float gsv = fmaf(Vx, Hx, fmaf(Vy, Hy, Vz * Hz));         // d/ds
    const float gVx = s * Hx, gVy = s * Hy, gVz = s * Hz;          // d/dV
    const float gc1 = fmaf(bx, gVx, fmaf(by, gVy, bz * gVz));      // d/dc1
    const float gss = gsv * s;
    // d/dkappa, with ds/dkappa = -3 s / kappa
    const float gk = -fmaf(bdx, gVx, fmaf(bdy, gVy, fmaf(bdz, gVz, 3.f * gss * ik)));
    // V = (n - beta) c1 - kappa betadot;  c1 = gamma^-2/R + n.betadot;  kappa = 1 - n.beta
    const float betx = -r.nbx, bety = -r.nby, betz = -r.nbz;
    gnx = fmaf(c1, gVx, fmaf(gc1, bdx, fmaf(-gk, betx, gnx)));
    gny = fmaf(c1, gVy, fmaf(gc1, bdy, fmaf(-gk, bety, gny)));
    gnz = fmaf(c1, gVz, fmaf(gc1, bdz, fmaf(-gk, betz, gnz)));
    const float g2 = -2.f * (gc1 * rinv * near);                  // d/d(gamma^-2) x (-2), gamma^-2 = 1 - beta^2
    const float gbetx = fmaf(-c1, gVx, fmaf(-gk, nx, g2 * betx));
    const float gbety = fmaf(-c1, gVy, fmaf(-gk, ny, g2 * bety));
    const float gbetz = fmaf(-c1, gVz, fmaf(-gk, nz, g2 * betz));
    const float kf = kap * far, gcf = gc1 * far;                   // d/dbetadot
    const float gbdx = fmaf(gcf, nx, -kf * gVx), gbdy = fmaf(gcf, ny, -kf * gVy), gbdz = fmaf(gcf, nz, -kf * gVz);
    // R: s = q/(kappa^3 R), c1 contains gamma^-2/R, and the arrival time u_k contains R/dt_det
    const float gR = fmaf(a_end, P.inv_dt_det_f, -(fmaf(gc1 * r.ig2n, rinv, gss) * rinv));
    // d = x_cell - x:  n = d/R, dn/dd = (I - n n^T)/R, dR/dd = n, so
    //   d/dd = gn/R + n (gR - n.gn/R)
    const float ndg = fmaf(nx, gnx, fmaf(ny, gny, nz * gnz));
    const float tn = fmaf(-ndg, rinv, gR);
    const float gdx = fmaf(gnx, rinv, nx * tn);
    const float gdy = fmaf(gny, rinv, ny * tn);
    const float gdz = fmaf(gnz, rinv, nz * tn);
    const float inv_dt = P.inv_dt_f;

    // sample k-1: its arrival time starts this interval; betadot_k depends on beta_{k-1}
    const float cb = a_beg * P.inv_dt_det_f;                        // -dL/dR_{k-1} from this interval
    out[0] = c.pend[0] + cb * c.np[0];
    out[1] = c.pend[1] + cb * c.np[1];
    out[2] = c.pend[2] + cb * c.np[2];
    out[3] = c.pend[3] - gbdx * inv_dt;
    out[4] = c.pend[4] - gbdy * inv_dt;
    out[5] = c.pend[5] - gbdz * inv_dt;
    // sample k (partial until the next interval adds its terms)
    c.pend[0] = -gdx;
    c.pend[1] = -gdy;
    c.pend[2] = -gdz;
    c.pend[3] = gbetx + gbdx * inv_dt;
    c.pend[4] = gbety + gbdy * inv_dt;
    c.pend[5] = gbetz + gbdz * inv_dt;
    c.np[0] = nx;
    c.np[1] = ny;
    c.np[2] = nz;
}


constexpr int NA = kAdjointCells;
constexpr int kSaveWords = 19;             // f, Rpd, b, g[6], pend[6], np[3], bx

__device__ __forceinline__ void save_cell(const ACell& c, float (*sv)[kAdjointThreads], int tid)
{
    sv[0][tid] = c.f;
    sv[1][tid] = c.Rpd;
    sv[2][tid] = __int_as_float(c.b);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        sv[3 + i][tid] = c.g[i];
        sv[9 + i][tid] = c.pend[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) sv[15 + i][tid] = c.np[i];
    sv[18][tid] = __int_as_float(c.bx);
}

__device__ __forceinline__ void restore_cell(ACell& c, float (*sv)[kAdjointThreads], int tid)
{
    c.f = sv[0][tid];
    c.Rpd = sv[1][tid];
    c.b = __float_as_int(sv[2][tid]);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        c.g[i] = sv[3 + i][tid];
        c.pend[i] = sv[9 + i][tid];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) c.np[i] = sv[15 + i][tid];
    c.bx = __float_as_int(sv[18][tid]);
}

}  // namespace

// One CTA = (step chunk, block of kAdjointThreads x NA cells, particle); thread tid walks cells
// tid + j kAdjointThreads of the block (j < NA), whose outputs it adds before the warp sum.
__global__ void __launch_bounds__(kAdjointThreads, RD_ADJ_MINBLOCKS) k_adjoint_mixed(const AdjointParams P)
{
    __shared__ __align__(128) RecS tile[2][kTileSteps];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float red[kAdjointThreads / 32][kTileSteps][6];
    __shared__ __align__(16) float stage[kAdjointThreads / 32][kSub][6][32];
    __shared__ float sv[NA][kSaveWords][kAdjointThreads];

    const unsigned bid = blockIdx.x;
    const int p = (int)(bid % (unsigned)P.n_part);
    const unsigned rest = bid / (unsigned)P.n_part;
    const int cb = (int)(rest % (unsigned)P.n_cell_blocks);
    const int ch = (int)(rest / (unsigned)P.n_cell_blocks);
    const int S = P.n_samples - 1;
    const int k_begin = 1 + ch * P.chunk;
    const int k_end = min(S, k_begin + P.chunk - 1);
    const int n_int = k_end - k_begin + 1;
    const int n_tiles = (n_int + kTileSteps - 1) / kTileSteps;
    const RecS* rec = P.rec + (size_t)p * P.n_samples;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int t = 0; t < 2 && t < n_tiles; ++t) {
            const int k0 = k_begin + t * kTileSteps;
            const unsigned bytes = (unsigned)min(kTileSteps, k_end - k0 + 1) * sizeof(RecS);
            mbar_arrive_expect_tx(&bar[t], bytes);
            bulk_g2s(tile[t], rec + k0, bytes, &bar[t]);
        }
    }

    const float q = P.q ? (float)P.q[p] : 1.f;
    const float near = (P.flags & RD_NEAR) ? 1.f : 0.f, far = (P.flags & RD_FAR) ? 1.f : 0.f;
    const double* xp = P.x + (size_t)p * P.n_samples * 3;
    ACell c[NA];
    int b_end[NA];
    float f_end[NA];
    int cells[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        // a cell with no arrival in the window (or past the last cell) walks the same steps from a
        // time that never reaches a bin edge, with zero seeds and partials: all its outputs are
        // exactly zero, and the step needs no per-cell branch
        c[j].b = 0;
        c[j].f = -1e30f;
        b_end[j] = 0;
        f_end[j] = -1e30f;
        c[j].Rpd = 1e6f;
        c[j].Px = 1e6f;
        c[j].Py = c[j].Pz = 0.f;
        c[j].row = P.seed;
#pragma unroll
        for (int i = 0; i < 6; ++i) c[j].pend[i] = c[j].g[i] = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) c[j].np[i] = 0.f;
        const int cell = cb * kAdjointCellsPerCta + j * kAdjointThreads + tid;
        cells[j] = cell;
        if (cell < P.n_pix) {
            const D4 cl = P.cells[cell];
            const double* xa = xp + 3 * (size_t)(k_begin - 1);
            const double* xe = xp + 3 * (size_t)k_end;
            double Ra, Re;
            const double ua = arrival_bins(xa[0], xa[1], xa[2], cl, P.t0, k_begin - 1, P.dt, P.inv_dt_det, Ra);
            const double ue = arrival_bins(xe[0], xe[1], xe[2], cl, P.t0, k_end, P.dt, P.inv_dt_det, Re);
            if ((ue > 0.0) && (ua < (double)P.n_bins)) {
                const double fa = floor(ua), fe = floor(ue);
                c[j].b = clamp_bin(fa);
                c[j].f = (float)(ua - fa) * P.W;
                b_end[j] = clamp_bin(fe);
                f_end[j] = (float)(ue - fe) * P.W;
                c[j].Rpd = (float)Ra + P.dt_f;
                c[j].Px = (float)cl.x;
                c[j].Py = (float)cl.y;
                c[j].Pz = (float)cl.z;
                c[j].row = P.seed + (size_t)cell * P.n_bins * 8;
                load_seed(c[j].row, P.n_bins, c[j].b, c[j].g);
                c[j].np[0] = (float)((cl.x - xa[0]) / Ra);
                c[j].np[1] = (float)((cl.y - xa[1]) / Ra);
                c[j].np[2] = (float)((cl.z - xa[2]) / Ra);
            }
        }
        c[j].bx = c[j].b;
    }

    float* const my_stage = &stage[warp][0][0][lane];                     // + (step * 6 + value) * 32
    const float4* const my_row = reinterpret_cast<const float4*>(&stage[warp][0][0][0]) + 8 * lane;
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
        const int k0 = k_begin + t * kTileSteps;
        const int cnt = min(kTileSteps, k_end - k0 + 1);
        const bool last_tile = (t == n_tiles - 1);
        // walk state at the tile start: the exact walk restarts from it
        int kstop[NA];                                // step at which the fast walk stopped each cell
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            save_cell(c[j], sv[j], tid);
            kstop[j] = cnt;
        }
        for (int i = 0; i < cnt; ++i) {
            float out[6];
            const RecS& r = tile[buf][i];
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                bool st = false;
                float o[6];
                if (last_tile && i == cnt - 1)
                    adj_step<true, false>(c[j], r, P, q, near, far, b_end[j], f_end[j], o, st, xp, cells[j], k0 + i);
                else
                    adj_step<false, false>(c[j], r, P, q, near, far, 0, 0.f, o, st, xp, cells[j], k0 + i);
                kstop[j] = (st && kstop[j] == cnt) ? i : kstop[j];
#pragma unroll
                for (int e = 0; e < 6; ++e) out[e] = j == 0 ? o[e] : out[e] + o[e];
            }
            // per-lane outputs to the warp's staging rows; every kSub steps (and at the tile's end)
            // the warp sums them into red[warp]
            const int sub = i & (kSub - 1);
#pragma unroll
            for (int e = 0; e < 6; ++e) my_stage[(sub * 6 + e) * 32] = out[e];
            if (sub == kSub - 1 || i == cnt - 1) {
                __syncwarp();
                sum_rows(my_row, sub + 1, lane, &red[warp][i - sub][0]);
                __syncwarp();
            }
        }
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            if (!__any_sync(0xffffffffu, kstop[j] < cnt)) continue;
            // some interval of this warp passed two or more bin edges: walk the tile again exactly and
            // add the stopped cells' outputs from their stopping step on
            restore_cell(c[j], sv[j], tid);
#pragma unroll 1
            for (int i = 0; i < cnt; ++i) {
                float out[6];
                bool st = false;
                if (last_tile && i == cnt - 1)
                    adj_step<true, true>(c[j], tile[buf][i], P, q, near, far, b_end[j], f_end[j], out, st, xp,
                                         cells[j], k0 + i);
                else
                    adj_step<false, true>(c[j], tile[buf][i], P, q, near, far, 0, 0.f, out, st, xp, cells[j],
                                          k0 + i);
#pragma unroll
                for (int e = 0; e < 6; ++e) out[e] = i >= kstop[j] ? out[e] : 0.f;
                const float v = warp_sum6(out, lane);
                const int e = lane >> 2;
                if ((lane & 3) == 0 && e < 6) red[warp][i][e] += v;
            }
        }
        __syncthreads();
        // sample k0 - 1 + i gets the sum over the CTA's warps
        for (int e = tid; e < cnt * 6; e += kAdjointThreads) {
            const int i = e / 6, j = e - 6 * (e / 6);
            float v = 0.f;
#pragma unroll
            for (int w = 0; w < kAdjointThreads / 32; ++w) v += red[w][i][j];
            if (v != 0.f) {
                const size_t o = ((size_t)p * P.n_samples + (size_t)(k0 - 1 + i)) * 3;
                if (j < 3) atomicAdd(P.gx + o + j, (double)v);
                else atomicAdd(P.gbeta + o + (j - 3), (double)v);
            }
        }
        __syncthreads();
        if (tid == 0 && t + 2 < n_tiles) {
            fence_proxy_async();
            const int k2 = k_begin + (t + 2) * kTileSteps;
            const unsigned bytes = (unsigned)min(kTileSteps, k_end - k2 + 1) * sizeof(RecS);
            mbar_arrive_expect_tx(&bar[buf], bytes);
            bulk_g2s(tile[buf], rec + k2, bytes, &bar[buf]);
        }
    }
    // the chunk's last sample keeps the partial of its last interval
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        float pv = 0.f;
#pragma unroll
        for (int j = 0; j < NA; ++j) pv += c[j].pend[e];
        const float v = warp_sum(pv);
        if (lane == 0 && v != 0.f) {
            const size_t o = ((size_t)p * P.n_samples + (size_t)k_end) * 3;
            if (e < 3) atomicAdd(P.gx + o + e, (double)v);
            else atomicAdd(P.gbeta + o + (e - 3), (double)v);
        }
    }
}

// =============================================================================================
// Plain FP64 adjoint: the transpose of the plain FP64 deposit (arrival time from Eq. 2 for every
// sample, Eq. 1 in FP64, every bin of an interval gathered in one pass).  Per (cell, interval k):
//   G_k = sum_b w_b g_b over the bins b of [u_{k-1}, u_k] (w_b = overlap in bins)
//   d loss / d u_k += F_k . g(bin(u_k)),  d loss / d u_{k-1} -= F_k . g(bin(u_{k-1})),  du/dR = 1/dt_det
// and the vector-Jacobian product of
//   E = s V,  s = q / (kappa^3 R),  V = (n - beta) c1 - kappa betadot,  c1 = gamma^-2 / R + n.betadot,
//   B = n x E,  kappa = 1 - n.beta,  n = d / R,  d = x_cell - x_k,  gamma^-2 = 1 - beta^2,
//   betadot_k = (beta_k - beta_{k-1}) / dt
// with seed (G_E, G_B) = G_k.  The same algebra as the mixed kernel, all in FP64.
// =============================================================================================
namespace {

struct A64Cell {
    double u;           // arrival (bins) of the previous sample
    int b;              // its bin
    double g[6];        // seed of bin b (zero outside the window)
    double np[3];       // n of the previous sample
    double pend[6];     // partial gradient of the previous sample: d/dx (3), d/dbeta (3)
};

__device__ __forceinline__ void load_seed64(const double* row, int n_bins, int b, double* g)
{
    if ((unsigned)b < (unsigned)n_bins) {
#pragma unroll
        for (int i = 0; i < 6; ++i) g[i] = row[(size_t)b * 6 + i];
    } else {
#pragma unroll
        for (int i = 0; i < 6; ++i) g[i] = 0.0;
    }
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One interval k of one cell; returns in out the finished gradient of sample k-1.
__device__ __forceinline__ void adj64_step(A64Cell& c, const RecD& r, const D4& cl, const double* row,
                                           const AdjointParams& P, int k, double q, double near, double far,
                                           double* out)
{
    // ---- forward: arrival time (Eq. 2) and Eq. 1 ----
    double R;
    const double u = arrival_bins(r.xa.x, r.xa.y, r.xa.z, cl, P.t0, k, P.dt, P.inv_dt_det, R);
    const double dx = cl.x - r.xa.x, dy = cl.y - r.xa.y, dz = cl.z - r.xa.z;
    const double betx = r.bb.x, bety = r.bb.y, betz = r.bb.z;
    const double g2m = near * r.bb.w;                                   // gamma^-2 (velocity term)
    const double bdx = far * r.bd.x, bdy = far * r.bd.y, bdz = far * r.bd.z;   // betadot (acceleration term)
    const double kR = R - (betx * dx + bety * dy + betz * dz);          // kappa R
    const double inv = 1.0 / (R * kR);
    const double rinv = kR * inv;
    const double ik = (R * R) * inv;                                    // 1 / kappa
    const double kap = kR * rinv;
    const double nx = dx * rinv, ny = dy * rinv, nz = dz * rinv;
    const double bx = nx - betx, by = ny - bety, bz = nz - betz;
    const double c1 = g2m * rinv + (nx * bdx + ny * bdy + nz * bdz);
    const double s = q * (ik * ik * ik) * rinv;
    const double Vx = bx * c1 - kap * bdx, Vy = by * c1 - kap * bdy, Vz = bz * c1 - kap * bdz;
    const double Ex = s * Vx, Ey = s * Vy, Ez = s * Vz;
    const double Bx = ny * Ez - nz * Ey, By = nz * Ex - nx * Ez, Bz = nx * Ey - ny * Ex;

    // ---- transpose of the integrating deposit ----
    const double a_beg = Ex * c.g[0] + Ey * c.g[1] + Ez * c.g[2] + Bx * c.g[3] + By * c.g[4] + Bz * c.g[5];
    const int b1 = clamp_bin(floor(u));
    double G[6];
    if (b1 <= c.b) {
        const double w = u - c.u;
#pragma unroll
        for (int i = 0; i < 6; ++i) G[i] = c.g[i] * w;
    } else {
        const double w0 = (double)(c.b + 1) - c.u;
#pragma unroll
        for (int i = 0; i < 6; ++i) G[i] = c.g[i] * w0;
        // whole bins strictly inside the interval, bounded by the window
        const int lo = max(c.b + 1, 0), hi = min(b1 - 1, P.n_bins - 1);
        for (int b = lo; b <= hi; ++b) {
            double t[6];
            load_seed64(row, P.n_bins, b, t);
#pragma unroll
            for (int i = 0; i < 6; ++i) G[i] += t[i];
        }
        load_seed64(row, P.n_bins, b1, c.g);
        const double w1 = u - (double)b1;
#pragma unroll
        for (int i = 0; i < 6; ++i) G[i] += c.g[i] * w1;
        c.b = b1;
    }
    c.u = u;
    const double a_end = Ex * c.g[0] + Ey * c.g[1] + Ez * c.g[2] + Bx * c.g[3] + By * c.g[4] + Bz * c.g[5];

    // ---- VJP of Eq. 1 with B = n x E, seed (GE, GB) = G ----
    const double GEx = G[0], GEy = G[1], GEz = G[2], GBx = G[3], GBy = G[4], GBz = G[5];
    // L = E.H + n.(E x GB),  H = GE + GB x n
    const double Hx = GEx + (GBy * nz - GBz * ny), Hy = GEy + (GBz * nx - GBx * nz), Hz = GEz + (GBx * ny - GBy * nx);
    double gnx = Ey * GBz - Ez * GBy, gny = Ez * GBx - Ex * GBz, gnz = Ex * GBy - Ey * GBx;
    const double gsv = Vx * Hx + Vy * Hy + Vz * Hz;                   // d/ds
    const double gVx = s * Hx, gVy = s * Hy, gVz = s * Hz;            // d/dV
    const double gc1 = bx * gVx + by * gVy + bz * gVz;                // d/dc1
    const double gk = -(bdx * gVx + bdy * gVy + bdz * gVz) - 3.0 * gsv * s * ik;   // d/dkappa
    gnx += c1 * gVx + gc1 * bdx - gk * betx;
    gny += c1 * gVy + gc1 * bdy - gk * bety;
    gnz += c1 * gVz + gc1 * bdz - gk * betz;
    const double gig2 = gc1 * rinv * near;                            // d/d(gamma^-2)
    const double gbetx = -c1 * gVx - gk * nx - 2.0 * gig2 * betx;
    const double gbety = -c1 * gVy - gk * ny - 2.0 * gig2 * bety;
    const double gbetz = -c1 * gVz - gk * nz - 2.0 * gig2 * betz;
    const double gbdx = (gc1 * nx - kap * gVx) * far, gbdy = (gc1 * ny - kap * gVy) * far,
                 gbdz = (gc1 * nz - kap * gVz) * far;                 // d/dbetadot
    // R: s = q/(kappa^3 R), c1 contains gamma^-2/R, the arrival time u_k contains R/dt_det
    const double gR = a_end * P.inv_dt_det - gsv * s * rinv - gc1 * g2m * rinv * rinv;
    // d = x_cell - x: d/dd = gn/R + n (gR - n.gn/R)
    const double ndg = nx * gnx + ny * gny + nz * gnz;
    const double tn = gR - ndg * rinv;
    const double gdx = gnx * rinv + nx * tn, gdy = gny * rinv + ny * tn, gdz = gnz * rinv + nz * tn;
    const double inv_dt = 1.0 / P.dt;

    // sample k-1: its arrival time starts this interval; betadot_k depends on beta_{k-1}
    const double cb = a_beg * P.inv_dt_det;
    out[0] = c.pend[0] + cb * c.np[0];
    out[1] = c.pend[1] + cb * c.np[1];
    out[2] = c.pend[2] + cb * c.np[2];
    out[3] = c.pend[3] - gbdx * inv_dt;
    out[4] = c.pend[4] - gbdy * inv_dt;
    out[5] = c.pend[5] - gbdz * inv_dt;
    // sample k (partial until the next interval adds its terms)
    c.pend[0] = -gdx;
    c.pend[1] = -gdy;
    c.pend[2] = -gdz;
    c.pend[3] = gbetx + gbdx * inv_dt;
    c.pend[4] = gbety + gbdy * inv_dt;
    c.pend[5] = gbetz + gbdz * inv_dt;
    c.np[0] = nx;
    c.np[1] = ny;
    c.np[2] = nz;
}

}  // namespace

// One CTA = (step chunk, block of 128 cells, particle); one cell per thread.  Per step the six
// gradient components are summed over each warp (shuffles), the warps' sums over the CTA per
// tile, and added to the FP64 buffers with atomics.
__global__ void __launch_bounds__(kAdjointFp64Threads) k_adjoint_fp64(const AdjointParams P)
{
    __shared__ __align__(128) RecD tile[2][kTileSteps];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double red[kAdjointFp64Threads / 32][kTileSteps][6];

    const unsigned bid = blockIdx.x;
    const int p = (int)(bid % (unsigned)P.n_part);
    const unsigned rest = bid / (unsigned)P.n_part;
    const int cb = (int)(rest % (unsigned)P.n_cell_blocks);
    const int ch = (int)(rest / (unsigned)P.n_cell_blocks);
    const int S = P.n_samples - 1;
    const int k_begin = 1 + ch * P.chunk;
    const int k_end = min(S, k_begin + P.chunk - 1);
    const int n_int = k_end - k_begin + 1;
    const int n_tiles = (n_int + kTileSteps - 1) / kTileSteps;
    const RecD* rec = P.recd + (size_t)p * P.n_samples;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cell = cb * kAdjointFp64Threads + tid;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int t = 0; t < 2 && t < n_tiles; ++t) {
            const int k0 = k_begin + t * kTileSteps;
            const unsigned bytes = (unsigned)min(kTileSteps, k_end - k0 + 1) * sizeof(RecD);
            mbar_arrive_expect_tx(&bar[t], bytes);
            bulk_g2s(tile[t], rec + k0, bytes, &bar[t]);
        }
    }

    const double q = P.q ? P.q[p] : 1.0;
    const double near = (P.flags & RD_NEAR) ? 1.0 : 0.0, far = (P.flags & RD_FAR) ? 1.0 : 0.0;
    const double* xp = P.x + (size_t)p * P.n_samples * 3;
    A64Cell c;
    D4 cl = {0.0, 0.0, 0.0, 0.0};
    const double* row = P.seedd;
    bool live = false;
#pragma unroll
    for (int i = 0; i < 6; ++i) c.pend[i] = c.g[i] = 0.0;
    c.u = 0.0;
    c.b = 0;
    c.np[0] = c.np[1] = c.np[2] = 0.0;
    if (cell < P.n_pix) {
        cl = P.cells[cell];
        const double* xa = xp + 3 * (size_t)(k_begin - 1);
        const double* xe = xp + 3 * (size_t)k_end;
        double Ra, Re;
        const double ua = arrival_bins(xa[0], xa[1], xa[2], cl, P.t0, k_begin - 1, P.dt, P.inv_dt_det, Ra);
        const double ue = arrival_bins(xe[0], xe[1], xe[2], cl, P.t0, k_end, P.dt, P.inv_dt_det, Re);
        live = (ue > 0.0) && (ua < (double)P.n_bins);
        if (live) {
            row = P.seedd + (size_t)cell * P.n_bins * 6;
            c.u = ua;
            c.b = clamp_bin(floor(ua));
            load_seed64(row, P.n_bins, c.b, c.g);
            c.np[0] = (cl.x - xa[0]) / Ra;
            c.np[1] = (cl.y - xa[1]) / Ra;
            c.np[2] = (cl.z - xa[2]) / Ra;
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
        const int k0 = k_begin + t * kTileSteps;
        const int cnt = min(kTileSteps, k_end - k0 + 1);
        for (int i = 0; i < cnt; ++i) {
            double out[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            if (live) adj64_step(c, tile[buf][i], cl, row, P, k0 + i, q, near, far, out);
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                const double v = warp_sum_d(out[e]);
                if (lane == 0) red[warp][i][e] = v;
            }
        }
        __syncthreads();
        // sample k0 - 1 + i gets the sum over the CTA's warps
        for (int e = tid; e < cnt * 6; e += kAdjointFp64Threads) {
            const int i = e / 6, j = e - 6 * (e / 6);
            double v = 0.0;
#pragma unroll
            for (int w = 0; w < kAdjointFp64Threads / 32; ++w) v += red[w][i][j];
            if (v != 0.0) {
                const size_t o = ((size_t)p * P.n_samples + (size_t)(k0 - 1 + i)) * 3;
                if (j < 3) atomicAdd(P.gx + o + j, v);
                else atomicAdd(P.gbeta + o + (j - 3), v);
            }
        }
        __syncthreads();
        if (tid == 0 && t + 2 < n_tiles) {
            fence_proxy_async();
            const int k2 = k_begin + (t + 2) * kTileSteps;
            const unsigned bytes = (unsigned)min(kTileSteps, k_end - k2 + 1) * sizeof(RecD);
            mbar_arrive_expect_tx(&bar[buf], bytes);
            bulk_g2s(tile[buf], rec + k2, bytes, &bar[buf]);
        }
    }
    // the chunk's last sample keeps the partial of its last interval
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const double v = warp_sum_d(live ? c.pend[e] : 0.0);
        if (lane == 0 && v != 0.0) {
            const size_t o = ((size_t)p * P.n_samples + (size_t)k_end) * 3;
            if (e < 3) atomicAdd(P.gx + o + e, v);
            else atomicAdd(P.gbeta + o + (e - 3), v);
        }
    }
}

// upstream gradient (E, B) [n_pix][n_bins][3] of any type -> [n_pix][n_bins][6] double
template <typename T>
__global__ void k_pack_seed64(const T* __restrict__ gE, const T* __restrict__ gB, long long n, double* __restrict__ seed)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            seed[6 * i + c] = gE ? (double)gE[3 * i + c] : 0.0;
            seed[6 * i + 3 + c] = gB ? (double)gB[3 * i + c] : 0.0;
        }
    }
}

// upstream gradient (E, B) [n_pix][n_bins][3] of any type -> field layout [n_pix][n_bins][8] float
template <typename T>
__global__ void k_pack_seed(const T* __restrict__ gE, const T* __restrict__ gB, long long n, float* __restrict__ seed)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (gE) {
            v[0] = (float)gE[3 * i];
            v[1] = (float)gE[3 * i + 1];
            v[2] = (float)gE[3 * i + 2];
        }
        if (gB) {
            v[3] = (float)gB[3 * i];
            v[4] = (float)gB[3 * i + 1];
            v[5] = (float)gB[3 * i + 2];
        }
        float4* o = reinterpret_cast<float4*>(seed + 8 * i);
        o[0] = make_float4(v[0], v[1], v[2], v[3]);
        o[1] = make_float4(v[4], v[5], 0.f, 0.f);
    }
}

// d loss / d u = (dbeta/du)^T d loss / d beta,  dbeta/du = (I - beta beta^T) / gamma
__global__ void k_gbeta_to_gu(const double* __restrict__ u, const double* __restrict__ gbeta,
                              double* __restrict__ gu, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double ux = u[3 * i], uy = u[3 * i + 1], uz = u[3 * i + 2];
        const double g = sqrt(1.0 + (ux * ux + uy * uy + uz * uz));
        const double bx = ux / g, by = uy / g, bz = uz / g;
        const double gx = gbeta[3 * i], gy = gbeta[3 * i + 1], gz = gbeta[3 * i + 2];
        const double bg = bx * gx + by * gy + bz * gz;
        gu[3 * i] += (gx - bx * bg) / g;
        gu[3 * i + 1] += (gy - by * bg) / g;
        gu[3 * i + 2] += (gz - bz * bg) / g;
    }
}

static int grid_for(long long n, int threads) { return grid_stride_blocks(n, threads, 16); }

cudaError_t launch_pack_seed(const void* gE, const void* gB, int dtype, int n_pix, int n_bins, float* seed,
                             cudaStream_t s)
{
    const long long n = (long long)n_pix * n_bins;
    if (dtype == RD_F32)
        k_pack_seed<float><<<grid_for(n, 256), 256, 0, s>>>(static_cast<const float*>(gE),
                                                          static_cast<const float*>(gB), n, seed);
    else
        k_pack_seed<double><<<grid_for(n, 256), 256, 0, s>>>(static_cast<const double*>(gE),
                                                           static_cast<const double*>(gB), n, seed);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_mixed(const AdjointParams& p, cudaStream_t s)
{
    const long long blocks = (long long)p.n_cell_blocks * p.n_part * p.n_chunks;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_adjoint_mixed<<<(unsigned)blocks, kAdjointThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_pack_seed64(const void* gE, const void* gB, int dtype, int n_pix, int n_bins, double* seed,
                               cudaStream_t s)
{
    const long long n = (long long)n_pix * n_bins;
    if (dtype == RD_F32)
        k_pack_seed64<float><<<grid_for(n, 256), 256, 0, s>>>(static_cast<const float*>(gE),
                                                            static_cast<const float*>(gB), n, seed);
    else
        k_pack_seed64<double><<<grid_for(n, 256), 256, 0, s>>>(static_cast<const double*>(gE),
                                                             static_cast<const double*>(gB), n, seed);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_fp64(const AdjointParams& p, cudaStream_t s)
{
    const long long blocks = (long long)p.n_cell_blocks * p.n_part * p.n_chunks;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_adjoint_fp64<<<(unsigned)blocks, kAdjointFp64Threads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_gbeta_to_gu(const double* u, const double* gbeta, double* gu, long long n, cudaStream_t s)
{
    k_gbeta_to_gu<<<grid_for(n, 256), 256, 0, s>>>(u, gbeta, gu, n);
    return cudaGetLastError();
}

}  // namespace rd
