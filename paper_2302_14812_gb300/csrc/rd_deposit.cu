// Per-sample precompute (both precisions), the plain FP64 deposit and the field readout and
// write-in (the mixed-precision deposit is in rd_mixed.cu).
//
// Work decomposition of the FP64 deposit: one CTA = 256 detector cells (one per thread) x one
// particle x one chunk of consecutive intervals.  The chunk's per-sample records are streamed
// through shared memory in tiles of 64 samples by bulk asynchronous copies (double buffered,
// mbarrier completion); every thread reads each record as a broadcast.  Each thread evaluates its
// cell's arrival time from Eq. 2 for every sample (they increase for sub-luminal chords), keeps
// the bin it is filling in registers and adds the bin to global memory only when its arrival time
// leaves the bin.  The FP64 pipe is the bound (on GB300 it runs at 1.6 % of the FP32 rate), so in a
// warp whose lanes all walk a cell, the FP64 work of the few lanes that start a new bin is spread
// over the warp by shuffles and the bin-edge tests run on the integer pipe (fp64_deposit_warp).
#include <math.h>

#include "rd_internal.cuh"

namespace rd {

// =============================================================================================
// Algorithm 1, per-sample part: beta, betadot (backward difference), 1/gamma^2, chord velocity.
// =============================================================================================
__device__ __forceinline__ void beta_of(const double* u, double& bx, double& by, double& bz,
                                        double& ig2)
{
    const double ux = u[0], uy = u[1], uz = u[2];
    const double uu = ux * ux + uy * uy + uz * uz;
    const double g = sqrt(1.0 + uu);
    bx = ux / g;
    by = uy / g;
    bz = uz / g;
    ig2 = 1.0 / (1.0 + uu);
}

__device__ __forceinline__ bool finite3(const double* v)
{
    return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

__global__ void k_precompute_mixed(const double* __restrict__ x, const double* __restrict__ u,
                                   const double* __restrict__ q, double qscale, int n_part, int n_samples,
                                   double dt, int flags, RecS* __restrict__ rec, DevCounters* counters)
{
    const long long total = (long long)n_part * n_samples;
    const double near_on = (flags & RD_NEAR) ? 1.0 : 0.0;
    const bool far_on = (flags & RD_FAR) != 0;
    const double inv_dt = 1.0 / dt;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % n_samples);
        // charge factor folded into the betadot and gamma^-2 terms of Eq. 1 (deposit records)
        const double qf = qscale != 0.0 ? -(q ? q[i / n_samples] : 1.0) * qscale : 1.0;
        const double* xk = x + 3 * i;
        const double* uk = u + 3 * i;
        bool bad = !finite3(xk) || !finite3(uk);
        double bx, by, bz, ig2;
        beta_of(uk, bx, by, bz, ig2);
        double ax = 0.0, ay = 0.0, az = 0.0, vx = 0.0, vy = 0.0, vz = 0.0, g = 1.0;
        if (k > 0) {
            double px, py, pz, pig2;
            beta_of(uk - 3, px, py, pz, pig2);
            ax = (bx - px) * inv_dt;
            ay = (by - py) * inv_dt;
            az = (bz - pz) * inv_dt;
            vx = (xk[0] - xk[-3]) * inv_dt;
            vy = (xk[1] - xk[-2]) * inv_dt;
            vz = (xk[2] - xk[-1]) * inv_dt;
            g = 1.0 - (vx * vx + vy * vy + vz * vz);
            bad = bad || !(g > 0.0);
        }
        if (bad) atomicOr(&counters->errors, ERRBIT_INPUT);
        // delta = beta_k - vbar_k (difference of end-point and chord velocities)
        const double ex = bx - vx, ey = by - vy, ez = bz - vz;
        auto put = [](double v) { return (float)v; };
        RecS r;
        r.nx = put(-xk[0]);
        r.ny = put(-xk[1]);
        r.nz = put(-xk[2]);
        r.nhig2 = put(-0.5 * ig2);
        r.nbx = put(-bx);
        r.nby = put(-by);
        r.nbz = put(-bz);
        r.ig2n = put(qf * (near_on * ig2));
        r.bdx = put(far_on ? qf * ax : 0.0);
        r.bdy = put(far_on ? qf * ay : 0.0);
        r.bdz = put(far_on ? qf * az : 0.0);
        r.dtg = put(dt * g);
        r.d2x = put(2.0 * ex);
        r.d2y = put(2.0 * ey);
        r.d2z = put(2.0 * ez);
        r.gd = put(g + (ex * ex + ey * ey + ez * ez));
        rec[i] = r;
    }
}

__global__ void k_precompute_fp64(const double* __restrict__ x, const double* __restrict__ u,
                                  const double* __restrict__ q, int n_part, int n_samples, double t0,
                                  double dt, int flags, RecD* __restrict__ rec, DevCounters* counters)
{
    const double near = (flags & RD_NEAR) ? 1.0 : 0.0, far = (flags & RD_FAR) ? 1.0 : 0.0;
    const long long total = (long long)n_part * n_samples;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % n_samples);
        const double* xk = x + 3 * i;
        const double* uk = u + 3 * i;
        bool bad = !finite3(xk) || !finite3(uk);
        double bx, by, bz, ig2;
        beta_of(uk, bx, by, bz, ig2);
        double ax = 0.0, ay = 0.0, az = 0.0;
        if (k > 0) {
            double px, py, pz, pig2;
            beta_of(uk - 3, px, py, pz, pig2);
            ax = (bx - px) / dt;
            ay = (by - py) / dt;
            az = (bz - pz) / dt;
            const double vx = xk[0] - xk[-3], vy = xk[1] - xk[-2], vz = xk[2] - xk[-1];
            bad = bad || !((vx * vx + vy * vy) + vz * vz < dt * dt);
        }
        if (bad) atomicOr(&counters->errors, ERRBIT_INPUT);
        RecD r;
        const double qp = q ? q[i / n_samples] : 1.0;
        r.xa = D4{xk[0], xk[1], xk[2], __dadd_rn(t0, __dmul_rn((double)k, dt))};
        r.bb = D4{bx, by, bz, (near * qp) * ig2};
        r.bd = D4{(far * qp) * ax, (far * qp) * ay, (far * qp) * az, 0.0};
        rec[i] = r;
    }
}

// =============================================================================================
// Plain FP64 deposit: Eq. 1 as printed, Eq. 2 evaluated directly for every sample.
// =============================================================================================
struct D64State {
    int b;
    double a;       // arrival (bins) of the previous sample
    double acc[6];
    double Fp[6];   // RD_LINEAR / RD_QUADRATIC: field of the previous sample
    double Fpp[6];  // RD_QUADRATIC: field two samples back ...
    double ap;      // ... and its arrival (bins)
    double e;       // held field: upper edge of bin b (b + 1) ...
    long long ke;   // ... and its order key (dkey)
    int n_below;
    int n_above;
};

// An integer that orders like the double x (finite x): the bit pattern for x >= 0, the magnitude bits
// flipped for x < 0, so that bin-edge tests run on the integer pipe.
__device__ __forceinline__ long long dkey(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

__device__ __forceinline__ void set_edge(D64State& st, double e)
{
    st.e = e;
    st.ke = dkey(e);
}

// The double n (|n| < 2^31) assembled from its integer on the integer pipe: sign, exponent
// 1023 + floor(log2 |n|), and the bits of |n| below its leading one as the mantissa's top bits.
__device__ __forceinline__ double int_to_double_bits(int n)
{
    const unsigned m = (unsigned)(n < 0 ? -n : n);
    const int hb = 31 - __clz((int)m);
    const long long bits = ((long long)(n < 0) << 63) | ((long long)(1023 + hb) << 52) |
                           ((long long)(m ^ (1u << hb)) << (52 - hb));
    return __longlong_as_double(n == 0 ? 0LL : bits);
}


__device__ __forceinline__ void flush_f64(double* row, int n_bins, int b, const double* v)
{
    if ((unsigned)b < (unsigned)n_bins) {
        double* p = row + (size_t)b * 6;
#pragma unroll
        for (int i = 0; i < 6; ++i) red_add_f64(p + i, v[i]);
    }
}

// 1/d by Newton-Raphson iteration from the hardware's approximate reciprocal: each step
// y <- y + y (1 - d y) squares the relative error, so two steps take the approximation to FP64
// rounding.  For the positive, normal arguments the field passes (kappa R >= R / (2 gamma^2)).
__device__ __forceinline__ double rcp_newton(double d)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    double e = fma(-d, y, 1.0);
    y = fma(y, e, y);
    e = fma(-d, y, 1.0);
    return fma(y, e, y);
}

// Eq. 1 at one cell, with d = x_cell - x_k and R = |d| as computed for the arrival time (Eq. 2).
// Writing n = d / R and kappa R = R - beta.d, Eq. 1 multiplies out to
//   E = q / (kappa R)^3 [a d - R v],   B = n x E = q / (kappa R)^3 v x d,
//   a = gamma^-2 + d.betadot,   v = a beta + (kappa R) betadot,
// so the only reciprocal is 1/(kappa R).  The record holds q gamma^-2 and q betadot, with gamma^-2 = 0
// without the velocity term (RD_NEAR) and betadot = 0 without the acceleration term (RD_FAR), so that
// a and v carry the charge.
__device__ __forceinline__ void fp64_field(const RecD& r, double dx, double dy, double dz, double R, double* F)
{
    const double kR = fma(-r.bb.z, dz, fma(-r.bb.y, dy, fma(-r.bb.x, dx, R)));
    const double a = fma(r.bd.z, dz, fma(r.bd.y, dy, fma(r.bd.x, dx, r.bb.w)));
    const double w = rcp_newton(kR);
    const double Q = w * (w * w);
    const double Qa = Q * a, Qk = Q * kR;
    const double vx = fma(Qa, r.bb.x, Qk * r.bd.x);     // Q v
    const double vy = fma(Qa, r.bb.y, Qk * r.bd.y);
    const double vz = fma(Qa, r.bb.z, Qk * r.bd.z);
    F[0] = fma(Qa, dx, -R * vx);
    F[1] = fma(Qa, dy, -R * vy);
    F[2] = fma(Qa, dz, -R * vz);
    F[3] = fma(vy, dz, -vz * dy);
    F[4] = fma(vz, dx, -vx * dz);
    F[5] = fma(vx, dy, -vy * dx);
}

// Eq. 2 for a record: the cell offset d, R = |d| and the arrival time in bins, with the same
// separately rounded operations as arrival_bins (t_k from the record).
__device__ __forceinline__ double fp64_arrival(const RecD& r, const D4& cl, double inv_dt_det, double& dx,
                                               double& dy, double& dz, double& R)
{
    dx = __dsub_rn(cl.x, r.xa.x);
    dy = __dsub_rn(cl.y, r.xa.y);
    dz = __dsub_rn(cl.z, r.xa.z);
    R = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    return __dmul_rn(__dsub_rn(__dadd_rn(r.xa.w, R), cl.w), inv_dt_det);
}

// Far-field limit of the radiation term: E = q n_c x ((n_c - beta) x betadot) / (kappa^3 R_c),
// kappa = 1 - beta.n_c, B = n_c x E (the record's betadot carries q, and is zero without RD_FAR).
__device__ __forceinline__ void fp64_field_ff(const RecD& r, double nx, double ny, double nz, double Rc,
                                              double* F)
{
    const double mx = nx - r.bb.x, my = ny - r.bb.y, mz = nz - r.bb.z;
    const double kap = 1.0 - (r.bb.x * nx + r.bb.y * ny + r.bb.z * nz);
    const double s = 1.0 / (kap * kap * kap * Rc);
    const double wx = my * r.bd.z - mz * r.bd.y;
    const double wy = mz * r.bd.x - mx * r.bd.z;
    const double wz = mx * r.bd.y - my * r.bd.x;
    const double Ex = s * (ny * wz - nz * wy), Ey = s * (nz * wx - nx * wz), Ez = s * (nx * wy - ny * wx);
    F[0] = Ex;
    F[1] = Ey;
    F[2] = Ez;
    F[3] = ny * Ez - nz * Ey;
    F[4] = nz * Ex - nx * Ez;
    F[5] = nx * Ey - ny * Ex;
}

// Deposit [st.a, c] with the bin-overlap arithmetic of the integrator detector.  The part inside the
// filling bin (up to its upper edge st.e = st.b + 1) is added on every step; only an interval that
// passes the edge flushes the bin and starts the next one with the rest, so the operations that
// every lane of a warp runs stay few (nearly every warp has a lane that crosses on each step).
__device__ __forceinline__ void fp64_deposit(D64State& st, const double* F, double c, double* row,
                                             int n_bins, int k, int k_begin, int k_end)
{
    const bool cr = c >= st.e;
    const double wi = (cr ? st.e : c) - st.a;
#pragma unroll
    for (int i = 0; i < 6; ++i) st.acc[i] = fma(F[i], wi, st.acc[i]);
    if (cr) {
        flush_f64(row, n_bins, st.b, st.acc);
        int b = st.b + 1;
        double e = st.e;                       // lower edge of bin b
        if (c >= e + 1.0) {                    // more than one edge: whole bins in between
            const int bc = clamp_bin(floor(c));
            const int lo = max(b, 0), hi = min(bc - 1, n_bins - 1);
            for (int j = lo; j <= hi; ++j) flush_f64(row, n_bins, j, F);
            b = bc;
            e = (double)bc;
        }
        const double wl = c - e;
#pragma unroll
        for (int i = 0; i < 6; ++i) st.acc[i] = F[i] * wl;
        if (st.b < 0 && b >= 0) st.n_below = k - k_begin + 1;
        if (st.b < n_bins && b >= n_bins) st.n_above = k_end - k + 1;
        st.b = b;
        set_edge(st, e + 1.0);
    }
    st.a = c;
}

// fp64_deposit for a warp whose 32 lanes all walk a cell (`warp` converged on every call).  The
// lanes whose arrival passed their bin's upper edge (about one in five) start their next bin with
// the rest of the interval, F times (c - e): instead of each lane's six multiplies taking six
// warp-wide FP64 instructions, the warp's crossing lanes' products are spread over all 32 lanes by
// shuffles (one or two FP64 instructions); the edge tests are integer compares and the next edge is
// assembled on the integer pipe, so that the FP64 pipe does the arithmetic of Eq. 1 and 2.
__device__ __forceinline__ void fp64_deposit_warp(D64State& st, const double* F, double c, double* row,
                                                  int n_bins, int k, int k_begin, int k_end)
{
    constexpr unsigned warp = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long kc = dkey(c);
    const bool cr = kc >= st.ke;
    const double wi = (cr ? st.e : c) - st.a;
#pragma unroll
    for (int i = 0; i < 6; ++i) st.acc[i] = fma(F[i], wi, st.acc[i]);
    st.a = c;
    const unsigned m = __ballot_sync(warp, cr);
    if (m == 0u) return;
    double wl = 0.0;
    if (cr) {
        flush_f64(row, n_bins, st.b, st.acc);
        int b = st.b + 1;
        wl = c - st.e;                         // st.e: lower edge of bin b
        // c - e >= 1 (compared on the bits: both are >= 0): more than one edge, whole bins in between
        if (__double_as_longlong(wl) >= 0x3FF0000000000000LL) {
            const int bc = clamp_bin(floor(c));
            const int lo = max(b, 0), hi = min(bc - 1, n_bins - 1);
            for (int j = lo; j <= hi; ++j) flush_f64(row, n_bins, j, F);
            b = bc;
            wl = c - (double)bc;
        }
        if (st.b < 0 && b >= 0) st.n_below = k - k_begin + 1;
        if (st.b < n_bins && b >= n_bins) st.n_above = k_end - k + 1;
        st.b = b;
        set_edge(st, int_to_double_bits(b + 1));
    }
    // product p = 6 r + q (r: rank of a crossing lane, q: component) is formed by lane p % 32 in
    // round p / 32 and handed back to its crossing lane
    const int n = __popc(m);
    const int rank = __popc(m & ((1u << lane) - 1u));
    for (int base = 0; base < 6 * n; base += 32) {
        const int pi = base + lane;
        const int r = pi / 6, q = pi - 6 * (pi / 6);
        const int src = pi < 6 * n ? (int)__fns(m, 0u, r + 1) : lane;
        double f = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const double v = __shfl_sync(warp, F[i], src);
            f = (q == i) ? v : f;
        }
        const double prod = f * __shfl_sync(warp, wl, src);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const int idx = 6 * rank + i;
            const double v = __shfl_sync(warp, prod, idx & 31);
            if (cr && idx >= base && idx < base + 32) st.acc[i] = v;
        }
    }
}

// RD_LINEAR: the field goes linearly from F0 at st.a to F1 at c; the overlap [u0, u1] of the interval
// with a bin weighs F0 (u1 - u0) + (F1 - F0) ((u1 - a)^2 - (u0 - a)^2) / (2 (c - a)).
__device__ __forceinline__ void fp64_lin_part(const double* F0, const double* F1, double a, double c, double u0,
                                              double u1, double* out, bool add)
{
    const double len = u1 - u0;
    const double ramp = ((u1 - a) * (u1 - a) - (u0 - a) * (u0 - a)) / (2.0 * (c - a));
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double v = F0[i] * len + (F1[i] - F0[i]) * ramp;
        out[i] = add ? out[i] + v : v;
    }
}

__device__ __forceinline__ void fp64_deposit_lin(D64State& st, const double* F0, const double* F1, double c,
                                                 double* row, int n_bins, int k, int k_begin, int k_end)
{
    const double a = st.a;
    const double fc = floor(c);
    const int bc = clamp_bin(fc);
    if (!(c > a)) {
        st.a = c;
        return;
    }
    if (bc <= st.b) {
        fp64_lin_part(F0, F1, a, c, a, c, st.acc, true);
        st.a = c;
        return;
    }
    fp64_lin_part(F0, F1, a, c, a, (double)(st.b + 1), st.acc, true);
    flush_f64(row, n_bins, st.b, st.acc);
    const int lo = max(st.b + 1, 0), hi = min(bc - 1, n_bins - 1);
    for (int j = lo; j <= hi; ++j) {
        double v[6];
        fp64_lin_part(F0, F1, a, c, (double)j, (double)(j + 1), v, false);
        flush_f64(row, n_bins, j, v);
    }
    fp64_lin_part(F0, F1, a, c, fc, c, st.acc, false);
    if (st.b < 0 && bc >= 0) st.n_below = k - k_begin + 1;
    if (st.b < n_bins && bc >= n_bins) st.n_above = k_end - k + 1;
    st.b = bc;
    st.a = c;
}

// RD_QUADRATIC: over [a, c] the quadratic through (p, Fpp), (a, Fa), (c, Fc) in arrival time, in Newton
// form about a (s = tau - a, L = c - a, h = a - p): F(s) = Fa + D1 s + D2 s (s - L), D1 = (Fc - Fa) / L,
// D2 = (D1 - (Fa - Fpp) / h) / (L + h); the overlap [u0, u1] receives
// Fa (s1 - s0) + D1 (s1^2 - s0^2) / 2 + D2 ((s1^3 - s0^3) / 3 - L (s1^2 - s0^2) / 2).
__device__ __forceinline__ void fp64_quad_part(const double* Fa, const double* D1, const double* D2, double a,
                                               double L, double u0, double u1, double* out, bool add)
{
    const double s0 = u0 - a, s1 = u1 - a;
    const double sq = (s1 * s1 - s0 * s0) / 2.0;
    const double cu = (s1 * s1 * s1 - s0 * s0 * s0) / 3.0 - L * sq;
    const double len = u1 - u0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double v = Fa[i] * len + D1[i] * sq + D2[i] * cu;
        out[i] = add ? out[i] + v : v;
    }
}

__device__ __forceinline__ void fp64_deposit_quad(D64State& st, const double* Fc, double c, double* row, int n_bins,
                                                  int k, int k_begin, int k_end)
{
    const double a = st.a;
    const double fc = floor(c);
    const int bc = clamp_bin(fc);
    if (!(c > a)) {
        st.a = c;
        return;
    }
    const double L = c - a, h = a - st.ap;
    double D1[6], D2[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double D0 = (st.Fp[i] - st.Fpp[i]) / h;
        D1[i] = (Fc[i] - st.Fp[i]) / L;
        D2[i] = (D1[i] - D0) / (L + h);
    }
    if (bc <= st.b) {
        fp64_quad_part(st.Fp, D1, D2, a, L, a, c, st.acc, true);
        st.a = c;
        return;
    }
    fp64_quad_part(st.Fp, D1, D2, a, L, a, (double)(st.b + 1), st.acc, true);
    flush_f64(row, n_bins, st.b, st.acc);
    const int lo = max(st.b + 1, 0), hi = min(bc - 1, n_bins - 1);
    for (int j = lo; j <= hi; ++j) {
        double v[6];
        fp64_quad_part(st.Fp, D1, D2, a, L, (double)j, (double)(j + 1), v, false);
        flush_f64(row, n_bins, j, v);
    }
    fp64_quad_part(st.Fp, D1, D2, a, L, fc, c, st.acc, false);
    if (st.b < 0 && bc >= 0) st.n_below = k - k_begin + 1;
    if (st.b < n_bins && bc >= n_bins) st.n_above = k_end - k + 1;
    st.b = bc;
    st.a = c;
}

#ifndef RD_FP64_MINBLOCKS
#define RD_FP64_MINBLOCKS 2      // CTAs of 256 threads per SM the held-field FP64 kernel is compiled for
#endif

// LM: interpolation family, 0 held field (default), 1 linear or held-previous (P.lin 1, 2), 2 quadratic
template <int LM>
__global__ void __launch_bounds__(kDepositThreads, LM == 0 ? RD_FP64_MINBLOCKS : 2) k_deposit_fp64(const DepositParams P,
                                                                       int flags)
{
    __shared__ __align__(128) RecD tile[2][kTileSteps];
    __shared__ __align__(8) uint64_t bar[2];

    const unsigned bid = blockIdx.x;
    const int p = (int)(bid % (unsigned)P.n_part);
    const unsigned rest = bid / (unsigned)P.n_part;
    const int cb = (int)(rest % (unsigned)P.n_cell_blocks);
    const int c = (int)(rest / (unsigned)P.n_cell_blocks);
    const int S = P.n_samples - 1;
    const int k_begin = P.k_first + c * P.chunk;
    const int k_end = min(S, k_begin + P.chunk - 1);
    const int n_int = k_end - k_begin + 1;
    const int n_tiles = (n_int + kTileSteps - 1) / kTileSteps;
    const RecD* rec = static_cast<const RecD*>(P.rec) + (size_t)p * P.n_samples;
    const int tid = threadIdx.x;
    const int cell = cb * kDepositThreads + tid;
    const bool active = cell < P.n_pix;

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

    D64State st;
    D4 cl = {0.0, 0.0, 0.0, 0.0};
    double ncx = 0.0, ncy = 0.0, ncz = 1.0, Rc = 1.0;       // far-field limit: cell direction, distance
    const bool ff = P.ff != 0;
    bool live = false;
    double* row = nullptr;
    const double* xp = P.x + (size_t)p * P.n_samples * 3;
    if (active) {
        cl = P.cells[cell];
        double Ra, Re;
        const double* xa = xp + 3 * (size_t)(k_begin - 1);
        const double* xe = xp + 3 * (size_t)k_end;
        double ua, ue;
        if (ff) {
            farfield_cell(cl, ncx, ncy, ncz, Rc);
            ua = arrival_bins_ff(xa[0], xa[1], xa[2], ncx, ncy, ncz, Rc, cl.w, P.t0, k_begin - 1, P.dt, P.inv_dt_det);
            ue = arrival_bins_ff(xe[0], xe[1], xe[2], ncx, ncy, ncz, Rc, cl.w, P.t0, k_end, P.dt, P.inv_dt_det);
        } else {
            ua = arrival_bins(xa[0], xa[1], xa[2], cl, P.t0, k_begin - 1, P.dt, P.inv_dt_det, Ra);
            ue = arrival_bins(xe[0], xe[1], xe[2], cl, P.t0, k_end, P.dt, P.inv_dt_det, Re);
        }
        live = (ue > 0.0) && (ua < (double)P.n_bins);
        st.a = ua;
        st.b = clamp_bin(floor(ua));
        if (LM == 0) set_edge(st, (double)st.b + 1.0);
        st.n_below = (ua < 0.0) ? n_int : 0;
        st.n_above = 0;
#pragma unroll
        for (int i = 0; i < 6; ++i) st.acc[i] = 0.0;
        row = static_cast<double*>(P.fields) + (size_t)cell * P.n_bins * 6;
        if (!live) atomicAdd(&P.counters->clipped, (unsigned long long)n_int);
    }
    // held field: warps whose every lane walks a cell share their bin-start work (fp64_deposit_warp)
    const bool full_warp = LM == 0 && __ballot_sync(0xffffffffu, live) == 0xffffffffu;
    if (LM && live) {
        // field of the sample before the chunk; a trajectory's first interval holds F_1
        const RecD r0 = rec[k_begin > 1 ? k_begin - 1 : 1];
        if (ff) {
            fp64_field_ff(r0, ncx, ncy, ncz, Rc, st.Fp);
        } else {
            double dx, dy, dz, R0;
            (void)fp64_arrival(r0, cl, P.inv_dt_det, dx, dy, dz, R0);
            fp64_field(r0, dx, dy, dz, R0, st.Fp);
        }
        // RD_QUADRATIC: the field and arrival of the sample two before the chunk (used from the
        // trajectory's third interval on)
        st.ap = st.a - 1.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) st.Fpp[i] = st.Fp[i];
        if (LM == 2 && k_begin >= 3) {
            const RecD r1 = rec[k_begin - 2];
            if (ff) {
                fp64_field_ff(r1, ncx, ncy, ncz, Rc, st.Fpp);
                st.ap = arrival_bins_ff(r1.xa.x, r1.xa.y, r1.xa.z, ncx, ncy, ncz, Rc, cl.w, P.t0, k_begin - 2, P.dt,
                                        P.inv_dt_det);
            } else {
                double dx, dy, dz, R1;
                st.ap = fp64_arrival(r1, cl, P.inv_dt_det, dx, dy, dz, R1);
                fp64_field(r1, dx, dy, dz, R1, st.Fpp);
            }
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
        if (live) {
            double F[6];
            for (int i = 0; i < cnt; ++i) {
                const RecD r = tile[buf][i];
                const int k = k0 + i;
                double cbin;
                if (ff) {
                    fp64_field_ff(r, ncx, ncy, ncz, Rc, F);
                    cbin = arrival_bins_ff(r.xa.x, r.xa.y, r.xa.z, ncx, ncy, ncz, Rc, cl.w, P.t0, k, P.dt, P.inv_dt_det);
                } else {
                    double dx, dy, dz, R;
                    cbin = fp64_arrival(r, cl, P.inv_dt_det, dx, dy, dz, R);
                    fp64_field(r, dx, dy, dz, R, F);
                }
                if (LM) {
                    const double a_prev = st.a;
                    if (LM == 2 && k + P.k_real0 >= 3)
                        fp64_deposit_quad(st, F, cbin, row, P.n_bins, k, k_begin, k_end);
                    else    // RD_HOLD_PREV (lin 2): the previous field at both ends, i.e. held
                        fp64_deposit_lin(st, st.Fp, P.lin == 2 ? st.Fp : F, cbin, row, P.n_bins, k, k_begin, k_end);
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        if (LM == 2) st.Fpp[j] = st.Fp[j];
                        st.Fp[j] = F[j];
                    }
                    if (LM == 2) st.ap = a_prev;
                } else {
                    if (full_warp)
                        fp64_deposit_warp(st, F, cbin, row, P.n_bins, k, k_begin, k_end);
                    else
                        fp64_deposit(st, F, cbin, row, P.n_bins, k, k_begin, k_end);
                }
            }
            if (t == n_tiles - 1) {
                flush_f64(row, P.n_bins, st.b, st.acc);
                const int clip = min(n_int, st.n_below + st.n_above);
                if (clip > 0) atomicAdd(&P.counters->clipped, (unsigned long long)clip);
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
}

// =============================================================================================
// readout: internal layout -> E[n_pix][n_bins][3], B[n_pix][n_bins][3]
// =============================================================================================
template <typename Tin, int STRIDE, typename Tout>
__global__ void k_read(const Tin* __restrict__ fields, long long n, Tout* __restrict__ E,
                       Tout* __restrict__ B)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const Tin* v = fields + i * STRIDE;
        if (E) {
            E[3 * i] = (Tout)v[0];
            E[3 * i + 1] = (Tout)v[1];
            E[3 * i + 2] = (Tout)v[2];
        }
        if (B) {
            B[3 * i] = (Tout)v[3];
            B[3 * i + 1] = (Tout)v[4];
            B[3 * i + 2] = (Tout)v[5];
        }
    }
}

// E[n_pix][n_bins][3], B[...] -> internal layout (the inverse of k_read); a NULL E or B sets that
// part to zero, and the padding of the mixed layout is cleared
template <typename Tin, int STRIDE, typename Tf>
__global__ void k_write(Tf* __restrict__ fields, long long n, const Tin* __restrict__ E, const Tin* __restrict__ B)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        Tf* v = fields + i * STRIDE;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[c] = E ? (Tf)E[3 * i + c] : (Tf)0;
            v[3 + c] = B ? (Tf)B[3 * i + c] : (Tf)0;
        }
#pragma unroll
        for (int c = 6; c < STRIDE; ++c) v[c] = (Tf)0;
    }
}

// =============================================================================================
// launchers
// =============================================================================================
static int grid_for(long long n, int threads) { return grid_stride_blocks(n, threads, 16); }

cudaError_t launch_precompute_mixed(const double* x, const double* u, const double* q, double qscale, int n_part,
                                    int n_samples, double dt, int flags, RecS* rec, DevCounters* counters,
                                    cudaStream_t s)
{
    const long long n = (long long)n_part * n_samples;
    k_precompute_mixed<<<grid_for(n, 256), 256, 0, s>>>(x, u, q, qscale, n_part, n_samples, dt, flags, rec,
                                                        counters);
    return cudaGetLastError();
}

cudaError_t launch_precompute_fp64(const double* x, const double* u, const double* q, int n_part, int n_samples,
                                   double t0, double dt, int flags, RecD* rec, DevCounters* counters, cudaStream_t s)
{
    const long long n = (long long)n_part * n_samples;
    k_precompute_fp64<<<grid_for(n, 256), 256, 0, s>>>(x, u, q, n_part, n_samples, t0, dt, flags, rec, counters);
    return cudaGetLastError();
}

cudaError_t launch_deposit_fp64(const DepositParams& p, int flags, cudaStream_t s)
{
    const long long blocks = (long long)p.n_cell_blocks * p.n_part * p.n_chunks;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (p.lin == 3)
        k_deposit_fp64<2><<<(unsigned)blocks, kDepositThreads, 0, s>>>(p, flags);
    else if (p.lin)
        k_deposit_fp64<1><<<(unsigned)blocks, kDepositThreads, 0, s>>>(p, flags);
    else
        k_deposit_fp64<0><<<(unsigned)blocks, kDepositThreads, 0, s>>>(p, flags);
    return cudaGetLastError();
}

cudaError_t launch_read_fields(const void* fields, int precision, int n_pix, int n_bins, void* E,
                               void* B, int dtype, cudaStream_t s)
{
    const long long n = (long long)n_pix * n_bins;
    const int g = grid_for(n, 256);
    if (precision == RD_MIXED) {
        if (dtype == RD_F32)
            k_read<float, 8, float><<<g, 256, 0, s>>>(static_cast<const float*>(fields), n,
                                                      static_cast<float*>(E), static_cast<float*>(B));
        else
            k_read<float, 8, double><<<g, 256, 0, s>>>(static_cast<const float*>(fields), n,
                                                       static_cast<double*>(E), static_cast<double*>(B));
    } else {
        if (dtype == RD_F32)
            k_read<double, 6, float><<<g, 256, 0, s>>>(static_cast<const double*>(fields), n,
                                                       static_cast<float*>(E), static_cast<float*>(B));
        else
            k_read<double, 6, double><<<g, 256, 0, s>>>(static_cast<const double*>(fields), n,
                                                        static_cast<double*>(E), static_cast<double*>(B));
    }
    return cudaGetLastError();
}

cudaError_t launch_write_fields(void* fields, int precision, int n_pix, int n_bins, const void* E, const void* B,
                                int dtype, cudaStream_t s)
{
    const long long n = (long long)n_pix * n_bins;
    const int g = grid_for(n, 256);
    if (precision == RD_MIXED) {
        if (dtype == RD_F32)
            k_write<float, 8, float><<<g, 256, 0, s>>>(static_cast<float*>(fields), n, static_cast<const float*>(E),
                                                       static_cast<const float*>(B));
        else
            k_write<double, 8, float><<<g, 256, 0, s>>>(static_cast<float*>(fields), n, static_cast<const double*>(E),
                                                        static_cast<const double*>(B));
    } else {
        if (dtype == RD_F32)
            k_write<float, 6, double><<<g, 256, 0, s>>>(static_cast<double*>(fields), n, static_cast<const float*>(E),
                                                        static_cast<const float*>(B));
        else
            k_write<double, 6, double><<<g, 256, 0, s>>>(static_cast<double*>(fields), n,
                                                         static_cast<const double*>(E), static_cast<const double*>(B));
    }
    return cudaGetLastError();
}

}  // namespace rd
