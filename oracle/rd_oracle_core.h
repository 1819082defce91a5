/*
 * Scalar-generic core of the FP64 oracle.  TEST INFRASTRUCTURE ONLY: see rd_oracle.c.
 *
 * Included three times by rd_oracle.c: with SCALAR = double (the oracle proper), with
 * SCALAR = double complex (complex-step differentiation: perturbing one input by i*h gives
 * d(output)/d(input) = Im(output)/h exactly up to rounding, because every operation used here
 * is analytic; comparisons and floor() act on real parts only) and with SCALAR = long double
 * (the same evaluation with a longer mantissa, to measure the rounding of the FP64 one).
 *
 * Macros expected: SCALAR, SUFFIX, S_SQRT(x), RE(x).
 */
#define RDO_CAT2(a, b) a##_##b
#define RDO_CAT(a, b) RDO_CAT2(a, b)
#define FN(name) RDO_CAT(name, SUFFIX)

/* beta = u / sqrt(1 + |u|^2): Algorithm 1, velocity of a particle from its momentum p/(mc). */
static void FN(beta_of)(const SCALAR u[3], SCALAR beta[3])
{
    SCALAR uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    SCALAR g = S_SQRT(1.0 + uu);
    beta[0] = u[0] / g;
    beta[1] = u[1] / g;
    beta[2] = u[2] / g;
}

/*
 * Eq. 1 (Lienard-Wiechert fields, Gaussian units with e -> q and c = 1), evaluated with the
 * particle quantities of one trajectory sample:
 *   E = q (n - beta) / (gamma^2 kappa^3 R^2)  +  q n x ((n - beta) x betadot) / (kappa^3 R)
 *   B = n x E,   kappa = 1 - beta.n,   1/gamma^2 = 1 - beta^2 (Section 2 definitions)
 * n is the unit vector from the particle to the detector cell (Section 2 text; Algorithm 1 prints
 * the opposite sign, which would reverse the outgoing wave).
 * flags bit 1 keeps the first (velocity, "near") term, bit 2 the second (acceleration, "far").
 */
static void FN(lw_field)(const SCALAR x[3], const SCALAR beta[3], const SCALAR bdot[3],
                         const double P[3], double q, int flags, SCALAR E[3], SCALAR B[3])
{
    SCALAR d[3] = {P[0] - x[0], P[1] - x[1], P[2] - x[2]};
    SCALAR R = S_SQRT(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    SCALAR n[3] = {d[0] / R, d[1] / R, d[2] / R};
    SCALAR nb[3] = {n[0] - beta[0], n[1] - beta[1], n[2] - beta[2]};
    SCALAR kappa = 1.0 - (beta[0] * n[0] + beta[1] * n[1] + beta[2] * n[2]);
    SCALAR inv_gamma2 = 1.0 - (beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2]);
    SCALAR k3 = kappa * kappa * kappa;
    for (int i = 0; i < 3; ++i) E[i] = 0.0;
    if (flags & 1) {
        SCALAR c = q * inv_gamma2 / (k3 * R * R);
        for (int i = 0; i < 3; ++i) E[i] += c * nb[i];
    }
    if (flags & 2) {
        /* w = (n - beta) x betadot ; far = n x w */
        SCALAR w[3] = {nb[1] * bdot[2] - nb[2] * bdot[1],
                       nb[2] * bdot[0] - nb[0] * bdot[2],
                       nb[0] * bdot[1] - nb[1] * bdot[0]};
        SCALAR f[3] = {n[1] * w[2] - n[2] * w[1],
                       n[2] * w[0] - n[0] * w[2],
                       n[0] * w[1] - n[1] * w[0]};
        SCALAR c = q / (k3 * R);
        for (int i = 0; i < 3; ++i) E[i] += c * f[i];
    }
    B[0] = n[1] * E[2] - n[2] * E[1];
    B[1] = n[2] * E[0] - n[0] * E[2];
    B[2] = n[0] * E[1] - n[1] * E[0];
}

/*
 * Far-field (Fraunhofer) limit, flags bit 4.  A cell at P is seen from the origin along
 * n_c = P/|P| at distance R_c = |P| (computed as R_c = sqrt((P0*P0 + P1*P1) + P2*P2), n_c = P/R_c).
 * The radiation term of Eq. 1 is taken with n = n_c and R = R_c:
 *   E = q n_c x ((n_c - beta) x betadot) / (kappa^3 R_c),  kappa = 1 - beta.n_c,  B = n_c x E;
 * the velocity term, of order 1/R^2, is not part of this limit (bit 1 is ignored).
 */
static void FN(ff_dir)(const double P[3], double nc[3], double* Rc)
{
    double R = sqrt((P[0] * P[0] + P[1] * P[1]) + P[2] * P[2]);
    *Rc = R;
    for (int i = 0; i < 3; ++i) nc[i] = P[i] / R;
}

static void FN(ff_field)(const SCALAR beta[3], const SCALAR bdot[3], const double P[3], double q, int flags,
                         SCALAR E[3], SCALAR B[3])
{
    double nc[3], Rc;
    FN(ff_dir)(P, nc, &Rc);
    SCALAR m[3] = {nc[0] - beta[0], nc[1] - beta[1], nc[2] - beta[2]};
    SCALAR kap = 1.0 - (beta[0] * nc[0] + beta[1] * nc[1] + beta[2] * nc[2]);
    SCALAR v[3] = {m[1] * bdot[2] - m[2] * bdot[1], m[2] * bdot[0] - m[0] * bdot[2], m[0] * bdot[1] - m[1] * bdot[0]};
    SCALAR s = (flags & 2) ? q / (kap * kap * kap * Rc) : 0.0;
    E[0] = s * (nc[1] * v[2] - nc[2] * v[1]);
    E[1] = s * (nc[2] * v[0] - nc[0] * v[2]);
    E[2] = s * (nc[0] * v[1] - nc[1] * v[0]);
    B[0] = nc[1] * E[2] - nc[2] * E[1];
    B[1] = nc[2] * E[0] - nc[0] * E[2];
    B[2] = nc[0] * E[1] - nc[1] * E[0];
}

/*
 * Arrival time of sample k at cell P in bin units of the cell's time axis (Eq. 2, c = 1):
 *   t_det = t_k + |x_k - P|,  t_k = t0 + k dt,   u = (t_det - T0) / dt_det
 * evaluated in this fixed order, with no fused multiply-add:
 *   t_k = t0 + (k*dt);  R = sqrt((dx*dx + dy*dy) + dz*dz);  u = ((t_k + R) - T0) * inv_dt_det.
 * flags bit 4: Eq. 3 in place of Eq. 2 (far-field limit above).
 */
static SCALAR FN(bin_coord)(double t0, long long k, double dt, const SCALAR x[3], const double P[3],
                            double T0, double inv_dt_det, int flags)
{
    double tk = t0 + (double)k * dt;
    if (flags & 4) {
        /* Eq. 3: t_det = t + R_c - x.n_c, as ((t_k + R_c) - ((x0*n0 + x1*n1) + x2*n2)) */
        double nc[3], Rc;
        FN(ff_dir)(P, nc, &Rc);
        SCALAR xn = (x[0] * nc[0] + x[1] * nc[1]) + x[2] * nc[2];
        SCALAR t_ff = (tk + Rc) - xn;
        return (t_ff - T0) * inv_dt_det;
    }
    SCALAR dx = P[0] - x[0], dy = P[1] - x[1], dz = P[2] - x[2];
    SCALAR R = S_SQRT((dx * dx + dy * dy) + dz * dz);
    SCALAR tdet = tk + R;
    return (tdet - T0) * inv_dt_det;
}

/*
 * Integrating deposit of one interval (Section 3.2, Algorithm 2 read as the integrator
 * detector): the field F (E then B, 6 values) is held constant over the arrival interval
 * [a, c] (bin units) and bin b = [b, b+1) receives F * |[a, c] ∩ [b, b+1)|.
 * Parts of the interval outside [0, n_bins) are dropped; the return value is 1 if anything
 * was dropped, else 0.
 */
static int FN(deposit_interval)(SCALAR a, SCALAR c, const SCALAR F[6], int n_bins, SCALAR* row)
{
    double ra = RE(a), rc = RE(c);
    int clipped = (ra < 0.0) || (rc > (double)n_bins);
    if (rc <= 0.0 || ra >= (double)n_bins) return 1;
    double flo = floor(ra), fhi = floor(rc);
    long long lo = flo < 0.0 ? 0 : (long long)flo;
    long long hi = fhi > (double)(n_bins - 1) ? (long long)(n_bins - 1) : (long long)fhi;
    for (long long b = lo; b <= hi; ++b) {
        SCALAR s = (ra > (double)b) ? a : (SCALAR)(double)b;
        SCALAR e = (rc < (double)(b + 1)) ? c : (SCALAR)(double)(b + 1);
        SCALAR w = e - s;
        if (RE(w) > 0.0) {
            for (int i = 0; i < 6; ++i) row[6 * b + i] += F[i] * w;
        }
    }
    return clipped;
}

/*
 * Linear-in-time variant (flags bit 8; an interpolation of higher order than the held field, of
 * the kind the paper's outlook names): over the arrival interval [a, c] the field varies linearly
 * in arrival time from F0 (sample k-1) at a to F1 (sample k) at c, and bin b receives the integral
 * of that line over [a, c] ∩ [b, b+1):
 *     F0 (e - s) + (F1 - F0) ((e - a)^2 - (s - a)^2) / (2 (c - a)),   [s, e] the overlap.
 */
static int FN(deposit_interval_lin)(SCALAR a, SCALAR c, const SCALAR F0[6], const SCALAR F1[6], int n_bins,
                                    SCALAR* row)
{
    double ra = RE(a), rc = RE(c);
    int clipped = (ra < 0.0) || (rc > (double)n_bins);
    if (rc <= 0.0 || ra >= (double)n_bins) return 1;
    long long first = floor(ra) < 0.0 ? 0 : (long long)floor(ra);
    long long last = floor(rc) > (double)(n_bins - 1) ? (long long)(n_bins - 1) : (long long)floor(rc);
    for (long long b = first; b <= last; ++b) {
        SCALAR u0 = (ra > (double)b) ? a : (SCALAR)(double)b;
        SCALAR u1 = (rc < (double)(b + 1)) ? c : (SCALAR)(double)(b + 1);
        SCALAR len = u1 - u0;
        if (RE(len) > 0.0) {
            SCALAR ramp = ((u1 - a) * (u1 - a) - (u0 - a) * (u0 - a)) / (2.0 * (c - a));
            for (int i = 0; i < 6; ++i) row[6 * b + i] += F0[i] * len + (F1[i] - F0[i]) * ramp;
        }
    }
    return clipped;
}

/*
 * Quadratic-in-time variant (flags bit 32; the next order after the linear one): over the arrival
 * interval [a, c] of sample k the field is the quadratic through (p, F_{k-2}), (a, F_{k-1}),
 * (c, F_k), p = t_det,k-2 < a, written in Newton form about a with s = tau - a, L = c - a, h = a - p:
 *     F(s) = Fa + D1 s + D2 s (s - L),   D1 = (Fc - Fa) / L,   D0 = (Fa - Fp) / h,
 *     D2 = (D1 - D0) / (L + h)   (the second divided difference),
 * and bin b receives its integral over the overlap [s0, s1] of [a, c] with [b, b+1):
 *     Fa (s1 - s0) + D1 (s1^2 - s0^2) / 2 + D2 ((s1^3 - s0^3) / 3 - L (s1^2 - s0^2) / 2).
 */
static int FN(deposit_interval_quad)(SCALAR p, SCALAR a, SCALAR c, const SCALAR Fp[6], const SCALAR Fa[6],
                                     const SCALAR Fc[6], int n_bins, SCALAR* row)
{
    double ra = RE(a), rc = RE(c);
    int clipped = (ra < 0.0) || (rc > (double)n_bins);
    if (rc <= 0.0 || ra >= (double)n_bins) return 1;
    SCALAR L = c - a, h = a - p;
    SCALAR D1[6], D2[6];
    for (int i = 0; i < 6; ++i) {
        SCALAR D0 = (Fa[i] - Fp[i]) / h;
        D1[i] = (Fc[i] - Fa[i]) / L;
        D2[i] = (D1[i] - D0) / (L + h);
    }
    long long first = floor(ra) < 0.0 ? 0 : (long long)floor(ra);
    long long last = floor(rc) > (double)(n_bins - 1) ? (long long)(n_bins - 1) : (long long)floor(rc);
    for (long long b = first; b <= last; ++b) {
        SCALAR u0 = (ra > (double)b) ? a : (SCALAR)(double)b;
        SCALAR u1 = (rc < (double)(b + 1)) ? c : (SCALAR)(double)(b + 1);
        SCALAR len = u1 - u0;
        if (RE(len) > 0.0) {
            SCALAR s0 = u0 - a, s1 = u1 - a;
            SCALAR sq = (s1 * s1 - s0 * s0) / 2.0;
            SCALAR cu = (s1 * s1 * s1 - s0 * s0 * s0) / 3.0 - L * sq;
            for (int i = 0; i < 6; ++i) row[6 * b + i] += Fa[i] * len + D1[i] * sq + D2[i] * cu;
        }
    }
    return clipped;
}

/*
 * One (cell, particle) pair: Algorithm 1 inner body for every interval k = 1..S.
 *   beta_k from u_k; betadot_k = (beta_k - beta_{k-1}) / dt (backward difference);
 *   the field of sample k is held over [t_det,k-1, t_det,k] (the algorithm passes the current
 *   step's field to the interpolator); sample 0 only provides the previous quantities.
 * flags bit 8: from interval 2 on, the field varies linearly from F_{k-1} to F_k over the
 * interval (deposit_interval_lin); interval 1 holds F_1 (sample 0 has no field: no betadot).
 * flags bit 16: from interval 2 on, the interval holds the field of its first sample, F_{k-1}
 * (the other reading of which field the interpolation holds: the worked example of Section 3.2
 * writes, for the interval ending at t'_4, the field at t'_3); interval 1 holds F_1.
 * flags bit 32: from interval 3 on, the quadratic through the fields of samples k-2, k-1, k at
 * their arrival times (deposit_interval_quad); interval 2 is linear (F_1 to F_2), interval 1 holds
 * F_1 (sample 0 has no field, so the first two intervals have fewer than three fields behind them).
 * x, u point at this particle's samples [n_samples][3]; row is [n_bins][6] (E xyz, B xyz).
 * Returns the number of intervals that had a part outside the window.
 */
static long long FN(pixel_particle)(const SCALAR* x, const SCALAR* u, int n_samples, double q,
                                    double t0, double dt, const double P[3], double T0,
                                    double inv_dt_det, int n_bins, int flags, SCALAR* row)
{
    SCALAR beta_prev[3], beta[3], bdot[3], E[3], B[3], F[6], Fprev[6], Fpp[6];
    long long clipped = 0;
    FN(beta_of)(u, beta_prev);
    SCALAR a = FN(bin_coord)(t0, 0, dt, x, P, T0, inv_dt_det, flags);
    SCALAR ap = a;                                   /* arrival of sample k-2 */
    for (int k = 1; k < n_samples; ++k) {
        const SCALAR* xk = x + 3 * (size_t)k;
        FN(beta_of)(u + 3 * (size_t)k, beta);
        for (int i = 0; i < 3; ++i) bdot[i] = (beta[i] - beta_prev[i]) / dt;
        if (flags & 4)
            FN(ff_field)(beta, bdot, P, q, flags, E, B);
        else
            FN(lw_field)(xk, beta, bdot, P, q, flags, E, B);
        for (int i = 0; i < 3; ++i) { F[i] = E[i]; F[3 + i] = B[i]; }
        SCALAR c = FN(bin_coord)(t0, k, dt, xk, P, T0, inv_dt_det, flags);
        if ((flags & 32) && k > 2)
            clipped += FN(deposit_interval_quad)(ap, a, c, Fpp, Fprev, F, n_bins, row);
        else if ((flags & (8 | 32)) && k > 1)
            clipped += FN(deposit_interval_lin)(a, c, Fprev, F, n_bins, row);
        else if ((flags & 16) && k > 1)
            clipped += FN(deposit_interval)(a, c, Fprev, n_bins, row);
        else
            clipped += FN(deposit_interval)(a, c, F, n_bins, row);
        for (int i = 0; i < 6; ++i) {
            Fpp[i] = Fprev[i];
            Fprev[i] = F[i];
        }
        ap = a;
        a = c;
        for (int i = 0; i < 3; ++i) beta_prev[i] = beta[i];
    }
    return clipped;
}

#undef FN
#undef RDO_CAT
#undef RDO_CAT2
