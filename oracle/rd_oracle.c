/*
 * FP64 CPU oracle of the RaDiO radiation deposit (Pardal et al., "RaDiO: an efficient
 * spatiotemporal radiation diagnostic for particle-in-cell codes").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load this library.  The product (the CUDA library) never calls it, and the two
 * share no code: not the kernels, not the headers, not any helper.
 *
 * What it computes: the integrator detector of Section 3.2 written out plainly.  For every
 * selected cell j, particle p and interval k = 1..S between trajectory samples k-1 and k:
 *     F_pk   = Eq. 1 at sample k (beta_k = u_k/sqrt(1+u_k^2), betadot_k = (beta_k-beta_{k-1})/dt)
 *     t'_pk  = t_k + |x_k - P_j|                                       (Eq. 2)
 *              (flags bit 4: the far-field limit, Eq. 3 and Eq. 1 with n, R of the cell seen
 *              from the origin; see rd_oracle_core.h)
 *     E_det[j][b] += F_pk * |[t'_p,k-1, t'_pk] ∩ [T_b, T_b+1)| / dt_det, T_b = t_min + pix_t0[j] + b dt_det
 * with times taken in bin units of the cell's axis so that bin edges are exact integers.
 * Loop order: cell -> particle -> interval -> bin (Algorithm 1 with Algorithm 2 inside).
 * Cells are independent, so cells are spread over threads; each cell's sum is formed in
 * exactly that order whatever the thread count.
 *
 * Inputs whose chord speed |x_k - x_{k-1}|/dt is not below 1 (or that are not finite) are
 * rejected (return 2): for such input the arrival times need not increase along the
 * trajectory and the deposit is undefined.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -pthread rd_oracle.c -lm
 * (-ffp-contract=off keeps every product and sum separately rounded, so the arrival times
 * are the same on every host.)
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- real instantiation ---- */
#define SCALAR double
#define SUFFIX r
#define S_SQRT(v) sqrt(v)
#define RE(v) (v)
#include "rd_oracle_core.h"
#undef SCALAR
#undef SUFFIX
#undef S_SQRT
#undef RE

/* ---- complex-step instantiation ---- */
#define SCALAR double complex
#define SUFFIX c
#define S_SQRT(v) csqrt(v)
#define RE(v) creal(v)
#include "rd_oracle_core.h"
#undef SCALAR
#undef SUFFIX
#undef S_SQRT
#undef RE

/* ---- extended-precision instantiation ----
 * The same formulas with long double particle quantities, arrival times and sums (64-bit
 * mantissa on x86-64, 113-bit on AArch64).  Cell positions, t_k = t0 + k dt and 1/dt_det stay
 * FP64 inputs, as in the other two.  Used to measure the rounding of the FP64 evaluation itself:
 * Eq. 2 adds R (large) to t, so a step's arrival increment dt (1 - beta.n) keeps only
 * ulp(R) / (dt kappa) of its digits, which grows as gamma^2 R. */
#define SCALAR long double
#define SUFFIX e
#define S_SQRT(v) sqrtl(v)
#define RE(v) ((double)(v))
#include "rd_oracle_core.h"
#undef SCALAR
#undef SUFFIX
#undef S_SQRT
#undef RE

typedef struct {
    int32_t n_pix;
    const double* pix_pos;   /* [n_pix][3] */
    const double* pix_t0;    /* [n_pix] or NULL */
    double t_min;
    double dt_det;
    int32_t n_bins;
    int32_t flags;
    int32_t n_part;
    int32_t n_samples;       /* S + 1 */
    const double* x;         /* [n_part][n_samples][3] */
    const double* u;         /* [n_part][n_samples][3] */
    const double* q;         /* [n_part] or NULL (all 1) */
    double t0;
    double dt;
} rdo_problem;

/* ------------------------------------------------------------------------------------------ */
/* single-point entry points (used by the pins)                                              */
/* ------------------------------------------------------------------------------------------ */
void rdo_field(const double x[3], const double beta[3], const double bdot[3], const double P[3],
               double q, int32_t flags, double E[3], double B[3])
{
    if (flags & 4)
        ff_field_r(beta, bdot, P, q, flags, E, B);
    else
        lw_field_r(x, beta, bdot, P, q, flags, E, B);
}

double rdo_arrival_time(double t, const double x[3], const double P[3])
{
    double dx = P[0] - x[0], dy = P[1] - x[1], dz = P[2] - x[2];
    return t + sqrt((dx * dx + dy * dy) + dz * dz);
}

double rdo_bin_coord(double t0, int64_t k, double dt, const double x[3], const double P[3],
                     double T0, double inv_dt_det, int32_t flags)
{
    return bin_coord_r(t0, (long long)k, dt, x, P, T0, inv_dt_det, flags);
}

/* Deposit one interval [a, c] (bin units) of the constant field F[6] into row[n_bins][6]. */
int32_t rdo_deposit_interval(double a, double c, const double F[6], int32_t n_bins, double* row)
{
    return deposit_interval_r(a, c, F, n_bins, row);
}

/* The linear-in-time interval (flags bit 8) and the quadratic one (flags bit 32), for the pins. */
int32_t rdo_deposit_interval_lin(double a, double c, const double F0[6], const double F1[6], int32_t n_bins,
                                 double* row)
{
    return deposit_interval_lin_r(a, c, F0, F1, n_bins, row);
}

int32_t rdo_deposit_interval_quad(double p, double a, double c, const double Fp[6], const double Fa[6],
                                  const double Fc[6], int32_t n_bins, double* row)
{
    return deposit_interval_quad_r(p, a, c, Fp, Fa, Fc, n_bins, row);
}

void rdo_beta(const double u[3], double beta[3]) { beta_of_r(u, beta); }

/* ------------------------------------------------------------------------------------------ */
/* validation                                                                                */
/* ------------------------------------------------------------------------------------------ */
static int check_problem(const rdo_problem* pr)
{
    if (!pr || pr->n_pix < 0 || pr->n_bins <= 0 || pr->n_part < 0 || pr->n_samples < 1) return 1;
    if (!(pr->dt > 0.0) || !(pr->dt_det > 0.0) || !isfinite(pr->t0) || !isfinite(pr->t_min)) return 1;
    if ((pr->n_pix > 0 && !pr->pix_pos) || (pr->n_part > 0 && (!pr->x || !pr->u))) return 1;
    const size_t ns = (size_t)pr->n_samples;
    for (int32_t p = 0; p < pr->n_part; ++p) {
        const double* x = pr->x + 3 * ns * (size_t)p;
        const double* u = pr->u + 3 * ns * (size_t)p;
        for (size_t k = 0; k < ns; ++k) {
            for (int i = 0; i < 3; ++i)
                if (!isfinite(x[3 * k + i]) || !isfinite(u[3 * k + i])) return 2;
            if (k > 0) {
                double d0 = x[3 * k] - x[3 * k - 3], d1 = x[3 * k + 1] - x[3 * k - 2],
                       d2 = x[3 * k + 2] - x[3 * k - 1];
                if (!((d0 * d0 + d1 * d1) + d2 * d2 < pr->dt * pr->dt)) return 2;
            }
        }
        if (pr->q && !isfinite(pr->q[p])) return 2;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* threaded drivers                                                                          */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    const rdo_problem* pr;
    const int32_t* sel;
    int32_t n_sel;
    int32_t tid, n_threads;
    double* E;             /* [n_sel][n_bins][3] */
    double* B;
    long long clipped;
    int status;
    /* complex-step: particle p, sample k, which (0: x, 1: u), component, step h */
    int32_t cs_p, cs_k, cs_which, cs_comp;
    double cs_h;
} rdo_job;

static void* run_real(void* arg)
{
    rdo_job* jb = (rdo_job*)arg;
    const rdo_problem* pr = jb->pr;
    const int nb = pr->n_bins;
    const size_t ns = (size_t)pr->n_samples;
    const double inv_dt_det = 1.0 / pr->dt_det;
    double* row = (double*)malloc(sizeof(double) * 6 * (size_t)nb);
    if (!row) { jb->status = 3; return NULL; }
    for (int32_t s = jb->tid; s < jb->n_sel; s += jb->n_threads) {
        const int32_t j = jb->sel ? jb->sel[s] : s;
        const double* P = pr->pix_pos + 3 * (size_t)j;
        const double T0 = pr->t_min + (pr->pix_t0 ? pr->pix_t0[j] : 0.0);
        memset(row, 0, sizeof(double) * 6 * (size_t)nb);
        for (int32_t p = 0; p < pr->n_part; ++p) {
            const double qp = pr->q ? pr->q[p] : 1.0;
            jb->clipped += pixel_particle_r(pr->x + 3 * ns * (size_t)p, pr->u + 3 * ns * (size_t)p,
                                            pr->n_samples, qp, pr->t0, pr->dt, P, T0, inv_dt_det,
                                            nb, pr->flags, row);
        }
        double* Eo = jb->E + 3 * (size_t)nb * (size_t)s;
        double* Bo = jb->B + 3 * (size_t)nb * (size_t)s;
        for (int b = 0; b < nb; ++b)
            for (int i = 0; i < 3; ++i) {
                Eo[3 * b + i] = row[6 * b + i];
                Bo[3 * b + i] = row[6 * b + 3 + i];
            }
    }
    free(row);
    return NULL;
}

static void* run_cstep(void* arg)
{
    rdo_job* jb = (rdo_job*)arg;
    const rdo_problem* pr = jb->pr;
    const int nb = pr->n_bins;
    const size_t ns = (size_t)pr->n_samples;
    const double inv_dt_det = 1.0 / pr->dt_det;
    const int32_t p = jb->cs_p;
    double complex* row = (double complex*)malloc(sizeof(double complex) * 6 * (size_t)nb);
    double complex* xs = (double complex*)malloc(sizeof(double complex) * 3 * ns);
    double complex* us = (double complex*)malloc(sizeof(double complex) * 3 * ns);
    if (!row || !xs || !us) { free(row); free(xs); free(us); jb->status = 3; return NULL; }
    for (size_t i = 0; i < 3 * ns; ++i) {
        xs[i] = pr->x[3 * ns * (size_t)p + i];
        us[i] = pr->u[3 * ns * (size_t)p + i];
    }
    double complex* tgt = jb->cs_which == 0 ? xs : us;
    tgt[3 * (size_t)jb->cs_k + (size_t)jb->cs_comp] += I * jb->cs_h;
    const double qp = pr->q ? pr->q[p] : 1.0;
    for (int32_t s = jb->tid; s < jb->n_sel; s += jb->n_threads) {
        const int32_t j = jb->sel ? jb->sel[s] : s;
        const double* P = pr->pix_pos + 3 * (size_t)j;
        const double T0 = pr->t_min + (pr->pix_t0 ? pr->pix_t0[j] : 0.0);
        for (size_t i = 0; i < 6 * (size_t)nb; ++i) row[i] = 0.0;
        pixel_particle_c(xs, us, pr->n_samples, qp, pr->t0, pr->dt, P, T0, inv_dt_det, nb,
                         pr->flags, row);
        double* Eo = jb->E + 3 * (size_t)nb * (size_t)s;
        double* Bo = jb->B + 3 * (size_t)nb * (size_t)s;
        for (int b = 0; b < nb; ++b)
            for (int i = 0; i < 3; ++i) {
                Eo[3 * b + i] = cimag(row[6 * b + i]) / jb->cs_h;
                Bo[3 * b + i] = cimag(row[6 * b + 3 + i]) / jb->cs_h;
            }
    }
    free(row);
    free(xs);
    free(us);
    return NULL;
}

static void* run_ext(void* arg)
{
    rdo_job* jb = (rdo_job*)arg;
    const rdo_problem* pr = jb->pr;
    const int nb = pr->n_bins;
    const size_t ns = (size_t)pr->n_samples;
    const double inv_dt_det = 1.0 / pr->dt_det;
    long double* row = (long double*)malloc(sizeof(long double) * 6 * (size_t)nb);
    long double* xs = (long double*)malloc(sizeof(long double) * 3 * ns);
    long double* us = (long double*)malloc(sizeof(long double) * 3 * ns);
    if (!row || !xs || !us) { free(row); free(xs); free(us); jb->status = 3; return NULL; }
    for (int32_t s = jb->tid; s < jb->n_sel; s += jb->n_threads) {
        const int32_t j = jb->sel ? jb->sel[s] : s;
        const double* P = pr->pix_pos + 3 * (size_t)j;
        const double T0 = pr->t_min + (pr->pix_t0 ? pr->pix_t0[j] : 0.0);
        for (size_t i = 0; i < 6 * (size_t)nb; ++i) row[i] = 0.0L;
        for (int32_t p = 0; p < pr->n_part; ++p) {
            for (size_t i = 0; i < 3 * ns; ++i) {
                xs[i] = pr->x[3 * ns * (size_t)p + i];
                us[i] = pr->u[3 * ns * (size_t)p + i];
            }
            const double qp = pr->q ? pr->q[p] : 1.0;
            jb->clipped += pixel_particle_e(xs, us, pr->n_samples, qp, pr->t0, pr->dt, P, T0, inv_dt_det,
                                            nb, pr->flags, row);
        }
        double* Eo = jb->E + 3 * (size_t)nb * (size_t)s;
        double* Bo = jb->B + 3 * (size_t)nb * (size_t)s;
        for (int b = 0; b < nb; ++b)
            for (int i = 0; i < 3; ++i) {
                Eo[3 * b + i] = (double)row[6 * b + i];
                Bo[3 * b + i] = (double)row[6 * b + 3 + i];
            }
    }
    free(row);
    free(xs);
    free(us);
    return NULL;
}

static int run_threads(rdo_job* proto, int32_t n_threads, void* (*fn)(void*), long long* clipped)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    rdo_job jobs[256];
    pthread_t th[256];
    int started[256];
    for (int t = 0; t < n_threads; ++t) {
        jobs[t] = *proto;
        jobs[t].tid = t;
        jobs[t].n_threads = n_threads;
        jobs[t].clipped = 0;
        jobs[t].status = 0;
        started[t] = (t > 0) ? (pthread_create(&th[t], NULL, fn, &jobs[t]) == 0) : 0;
    }
    fn(&jobs[0]);
    /* any worker that failed to start is run on this thread */
    for (int t = 1; t < n_threads; ++t)
        if (!started[t]) fn(&jobs[t]);
    int status = 0;
    long long total = 0;
    for (int t = 0; t < n_threads; ++t) {
        if (t > 0 && started[t]) pthread_join(th[t], NULL);
        if (jobs[t].status) status = jobs[t].status;
        total += jobs[t].clipped;
    }
    if (clipped) *clipped = total;
    return status;
}

/*
 * E, B: [n_sel][n_bins][3], overwritten.  sel: cell indices (NULL = the first n_sel cells).
 * Returns 0 ok, 1 bad arguments, 2 invalid trajectory, 3 out of memory.
 * n_clipped (optional) receives the number of (cell, particle, interval) triples that had a
 * part of their arrival interval outside the window.
 */
int32_t rdo_deposit(const rdo_problem* pr, const int32_t* sel, int32_t n_sel, double* E, double* B,
                    int32_t n_threads, int64_t* n_clipped)
{
    int st = check_problem(pr);
    if (st) return st;
    if (n_sel < 0 || (n_sel > 0 && (!E || !B))) return 1;
    for (int32_t s = 0; s < n_sel; ++s) {
        int32_t j = sel ? sel[s] : s;
        if (j < 0 || j >= pr->n_pix) return 1;
    }
    rdo_job proto;
    memset(&proto, 0, sizeof proto);
    proto.pr = pr;
    proto.sel = sel;
    proto.n_sel = n_sel;
    proto.E = E;
    proto.B = B;
    long long c = 0;
    st = run_threads(&proto, n_threads, run_real, &c);
    if (n_clipped) *n_clipped = (int64_t)c;
    return st;
}

/* rdo_deposit evaluated in long double (extended-precision instantiation above); same
 * arguments, outputs rounded to FP64. */
int32_t rdo_deposit_ext(const rdo_problem* pr, const int32_t* sel, int32_t n_sel, double* E, double* B,
                        int32_t n_threads, int64_t* n_clipped)
{
    int st = check_problem(pr);
    if (st) return st;
    if (n_sel < 0 || (n_sel > 0 && (!E || !B))) return 1;
    for (int32_t s = 0; s < n_sel; ++s) {
        int32_t j = sel ? sel[s] : s;
        if (j < 0 || j >= pr->n_pix) return 1;
    }
    rdo_job proto;
    memset(&proto, 0, sizeof proto);
    proto.pr = pr;
    proto.sel = sel;
    proto.n_sel = n_sel;
    proto.E = E;
    proto.B = B;
    long long c = 0;
    st = run_threads(&proto, n_threads, run_ext, &c);
    if (n_clipped) *n_clipped = (int64_t)c;
    return st;
}

/*
 * Complex-step derivative of particle p's contribution to the selected cells with respect to
 * one input coordinate: x[p][k][comp] (which = 0) or u[p][k][comp] (which = 1).
 * dE, dB: [n_sel][n_bins][3] receive d E_det / d coordinate (other particles do not depend on it).
 */
int32_t rdo_deposit_dir(const rdo_problem* pr, const int32_t* sel, int32_t n_sel, int32_t p,
                        int32_t k, int32_t which, int32_t comp, double h, double* dE, double* dB,
                        int32_t n_threads)
{
    int st = check_problem(pr);
    if (st) return st;
    if (p < 0 || p >= pr->n_part || k < 0 || k >= pr->n_samples || which < 0 || which > 1 ||
        comp < 0 || comp > 2 || !(h > 0.0) || n_sel < 0 || (n_sel > 0 && (!dE || !dB)))
        return 1;
    for (int32_t s = 0; s < n_sel; ++s) {
        int32_t j = sel ? sel[s] : s;
        if (j < 0 || j >= pr->n_pix) return 1;
    }
    rdo_job proto;
    memset(&proto, 0, sizeof proto);
    proto.pr = pr;
    proto.sel = sel;
    proto.n_sel = n_sel;
    proto.E = dE;
    proto.B = dB;
    proto.cs_p = p;
    proto.cs_k = k;
    proto.cs_which = which;
    proto.cs_comp = comp;
    proto.cs_h = h;
    return run_threads(&proto, n_threads, run_cstep, NULL);
}
