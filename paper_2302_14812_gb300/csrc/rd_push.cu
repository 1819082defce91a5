// Run-time coupling (Section 3.1: the deposit as a sub-step right after the particle push): a
// Boris pusher for charges in a uniform magnetic field, advancing the state on the device and
// writing the new samples where rd_deposit_stream takes them.
//
// Per step (c = 1, u = gamma beta, magnetic field only, so gamma is constant):
//   t = (qm dt / 2) B / gamma,  s = 2 t / (1 + |t|^2),  u' = u + u x t,  u <- u + u' x s,
//   x <- x + dt u / gamma
// (the Boris rotation: |u| is kept, and u turns about B by 2 atan(|t|) per step).
#include <math.h>

#include "rd_internal.cuh"

namespace rd {

namespace {

__global__ void k_push_boris(int n_part, int n_steps, double dt, double bx, double by, double bz, double qm,
                             double* __restrict__ x, double* __restrict__ u, double* __restrict__ x_out,
                             double* __restrict__ u_out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_part) return;
    double X[3] = {x[3 * p], x[3 * p + 1], x[3 * p + 2]};
    double U[3] = {u[3 * p], u[3 * p + 1], u[3 * p + 2]};
    const double g = sqrt(1.0 + (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]));
    const double h = 0.5 * qm * dt / g;
    const double t[3] = {h * bx, h * by, h * bz};
    const double f = 2.0 / (1.0 + (t[0] * t[0] + t[1] * t[1] + t[2] * t[2]));
    const double s[3] = {f * t[0], f * t[1], f * t[2]};
    const double w = dt / g;
    for (int k = 0; k < n_steps; ++k) {
        const double v[3] = {U[0] + (U[1] * t[2] - U[2] * t[1]), U[1] + (U[2] * t[0] - U[0] * t[2]),
                             U[2] + (U[0] * t[1] - U[1] * t[0])};
        U[0] += v[1] * s[2] - v[2] * s[1];
        U[1] += v[2] * s[0] - v[0] * s[2];
        U[2] += v[0] * s[1] - v[1] * s[0];
        X[0] += w * U[0];
        X[1] += w * U[1];
        X[2] += w * U[2];
        const size_t o = ((size_t)p * n_steps + k) * 3;
        x_out[o] = X[0];
        x_out[o + 1] = X[1];
        x_out[o + 2] = X[2];
        u_out[o] = U[0];
        u_out[o + 1] = U[1];
        u_out[o + 2] = U[2];
    }
    x[3 * p] = X[0];
    x[3 * p + 1] = X[1];
    x[3 * p + 2] = X[2];
    u[3 * p] = U[0];
    u[3 * p + 1] = U[1];
    u[3 * p + 2] = U[2];
}

}  // namespace

cudaError_t launch_push_boris(int n_part, int n_steps, double dt, const double* B, double qm, double* x, double* u,
                              double* x_out, double* u_out, cudaStream_t s)
{
    if (n_part <= 0 || n_steps <= 0) return cudaSuccess;
    k_push_boris<<<(n_part + 127) / 128, 128, 0, s>>>(n_part, n_steps, dt, B[0], B[1], B[2], qm, x, u, x_out, u_out);
    return cudaGetLastError();
}

}  // namespace rd
