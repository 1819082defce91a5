"""Seeded synthetic inputs: particle trajectories and virtual-detector geometries.

This module is the only code shared by the CUDA path's tests/benchmark and the
FP64 oracle.  It holds no part of the radiation method itself (no
Lienard-Wiechert field, no arrival time, no deposit): it only produces the
inputs the method consumes, in the units the paper uses (c = 1, momenta
u = p/(m c) = gamma*beta, Section 3.1 / Algorithm 1 inputs).

Layouts (all float64, C-contiguous):
  trajectories  x, u : [n_part][n_samples][3], sample k at t_k = t0 + k*dt
                 q    : [n_part] signed charge (macro-particle charge N*q, Section 4.2)
  detector      pix_pos : [n_pix][3] pixel (cell) centres
                 pix_t0  : [n_pix] per-pixel time origin or None
                 bin b of pixel j covers [t_min + pix_t0[j] + b*dt_det, ... + dt_det)

Workload shapes follow the paper's examples (Section 3.3 helical, Section 4
sinusoidal benchmark, Section 5 plasma mirror): see the individual generators.
Positions are obtained from analytic velocities by per-step Gauss-Legendre
quadrature (8 nodes), accurate to FP64 rounding for these smooth motions.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

RD_NEAR = 1
RD_FAR = 2
RD_FARFIELD = 4
RD_LINEAR = 8
RD_HOLD_PREV = 16
RD_QUADRATIC = 32


@dataclasses.dataclass
class Trajectories:
    x: np.ndarray            # [n_part][n_samples][3]
    u: np.ndarray            # [n_part][n_samples][3]
    q: np.ndarray            # [n_part]
    t0: float
    dt: float

    @property
    def n_part(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_samples(self) -> int:
        return int(self.x.shape[1])

    @property
    def n_steps(self) -> int:
        return self.n_samples - 1

    def subset(self, idx) -> "Trajectories":
        idx = np.asarray(idx)
        return Trajectories(np.ascontiguousarray(self.x[idx]), np.ascontiguousarray(self.u[idx]),
                            np.ascontiguousarray(self.q[idx]), self.t0, self.dt)

    def steps(self, k0: int, k1: int) -> "Trajectories":
        """Samples k0..k1 inclusive, as a trajectory of its own (start time shifted)."""
        return Trajectories(np.ascontiguousarray(self.x[:, k0:k1 + 1]),
                            np.ascontiguousarray(self.u[:, k0:k1 + 1]),
                            self.q.copy(), self.t0 + k0 * self.dt, self.dt)


@dataclasses.dataclass
class Detector:
    pix_pos: np.ndarray                  # [n_pix][3]
    pix_t0: Optional[np.ndarray]         # [n_pix] or None
    t_min: float
    dt_det: float
    n_bins: int
    flags: int = RD_NEAR | RD_FAR
    shape: tuple = ()                    # logical (rows, cols) of the pixel grid, informational

    @property
    def n_pix(self) -> int:
        return int(self.pix_pos.shape[0])

    def subset(self, idx) -> "Detector":
        idx = np.asarray(idx)
        t0 = None if self.pix_t0 is None else np.ascontiguousarray(self.pix_t0[idx])
        return Detector(np.ascontiguousarray(self.pix_pos[idx]), t0, self.t_min, self.dt_det,
                        self.n_bins, self.flags, (len(idx),))


# ----------------------------------------------------------------------------------------
# quadrature helper: positions from analytic velocities
# ----------------------------------------------------------------------------------------
_GL_X, _GL_W = np.polynomial.legendre.leggauss(8)


def _integrate_positions(beta_fn: Callable[[np.ndarray], np.ndarray], x0: np.ndarray,
                         t0: float, dt: float, n_steps: int) -> np.ndarray:
    """x_k = x0 + int_{t0}^{t_k} beta(t) dt for k = 0..n_steps.

    beta_fn(t) takes t of shape [n_part][m] and returns [n_part][m][3].
    """
    n_part = x0.shape[0]
    k = np.arange(n_steps, dtype=np.float64)
    # nodes inside step k: t0 + dt*(k + (1+xi)/2)
    tn = t0 + dt * (k[:, None] + 0.5 * (1.0 + _GL_X[None, :]))          # [S][8]
    out = np.empty((n_part, n_steps + 1, 3))
    out[:, 0] = x0
    chunk = max(1, int(2_000_000 // max(1, n_steps * 8)))
    for p0 in range(0, n_part, chunk):
        p1 = min(n_part, p0 + chunk)
        b = beta_fn(np.broadcast_to(tn.reshape(1, -1), (p1 - p0, tn.size)), slice(p0, p1))
        b = b.reshape(p1 - p0, n_steps, 8, 3)
        inc = 0.5 * dt * np.einsum("psnc,n->psc", b, _GL_W)
        out[p0:p1, 1:] = x0[p0:p1, None, :] + np.cumsum(inc, axis=1)
    return out


# ----------------------------------------------------------------------------------------
# trajectories
# ----------------------------------------------------------------------------------------
def circular_orbit(gamma: float = 5.0, radius: float = 1.0, n_steps: int = 2000,
                   dt_frac: float = 0.01, q: float = -1.0, phase0: float = 0.0,
                   t0: float = 0.0) -> Trajectories:
    """One charge on a circular orbit in the x-y plane (synchrotron test).

    Position and momentum are analytic at every sample: x = r(cos w t', sin w t', 0),
    u = gamma*beta*(-sin w t', cos w t', 0) with t' = t + phase0/w, w = beta/r.
    dt = dt_frac * orbit period.
    """
    beta = math.sqrt(1.0 - 1.0 / gamma ** 2)
    w0 = beta / radius
    period = 2.0 * math.pi / w0
    dt = dt_frac * period
    t = t0 + dt * np.arange(n_steps + 1)
    ph = w0 * t + phase0
    x = np.stack([radius * np.cos(ph), radius * np.sin(ph), np.zeros_like(ph)], axis=-1)
    u = gamma * beta * np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], axis=-1)
    return Trajectories(x[None].copy(), u[None].copy(), np.array([q]), t0, dt)


def helical_orbit(gamma: float = 57.3, K: float = 0.8, omega0: float = 1.0, n_steps: int = 400,
                  dt: float = 0.1, q: float = -1.0, t0: float = 0.0) -> Trajectories:
    """One charge on a helix along +x (Section 3.3 example: gamma 57.3, K = gamma r0 omega0 = 0.8,
    omega0 = 1, dt = 0.1).  Analytic at every sample: x = (beta_x t, r0 cos w t, r0 sin w t),
    beta = (beta_x, -r0 w sin w t, r0 w cos w t), r0 = K / (gamma w), beta_x from gamma."""
    b_perp = K / gamma
    r0 = b_perp / omega0
    b_x = math.sqrt(1.0 - 1.0 / gamma ** 2 - b_perp ** 2)
    t = t0 + dt * np.arange(n_steps + 1)
    ph = omega0 * t
    x = np.stack([b_x * t, r0 * np.cos(ph), r0 * np.sin(ph)], axis=-1)
    u = gamma * np.stack([np.full_like(ph, b_x), -b_perp * np.sin(ph), b_perp * np.cos(ph)], axis=-1)
    return Trajectories(x[None].copy(), u[None].copy(), np.array([q]), t0, dt)


def boris_uniform_field(x0: np.ndarray, u0: np.ndarray, n_steps: int, dt: float, B, qm: float,
                        q: float = -1.0, t0: float = 0.0) -> Trajectories:
    """Charges pushed by the Boris method (Boris 1970) in a uniform magnetic field B (c = 1, qm the
    charge-to-mass ratio): per step t = (qm dt/2) B/gamma, s = 2t/(1+|t|^2), u' = u + u x t,
    u <- u + u' x s, x <- x + dt u/gamma.  x0, u0: [n_part][3]; samples k = 0..n_steps."""
    B = np.asarray(B, dtype=np.float64)
    x = np.array(x0, dtype=np.float64)
    u = np.array(u0, dtype=np.float64)
    g = np.sqrt(1.0 + np.sum(u * u, axis=1))
    t = (0.5 * qm * dt / g)[:, None] * B[None, :]
    s = (2.0 / (1.0 + np.sum(t * t, axis=1)))[:, None] * t
    w = (dt / g)[:, None]
    X = np.empty((x.shape[0], n_steps + 1, 3))
    U = np.empty_like(X)
    X[:, 0], U[:, 0] = x, u
    for k in range(n_steps):
        v = u + np.cross(u, t)
        u = u + np.cross(v, s)
        x = x + w * u
        X[:, k + 1], U[:, k + 1] = x, u
    return Trajectories(X, U, np.full(x.shape[0], q), t0, dt)


def circular_ensemble(n_part: int, n_steps: int, gamma: float = 5.0, radius: float = 1.0,
                      n_orbits: float = 4.0, seed: int = 5, q: float = -1.0) -> Trajectories:
    """n_part charges on the same circular orbit (x-y plane) with random phases."""
    rng = np.random.default_rng(seed)
    ph0 = rng.uniform(0.0, 2.0 * math.pi, n_part)
    beta = math.sqrt(1.0 - 1.0 / gamma ** 2)
    w0 = beta / radius
    dt = n_orbits * (2.0 * math.pi / w0) / n_steps
    ph = w0 * (dt * np.arange(n_steps + 1))[None, :] + ph0[:, None]
    z = np.zeros_like(ph)
    x = np.stack([radius * np.cos(ph), radius * np.sin(ph), z], axis=-1)
    u = gamma * beta * np.stack([-np.sin(ph), np.cos(ph), z], axis=-1)
    return Trajectories(x, u, np.full(n_part, q), 0.0, dt)


def undulator_params(gamma: float, K: float, lambda_u: float = 1.0):
    """Mean longitudinal velocity and angular frequency of a planar-undulator orbit."""
    beta_z_bar = math.sqrt(1.0 - (1.0 + 0.5 * K * K) / gamma ** 2)
    k_u = 2.0 * math.pi / lambda_u
    return beta_z_bar, k_u * beta_z_bar


def undulator_ensemble(n_part: int = 1000, gamma: float = 20.0, K: float = 1.0,
                       n_periods: float = 10.0, n_steps: int = 4000, lambda_u: float = 1.0,
                       sigma_offset: float = 1e-3, seed: int = 2, q: float = -1.0,
                       k_scale: Optional[np.ndarray] = None, phase_shift: Optional[np.ndarray] = None
                       ) -> Trajectories:
    """Planar-undulator electrons moving along +z, wiggling in y (Section 4 benchmark shape).

    beta_y = (K_i/gamma) sin(w_u t + phi_i), beta_x = 0, |beta| fixed by gamma (a static magnetic
    field does no work); phi_i ~ U[0, 2pi); transverse offsets (x0, y0) ~ N(0, sigma_offset).
    k_scale / phase_shift optionally perturb K_i and phi_i per particle (used to build targets).
    """
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2.0 * math.pi, n_part)
    off = rng.normal(0.0, sigma_offset, (n_part, 2))
    if phase_shift is not None:
        phi = phi + phase_shift
    Ki = np.full(n_part, K) if k_scale is None else K * np.asarray(k_scale, dtype=np.float64)
    bz_bar, w_u = undulator_params(gamma, K, lambda_u)
    t_total = n_periods * lambda_u / bz_bar
    dt = t_total / n_steps
    t0 = 0.0
    g2 = gamma * gamma

    def beta_fn(t, sl):
        by = (Ki[sl, None] / gamma) * np.sin(w_u * t + phi[sl, None])
        bz = np.sqrt(1.0 - 1.0 / g2 - by * by)
        return np.stack([np.zeros_like(by), by, bz], axis=-1)

    x0 = np.zeros((n_part, 3))
    x0[:, 0] = off[:, 0]
    x0[:, 1] = off[:, 1]
    x = _integrate_positions(beta_fn, x0, t0, dt, n_steps)
    t = t0 + dt * np.arange(n_steps + 1)
    u = gamma * beta_fn(np.broadcast_to(t[None, :], (n_part, t.size)), slice(0, n_part))
    return Trajectories(x, u, np.full(n_part, q), t0, dt)


def plasma_mirror_surface(n_part: int = 100_000, n_steps: int = 10_000, n_periods: float = 12.0,
                          a0: float = 5.0, n_harm: int = 20, jitter: float = 0.01,
                          half_width_lambda: float = 3.0, phase_slope: float = 0.5,
                          seed: int = 3, q: float = -1.0, particles: Optional[slice] = None
                          ) -> Trajectories:
    """Electrons of a plasma-mirror surface driven by a relativistic laser (Section 5 shape).

    Laser frequency w = 1 (period T0 = 2pi, lambda0 = 2pi), n_periods under a sin^2 envelope.
    Longitudinal momentum u_x = a_i env(t) s(w t + phi_i)/max|s| with
    s(th) = cos th + sum_{n=2}^{n_harm} n^-2 cos(n th)  (harmonics decaying as n^-2);
    transverse u_z = 0.5 a_i env(t) sin(w t + phi_i) (figure-8-like); u_y = 0.
    a_i = a0 (1 + jitter*N(0,1)); phi_i = phase_slope * y_i (linear in transverse position);
    (y_i, z_i) ~ U[-3 lambda0, 3 lambda0]^2; x_i0 ~ U[0, 0.05 lambda0] (thin surface layer).
    `particles` selects a contiguous slice of the ensemble (same seed => same particles).
    """
    rng = np.random.default_rng(seed)
    lam0 = 2.0 * math.pi
    yz = rng.uniform(-half_width_lambda * lam0, half_width_lambda * lam0, (n_part, 2))
    xs = rng.uniform(0.0, 0.05 * lam0, n_part)
    amp = a0 * (1.0 + jitter * rng.standard_normal(n_part))
    if particles is not None:
        yz, xs, amp = yz[particles], xs[particles], amp[particles]
    n_sel = yz.shape[0]
    phi = phase_slope * yz[:, 0]
    harm = np.arange(2, n_harm + 1, dtype=np.float64)
    s_max = 1.0 + float(np.sum(harm ** -2.0))          # s attains its maximum at th = 0
    t_total = n_periods * 2.0 * math.pi
    dt = t_total / n_steps

    def s_fn(th):
        acc = np.cos(th)
        for n in harm:
            acc = acc + np.cos(n * th) / (n * n)
        return acc

    def mom(t, sl):
        env = np.sin(math.pi * np.clip(t / t_total, 0.0, 1.0)) ** 2
        th = t + phi[sl, None]
        ux = amp[sl, None] * env * s_fn(th) / s_max
        uz = 0.5 * amp[sl, None] * env * np.sin(th)
        return np.stack([ux, np.zeros_like(ux), uz], axis=-1)

    def beta_fn(t, sl):
        uu = mom(t, sl)
        return uu / np.sqrt(1.0 + np.sum(uu * uu, axis=-1, keepdims=True))

    x0 = np.stack([xs, yz[:, 0], yz[:, 1]], axis=-1)
    x = _integrate_positions(beta_fn, x0, 0.0, dt, n_steps)
    t = dt * np.arange(n_steps + 1)
    u = mom(np.broadcast_to(t[None, :], (n_sel, t.size)), slice(0, n_sel))
    return Trajectories(x, u, np.full(n_sel, q), 0.0, dt)


def plasma_mirror_surface_torch(particles: slice, n_part: int = 100_000, n_steps: int = 10_000,
                                n_periods: float = 12.0, a0: float = 5.0, n_harm: int = 20, jitter: float = 0.01,
                                half_width_lambda: float = 3.0, phase_slope: float = 0.5, seed: int = 3,
                                q: float = -1.0, device="cuda", sub: int = 1000):
    """plasma_mirror_surface(..., particles=particles) evaluated with PyTorch in FP64 on `device`:
    the same seeded particle parameters and formulas, positions by the same 8-node Gauss-Legendre
    quadrature (summed on the device, so values agree with the numpy generator to rounding).
    For ensembles too large to generate on the host.  Returns (x, u, q) tensors and (t0, dt)."""
    import torch
    rng = np.random.default_rng(seed)
    lam0 = 2.0 * math.pi
    yz = rng.uniform(-half_width_lambda * lam0, half_width_lambda * lam0, (n_part, 2))[particles]
    xs = rng.uniform(0.0, 0.05 * lam0, n_part)[particles]
    amp = (a0 * (1.0 + jitter * rng.standard_normal(n_part)))[particles]
    n_sel = yz.shape[0]
    f64 = dict(dtype=torch.float64, device=device)
    s_max = 1.0 + float(np.sum(np.arange(2, n_harm + 1, dtype=np.float64) ** -2.0))
    t_total = n_periods * 2.0 * math.pi
    dt = t_total / n_steps
    t = dt * torch.arange(n_steps + 1, **f64)
    k = torch.arange(n_steps, **f64)
    tn = (dt * (k[:, None] + 0.5 * (1.0 + torch.tensor(_GL_X, **f64)[None, :]))).reshape(-1)   # [S*8]
    glw = torch.tensor(_GL_W, **f64)

    def s_fn(th):
        acc = torch.cos(th)
        for n in range(2, n_harm + 1):
            acc = acc + torch.cos(n * th) / float(n * n)
        return acc

    def mom(tt, ph, a):
        env = torch.sin(math.pi * torch.clamp(tt / t_total, 0.0, 1.0)) ** 2
        th = tt[None, :] + ph[:, None]
        ux = a[:, None] * env[None, :] * s_fn(th) / s_max
        uz = 0.5 * a[:, None] * env[None, :] * torch.sin(th)
        return torch.stack([ux, torch.zeros_like(ux), uz], dim=-1)

    x = torch.empty((n_sel, n_steps + 1, 3), **f64)
    u = torch.empty((n_sel, n_steps + 1, 3), **f64)
    for p0 in range(0, n_sel, sub):
        p1 = min(n_sel, p0 + sub)
        ph = torch.tensor(phase_slope * yz[p0:p1, 0], **f64)
        a = torch.tensor(amp[p0:p1], **f64)
        u[p0:p1] = mom(t, ph, a)
        un = mom(tn, ph, a)
        b = un / torch.sqrt(1.0 + torch.sum(un * un, dim=-1, keepdim=True))
        inc = 0.5 * dt * torch.einsum("psnc,n->psc", b.reshape(p1 - p0, n_steps, 8, 3), glw)
        x0 = torch.tensor(np.stack([xs[p0:p1], yz[p0:p1, 0], yz[p0:p1, 1]], axis=-1), **f64)
        x[p0:p1, 0] = x0
        x[p0:p1, 1:] = x0[:, None, :] + torch.cumsum(inc, dim=1)
        del un, b, inc
    return x, u, torch.full((n_sel,), q, **f64), (0.0, dt)


def oscillator_ensemble(n_part: int, n_steps: int, amp_range=(0.1, 2.0), omega: float = 1.0,
                        n_periods: float = 6.0, seed: int = 4, q: float = -1.0) -> Trajectories:
    """Linear relativistic oscillators along x: u_x = a_i sin(w t + phi_i), random a_i, phi_i."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(amp_range[0], amp_range[1], n_part)
    phi = rng.uniform(0.0, 2.0 * math.pi, n_part)
    off = rng.normal(0.0, 1e-2, (n_part, 3))
    t_total = n_periods * 2.0 * math.pi / omega
    dt = t_total / n_steps

    def mom(t, sl):
        ux = a[sl, None] * np.sin(omega * t + phi[sl, None])
        return np.stack([ux, np.zeros_like(ux), np.zeros_like(ux)], axis=-1)

    def beta_fn(t, sl):
        uu = mom(t, sl)
        return uu / np.sqrt(1.0 + np.sum(uu * uu, axis=-1, keepdims=True))

    x = _integrate_positions(beta_fn, off, 0.0, dt, n_steps)
    t = dt * np.arange(n_steps + 1)
    u = mom(np.broadcast_to(t[None, :], (n_part, t.size)), slice(0, n_part))
    return Trajectories(x, u, np.full(n_part, q), 0.0, dt)


def uniform_motion(n_part: int, n_steps: int, dt: float, speed: float = 0.9,
                   seed: int = 11, q: float = 1.0) -> Trajectories:
    """Charges in uniform straight-line motion (constant u => zero acceleration field)."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n_part, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    gam = 1.0 / math.sqrt(1.0 - speed * speed)
    beta = speed * d
    x0 = rng.normal(0.0, 0.1, (n_part, 3))
    t = dt * np.arange(n_steps + 1)
    x = x0[:, None, :] + beta[:, None, :] * t[None, :, None]
    u = np.broadcast_to((gam * beta)[:, None, :], x.shape).copy()
    return Trajectories(x, u, np.full(n_part, q), 0.0, dt)


def random_smooth(n_part: int, n_steps: int, dt: float, max_u: float = 3.0,
                  seed: int = 7, n_modes: int = 3, q_range=(-1.0, 1.0)) -> Trajectories:
    """Random smooth bounded motions (sums of a few sinusoids per momentum component).

    Used for small parity cases: every sample carries a different beta and acceleration.
    """
    rng = np.random.default_rng(seed)
    amp = rng.uniform(-1.0, 1.0, (n_part, 3, n_modes)) * (max_u / n_modes)
    om = rng.uniform(0.2, 2.0, (n_part, 3, n_modes))
    ph = rng.uniform(0.0, 2.0 * math.pi, (n_part, 3, n_modes))
    drift = rng.uniform(-1.0, 1.0, (n_part, 3)) * max_u * 0.5
    qv = rng.uniform(q_range[0], q_range[1], n_part)

    def mom(t, sl):
        tt = t[..., None, None]
        val = np.sum(amp[sl, None] * np.sin(om[sl, None] * tt + ph[sl, None]), axis=-1)
        return val + drift[sl, None, :]

    def beta_fn(t, sl):
        uu = mom(t, sl)
        return uu / np.sqrt(1.0 + np.sum(uu * uu, axis=-1, keepdims=True))

    x0 = rng.normal(0.0, 0.2, (n_part, 3))
    x = _integrate_positions(beta_fn, x0, 0.0, dt, n_steps)
    t = dt * np.arange(n_steps + 1)
    u = mom(np.broadcast_to(t[None, :], (n_part, t.size)), slice(0, n_part))
    return Trajectories(x, u, qv, 0.0, dt)


# ----------------------------------------------------------------------------------------
# detectors
# ----------------------------------------------------------------------------------------
def arc_detector(n_pix: int, radius: float, dphi: float, phi0: float = 0.0) -> np.ndarray:
    """Pixels on a circle of given radius in the x-y plane at angles phi0 + j*dphi."""
    ph = phi0 + dphi * np.arange(n_pix)
    return np.stack([radius * np.cos(ph), radius * np.sin(ph), np.zeros_like(ph)], axis=-1)


def spherical_cap(n_side: int, radius: float, half_angle: float, axis: int = 2) -> np.ndarray:
    """n_side x n_side pixels on a sphere around the origin, centred on coordinate `axis`.

    Pixel (i, j) points along (sin th_i, sin th_j, sqrt(1 - sin^2 th_i - sin^2 th_j)) with
    th spanning [-half_angle, half_angle] at cell centres (Section 3.1 spherical detector).
    """
    th = -half_angle + (np.arange(n_side) + 0.5) * (2.0 * half_angle / n_side)
    a, b = np.meshgrid(np.sin(th), np.sin(th), indexing="ij")
    c2 = 1.0 - a * a - b * b
    if np.any(c2 <= 0.0):
        raise ValueError("half_angle too large: corner cells would leave the sphere")
    c = np.sqrt(c2)
    dirs = np.zeros((n_side, n_side, 3))
    others = [i for i in range(3) if i != axis]
    dirs[..., others[0]] = a
    dirs[..., others[1]] = b
    dirs[..., axis] = c
    return (radius * dirs).reshape(-1, 3)


def cartesian_plane(n_side: int, x_plane: float, half_width: float) -> np.ndarray:
    """n_side x n_side pixels on the plane x = x_plane, y,z in [-half_width, half_width]."""
    s = -half_width + (np.arange(n_side) + 0.5) * (2.0 * half_width / n_side)
    yy, zz = np.meshgrid(s, s, indexing="ij")
    return np.stack([np.full_like(yy, x_plane), yy, zz], axis=-1).reshape(-1, 3)


# ----------------------------------------------------------------------------------------
# the paper-shaped configurations
# ----------------------------------------------------------------------------------------
def config_circular(n_steps: int = 2000, n_pix: int = 64, n_bins: int = 1024,
                    gamma: float = 5.0, radius: float = 1.0, distance: float = 1e3):
    """Single electron on a circular orbit (gamma 5, r 1, dt = 0.01 period), 64-pixel arc
    in the orbit plane at 1e3 radii, pixel j at azimuth j*w0*2dt, 1024 bins of 2dt."""
    tr = circular_orbit(gamma=gamma, radius=radius, n_steps=n_steps)
    beta = math.sqrt(1.0 - 1.0 / gamma ** 2)
    w0 = beta / radius
    dt_det = 2.0 * tr.dt
    span = n_bins * dt_det
    emit = n_steps * tr.dt + 2.0 * radius
    margin = 0.5 * (span - emit)
    t_min = tr.t0 + distance - radius - margin
    pos = arc_detector(n_pix, distance, w0 * 2.0 * tr.dt)
    det = Detector(pos, None, t_min, dt_det, n_bins, RD_NEAR | RD_FAR, (n_pix,))
    return tr, det


def axial_window(distance: float, t_total: float, beta_bar: float, theta_max: float,
                 transverse: float, n_bins: int):
    """(t_min, dt_det) of a window holding every arrival from charges drifting along the axis
    of a spherical cap: arrivals run from ~distance to distance + t_total(1 - beta_bar cos th),
    widened by the transverse excursion and a 2% margin."""
    lo = distance - transverse
    hi = distance + t_total * (1.0 - beta_bar * math.cos(theta_max)) + transverse
    pad = 0.02 * (hi - lo)
    lo -= pad
    hi += pad
    return lo, (hi - lo) / n_bins


def config_undulator(n_part: int = 1000, n_steps: int = 4000, n_side: int = 128,
                     n_bins: int = 2048, gamma: float = 20.0, K: float = 1.0,
                     n_periods: float = 10.0, distance: float = 1e4, seed: int = 2,
                     half_angle_gamma: float = 1.5, **kw):
    """Planar-undulator ensemble (gamma 20, K 1, 10 periods of lambda_u = 1), spherical cap of
    n_side^2 pixels at 1e4 periods spanning +-1.5/gamma, n_bins bins covering all arrivals."""
    tr = undulator_ensemble(n_part=n_part, gamma=gamma, K=K, n_periods=n_periods,
                            n_steps=n_steps, seed=seed, **kw)
    half = half_angle_gamma / gamma
    pos = spherical_cap(n_side, distance, half)
    bz_bar, w_u = undulator_params(gamma, K)
    theta_corner = math.asin(min(1.0, math.sqrt(2.0) * math.sin(half)))
    transverse = K / (gamma * w_u) + 6e-3
    t_min, dt_det = axial_window(distance, n_steps * tr.dt, bz_bar, theta_corner, transverse,
                                 n_bins)
    det = Detector(pos, None, t_min, dt_det, n_bins, RD_NEAR | RD_FAR, (n_side, n_side))
    return tr, det


def config_helical(n_side: int = 64, n_steps: int = 400, n_bins: int = 8192, gamma: float = 57.3, K: float = 0.8,
                   distance: float = 1e6, aperture: float = 0.1, dt_det: float = 1.33e-5):
    """Section 3.3 example: one electron on a helix along +x (gamma 57.3, K 0.8, omega0 = 1,
    dt = 0.1), spherical detector of n_side^2 cells spanning `aperture` rad around +x at R = 1e6,
    bins of 1.33e-5.  Each cell's time origin is its earliest arrival minus 20 bins."""
    tr = helical_orbit(gamma=gamma, K=K, n_steps=n_steps)
    pos = spherical_cap(n_side, distance, 0.5 * aperture, axis=0)
    k = np.arange(tr.n_samples)
    tk = tr.t0 + k * tr.dt
    first = np.array([np.min(tk + np.linalg.norm(p - tr.x[0], axis=1)) for p in pos])
    det = Detector(pos, first - 20.0 * dt_det - distance, distance, dt_det, n_bins, RD_NEAR | RD_FAR,
                   (n_side, n_side))
    return tr, det


def config_sinusoidal_benchmark(n_cells: int = 512, n_periods: float = 5.0, n_bins: int = 131072,
                                gamma: float = 50.0, K: float = 10.0, k_beta: float = 0.1, dt: float = 0.01,
                                distance: float = 1e5, aperture: float = 0.1):
    """Section 4 benchmark: one electron (gamma 50) on a sinusoidal trajectory with K = 10
    (r_beta = K/(gamma k_beta) = 2, k_beta = 0.1) stepped with dt = 0.01, moving along +z and
    oscillating in y; a line of a spherical detector at 1e5 in the x-z plane (the plane normal to
    the motion plane through the axis), `aperture` rad wide around +z, n_cells cells, n_bins bins
    of 2.98e-5.  Each cell's time origin is its earliest arrival minus 0.01."""
    lam = 2.0 * math.pi / k_beta
    bz, _ = undulator_params(gamma, K, lam)
    n_steps = int(round(n_periods * lam / bz / dt))
    tr = undulator_ensemble(n_part=1, gamma=gamma, K=K, n_periods=n_periods, n_steps=n_steps, lambda_u=lam,
                            sigma_offset=0.0, seed=1)
    tr.x[:, :, :2] -= tr.x[:, :1, :2]
    th = np.linspace(-0.5 * aperture, 0.5 * aperture, n_cells)
    pos = np.stack([distance * np.sin(th), np.zeros_like(th), distance * np.cos(th)], axis=1)
    k = np.arange(tr.n_samples)
    first = np.array([np.min(tr.t0 + k * tr.dt + np.linalg.norm(p - tr.x[0], axis=1)) for p in pos])
    det = Detector(pos, first - 0.01 - distance, distance, 2.98e-5, n_bins, RD_NEAR | RD_FAR, (n_cells,))
    return tr, det, th


def plasma_mirror_detector(dt: float, n_side: int = 256, n_bins: int = 4096) -> Detector:
    """Cartesian plane at x = -6.4 lambda0 spanning +-6.4 lambda0 (reflected direction of the
    plasma-mirror surface), pix_t0 = |x_pix| - reach, dt_det = 5 dt."""
    lam0 = 2.0 * math.pi
    pos = cartesian_plane(n_side, -6.4 * lam0, 6.4 * lam0)
    reach = math.sqrt(2.0) * 3.0 * lam0 + 0.1 * lam0 + 5.0    # slab half-diagonal + depth + margin
    pix_t0 = np.linalg.norm(pos, axis=1) - reach
    return Detector(pos, pix_t0, 0.0, 5.0 * dt, n_bins, RD_NEAR | RD_FAR, (n_side, n_side))


def config_plasma_mirror(n_part: int = 100_000, n_steps: int = 10_000, n_side: int = 256,
                         n_bins: int = 4096, particles: Optional[slice] = None, seed: int = 3):
    """Plasma-mirror-like surface (a0 5, 20 harmonics, 12 periods) and its detector
    (plasma_mirror_detector)."""
    tr = plasma_mirror_surface(n_part=n_part, n_steps=n_steps, particles=particles, seed=seed)
    return tr, plasma_mirror_detector(tr.dt, n_side, n_bins)


def batch_problems(n_problems: int = 64, seed: int = 4, scale: float = 1.0):
    """Uneven ensembles: type in {undulator, circular, oscillator}, particle count log-uniform
    in [100, 5e4], steps uniform in [500, 8000], square detectors of side 32/64/128 with
    16*side bins.  `scale` (<= 1) shrinks particle counts for quick cases.

    Returns a list of (kind, Trajectories, Detector)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_problems):
        kind = ["undulator", "circular", "oscillator"][int(rng.integers(0, 3))]
        n_p = int(round(math.exp(rng.uniform(math.log(100.0), math.log(5e4))) * scale))
        n_p = max(1, n_p)
        n_s = int(rng.integers(500, 8001))
        side = [32, 64, 128][int(rng.integers(0, 3))]
        n_b = 16 * side
        sub = int(rng.integers(0, 2 ** 31 - 1))
        if kind == "undulator":
            tr, det = config_undulator(n_part=n_p, n_steps=n_s, n_side=side, n_bins=n_b,
                                       gamma=float(rng.uniform(5.0, 30.0)), K=float(rng.uniform(0.3, 2.0)),
                                       n_periods=5.0, distance=1e3, seed=sub)
        elif kind == "circular":
            gam = float(rng.uniform(2.0, 8.0))
            tr = circular_ensemble(n_p, n_s, gamma=gam, n_orbits=4.0, seed=sub)
            pos = spherical_cap(side, 1e3, 0.6, axis=2)
            span = n_s * tr.dt + 2.0
            det = Detector(pos, None, 1e3 - 1.0 - 0.02 * span, 1.04 * span / n_b, n_b,
                           RD_NEAR | RD_FAR, (side, side))
        else:
            tr = oscillator_ensemble(n_part=n_p, n_steps=n_s, seed=sub)
            pos = spherical_cap(side, 1e3, 0.6, axis=1)
            reach = 3.0
            span = n_s * tr.dt + 2.0 * reach
            det = Detector(pos, None, 1e3 - reach - 0.02 * span, 1.04 * span / n_b, n_b,
                           RD_NEAR | RD_FAR, (side, side))
        out.append((kind, tr, det))
    return out


def _integrate_positions_torch(beta_fn, x0, dt: float, n_steps: int, sub: int = 512):
    """_integrate_positions with PyTorch in FP64 on x0's device: x_k = x0 + sum over steps of the
    8-node Gauss-Legendre quadrature of beta; beta_fn(t [m], rows slice) -> [rows][m][3]."""
    import torch
    f64 = dict(dtype=torch.float64, device=x0.device)
    n_part = x0.shape[0]
    k = torch.arange(n_steps, **f64)
    tn = (dt * (k[:, None] + 0.5 * (1.0 + torch.tensor(_GL_X, **f64)[None, :]))).reshape(-1)
    glw = torch.tensor(_GL_W, **f64)
    x = torch.empty((n_part, n_steps + 1, 3), **f64)
    x[:, 0] = x0
    for p0 in range(0, n_part, sub):
        p1 = min(n_part, p0 + sub)
        b = beta_fn(tn, slice(p0, p1))
        inc = 0.5 * dt * torch.einsum("psnc,n->psc", b.reshape(p1 - p0, n_steps, 8, 3), glw)
        x[p0:p1, 1:] = x0[p0:p1, None, :] + torch.cumsum(inc, dim=1)
        del b, inc
    return x


def batch_problems_torch(n_problems: int = 64, seed: int = 4, scale: float = 1.0, device="cuda"):
    """batch_problems(n_problems, seed, scale) with the trajectories generated by PyTorch in FP64 on
    `device` (the full-scale set holds ~1e11 FP64 values): the same seeded draws in the same order
    and the same formulas, positions by the same quadrature summed on the device, so values agree
    with the numpy generator to rounding.  Returns a list of (kind, (x, u, q, t0, dt), Detector)."""
    import torch
    f64 = dict(dtype=torch.float64, device=device)
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_problems):
        kind = ["undulator", "circular", "oscillator"][int(rng.integers(0, 3))]
        n_p = max(1, int(round(math.exp(rng.uniform(math.log(100.0), math.log(5e4))) * scale)))
        n_s = int(rng.integers(500, 8001))
        side = [32, 64, 128][int(rng.integers(0, 3))]
        n_b = 16 * side
        sub = int(rng.integers(0, 2 ** 31 - 1))
        if kind == "undulator":
            gamma = float(rng.uniform(5.0, 30.0))
            K = float(rng.uniform(0.3, 2.0))
            n_periods, distance, sigma = 5.0, 1e3, 1e-3
            r2 = np.random.default_rng(sub)
            phi = torch.tensor(r2.uniform(0.0, 2.0 * math.pi, n_p), **f64)
            off = r2.normal(0.0, sigma, (n_p, 2))
            bz_bar, w_u = undulator_params(gamma, K, 1.0)
            dt = n_periods / bz_bar / n_s
            g2 = gamma * gamma

            def beta_fn(t, sl, phi=phi, K=K, gamma=gamma, w_u=w_u, g2=g2):
                by = (K / gamma) * torch.sin(w_u * t[None, :] + phi[sl, None])
                bz = torch.sqrt(1.0 - 1.0 / g2 - by * by)
                return torch.stack([torch.zeros_like(by), by, bz], dim=-1)
            x0 = torch.zeros((n_p, 3), **f64)
            x0[:, 0] = torch.tensor(off[:, 0], **f64)
            x0[:, 1] = torch.tensor(off[:, 1], **f64)
            x = _integrate_positions_torch(beta_fn, x0, dt, n_s)
            t = dt * torch.arange(n_s + 1, **f64)
            u = torch.cat([gamma * beta_fn(t, slice(p0, min(n_p, p0 + 512))) for p0 in range(0, n_p, 512)])
            _, det = config_undulator(n_part=1, n_steps=n_s, n_side=side, n_bins=n_b, gamma=gamma, K=K,
                                      n_periods=n_periods, distance=distance, seed=sub)
            t0 = 0.0
        elif kind == "circular":
            gam = float(rng.uniform(2.0, 8.0))
            r2 = np.random.default_rng(sub)
            ph0 = torch.tensor(r2.uniform(0.0, 2.0 * math.pi, n_p), **f64)
            beta = math.sqrt(1.0 - 1.0 / gam ** 2)
            w0 = beta
            dt = 4.0 * (2.0 * math.pi / w0) / n_s
            ph = w0 * (dt * torch.arange(n_s + 1, **f64))[None, :] + ph0[:, None]
            z = torch.zeros_like(ph)
            x = torch.stack([torch.cos(ph), torch.sin(ph), z], dim=-1)
            u = gam * beta * torch.stack([-torch.sin(ph), torch.cos(ph), z], dim=-1)
            del ph, z
            pos = spherical_cap(side, 1e3, 0.6, axis=2)
            span = n_s * dt + 2.0
            det = Detector(pos, None, 1e3 - 1.0 - 0.02 * span, 1.04 * span / n_b, n_b, RD_NEAR | RD_FAR, (side, side))
            t0 = 0.0
        else:
            r2 = np.random.default_rng(sub)
            a = torch.tensor(r2.uniform(0.1, 2.0, n_p), **f64)
            phi = torch.tensor(r2.uniform(0.0, 2.0 * math.pi, n_p), **f64)
            off = torch.tensor(r2.normal(0.0, 1e-2, (n_p, 3)), **f64)
            dt = 6.0 * 2.0 * math.pi / n_s

            def mom(t, sl, a=a, phi=phi):
                ux = a[sl, None] * torch.sin(t[None, :] + phi[sl, None])
                return torch.stack([ux, torch.zeros_like(ux), torch.zeros_like(ux)], dim=-1)

            def beta_fn(t, sl, mom=mom):
                uu = mom(t, sl)
                return uu / torch.sqrt(1.0 + torch.sum(uu * uu, dim=-1, keepdim=True))
            x = _integrate_positions_torch(beta_fn, off, dt, n_s)
            t = dt * torch.arange(n_s + 1, **f64)
            u = torch.cat([mom(t, slice(p0, min(n_p, p0 + 512))) for p0 in range(0, n_p, 512)])
            pos = spherical_cap(side, 1e3, 0.6, axis=1)
            reach = 3.0
            span = n_s * dt + 2.0 * reach
            det = Detector(pos, None, 1e3 - reach - 0.02 * span, 1.04 * span / n_b, n_b, RD_NEAR | RD_FAR, (side, side))
            t0 = 0.0
        out.append((kind, (x, u, torch.full((n_p,), -1.0, **f64), t0, dt), det))
    return out


def deposits(tr: Trajectories, det: Detector) -> int:
    """Number of (particle, interval, pixel) triples: the unit of the throughput metric."""
    return int(tr.n_part) * int(tr.n_steps) * int(det.n_pix)
