"""Second, independent transcription of Algorithms 1 and 2, in pure Python, for tiny inputs.

TEST INFRASTRUCTURE ONLY.  It follows the two algorithms step by step, in absolute detector
time, with a time grid t_array, so that it checks the C oracle (which evaluates the same
integral in bin units, cell by cell) through a different route.  Readings of the paper used:
  * Algorithm 2's iterator starts at the previous slot (the printed "t_slot,prev" is read as
    n_slot,prev, as the text that follows the algorithm describes it);
  * deposits accumulate (+=): Section 3.2 repeats the interpolation for every step and every
    particle and the detector holds their sum;
  * the closing deposit uses (t_det - t_tmp)/dt_det, t_tmp being t_det,prev when the while loop
    did not run (the printed t_array[n_slot] would count [t_array[n_slot], t_det,prev] twice);
  * the window test of Algorithm 1 is applied by clipping the interval to the detector grid;
  * n points from the particle to the cell (Section 2 text; Algorithm 1 prints the reverse).
"""
from __future__ import annotations

import math


def _sub(a, b):
    return [a[0] - b[0], a[1] - b[1], a[2] - b[2]]


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def lienard_wiechert(n, R, beta, beta_dot, q, flags=3):
    """Eq. 1 (e -> q, c = 1): returns E and B = n x E as lists."""
    kappa = 1.0 - _dot(beta, n)
    gamma2_inv = 1.0 - _dot(beta, beta)
    nmb = _sub(n, beta)
    E = [0.0, 0.0, 0.0]
    if flags & 1:
        s = q * gamma2_inv / (kappa ** 3 * R * R)
        E = [E[i] + s * nmb[i] for i in range(3)]
    if flags & 2:
        acc = _cross(n, _cross(nmb, beta_dot))
        s = q / (kappa ** 3 * R)
        E = [E[i] + s * acc[i] for i in range(3)]
    return E, _cross(n, E)


def slot(t_array, t):
    """Index i with t_array[i] <= t < t_array[i+1] on a uniform grid."""
    return int(math.floor((t - t_array[0]) / (t_array[1] - t_array[0])))


def radiation_interpolator(cell_row, field6, t_det, t_det_prev, t_array, dt_det):
    """Algorithm 2 for one cell: cell_row is a list of n_bins 6-lists (E then B)."""
    n_bins = len(t_array) - 1
    lo, hi = t_array[0], t_array[n_bins]
    if t_det <= lo or t_det_prev >= hi:
        return
    t_det_prev = max(t_det_prev, lo)
    t_det = min(t_det, hi)
    n_slot = min(slot(t_array, t_det), n_bins)
    n_slot_prev = slot(t_array, t_det_prev)
    n_itr = n_slot_prev
    t_tmp = t_det_prev
    while n_itr < n_slot:
        scale = (t_array[n_itr + 1] - t_tmp) / dt_det
        for i in range(6):
            cell_row[n_itr][i] += field6[i] * scale
        n_itr += 1
        t_tmp = t_array[n_itr]
    scale = (t_det - t_tmp) / dt_det
    if n_itr < n_bins and scale != 0.0:
        for i in range(6):
            cell_row[n_itr][i] += field6[i] * scale


def radiation_calculator(x, u, q, t0, dt, cells, t_min, dt_det, n_bins, cell_t0=None, flags=3):
    """Algorithm 1: particles outer, cells inner.  x, u: nested lists [n_part][n_samples][3].

    Returns det[cell][bin][6]."""
    n_cells = len(cells)
    det = [[[0.0] * 6 for _ in range(n_bins)] for _ in range(n_cells)]
    grids = []
    for j in range(n_cells):
        T0 = t_min + (cell_t0[j] if cell_t0 is not None else 0.0)
        grids.append([T0 + i * dt_det for i in range(n_bins + 1)])
    for p in range(len(x)):
        up = u[p][0]
        g = math.sqrt(_dot(up, up) + 1.0)
        beta_prev = [c / g for c in up]
        for k in range(1, len(x[p])):
            t = t0 + k * dt
            pk = u[p][k]
            g = math.sqrt(_dot(pk, pk) + 1.0)
            beta = [c / g for c in pk]
            beta_dot = [(beta[i] - beta_prev[i]) / dt for i in range(3)]
            for j in range(n_cells):
                d = _sub(cells[j], x[p][k])
                R = math.sqrt(_dot(d, d))
                n = [c / R for c in d]
                dp = _sub(cells[j], x[p][k - 1])
                R_prev = math.sqrt(_dot(dp, dp))
                t_det = R + t
                t_det_prev = R_prev + t - dt
                E, B = lienard_wiechert(n, R, beta, beta_dot, q[p], flags)
                radiation_interpolator(det[j], E + B, t_det, t_det_prev, grids[j], dt_det)
            beta_prev = beta
    return det
