"""The oracle pins must catch plausible mistakes.

Each case plants one mistake in a scratch copy of the oracle source (on the CPU), rebuilds it,
runs the pin suite against the copy in a subprocess and requires at least one pin to fail.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    # n from the cell to the particle (the sign printed in Algorithm 1)
    "n_reversed": ("SCALAR d[3] = {P[0] - x[0], P[1] - x[1], P[2] - x[2]};",
                   "SCALAR d[3] = {x[0] - P[0], x[1] - P[1], x[2] - P[2]};"),
    "no_inv_gamma2": ("SCALAR c = q * inv_gamma2 / (k3 * R * R);", "SCALAR c = q / (k3 * R * R);"),
    "kappa_squared": ("SCALAR k3 = kappa * kappa * kappa;", "SCALAR k3 = kappa * kappa;"),
    "cross_transposed": ("SCALAR w[3] = {nb[1] * bdot[2] - nb[2] * bdot[1],",
                         "SCALAR w[3] = {-nb[1] * bdot[2] + nb[2] * bdot[1],"),
    "advanced_time": ("SCALAR tdet = tk + R;", "SCALAR tdet = tk - R;"),
    "B_reversed": ("B[0] = n[1] * E[2] - n[2] * E[1];", "B[0] = -n[1] * E[2] + n[2] * E[1];"),
    "bin_off_by_one": ("for (int i = 0; i < 6; ++i) row[6 * b + i] += F[i] * w;",
                       "for (int i = 0; i < 6; ++i) row[6 * (b + (b + 1 < n_bins)) + i] += F[i] * w;"),
    "betadot_over_2dt": ("for (int i = 0; i < 3; ++i) bdot[i] = (beta[i] - beta_prev[i]) / dt;",
                         "for (int i = 0; i < 3; ++i) bdot[i] = (beta[i] - beta_prev[i]) / (2.0 * dt);"),
    "field_at_previous_sample": ("FN(lw_field)(xk, beta, bdot, P, q, flags, E, B);",
                                 "FN(lw_field)(xk - 3, beta, bdot, P, q, flags, E, B);"),
    "near_sign": ("for (int i = 0; i < 3; ++i) E[i] += c * nb[i];",
                  "for (int i = 0; i < 3; ++i) E[i] -= c * nb[i];"),
    "far_over_R2": ("SCALAR c = q / (k3 * R);", "SCALAR c = q / (k3 * R * R);"),
    "dropped_beta_z": ("SCALAR inv_gamma2 = 1.0 - (beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2]);",
                       "SCALAR inv_gamma2 = 1.0 - (beta[0] * beta[0] + beta[1] * beta[1]);"),
    "overlap_from_bin_start": ("SCALAR s = (ra > (double)b) ? a : (SCALAR)(double)b;",
                               "SCALAR s = (SCALAR)(double)b;"),
    # far-field limit: Eq. 3 with the projection added instead of subtracted; kappa^2
    "farfield_time_sign": ("SCALAR t_ff = (tk + Rc) - xn;", "SCALAR t_ff = (tk + Rc) + xn;"),
    "farfield_kappa_squared": ("SCALAR s = (flags & 2) ? q / (kap * kap * kap * Rc) : 0.0;",
                               "SCALAR s = (flags & 2) ? q / (kap * kap * Rc) : 0.0;"),
    # linear-in-time interpolation: ramp weight doubled; the two end fields exchanged
    "linear_ramp_doubled": ("SCALAR ramp = ((u1 - a) * (u1 - a) - (u0 - a) * (u0 - a)) / (2.0 * (c - a));",
                            "SCALAR ramp = ((u1 - a) * (u1 - a) - (u0 - a) * (u0 - a)) / (c - a);"),
    "linear_ends_exchanged": ("row[6 * b + i] += F0[i] * len + (F1[i] - F0[i]) * ramp;",
                              "row[6 * b + i] += F1[i] * len + (F0[i] - F1[i]) * ramp;"),
    # quadratic-in-time interpolation: the curvature term's sign; the second divided difference over
    # the interval alone instead of the span of the three points
    "quadratic_curvature_sign": ("row[6 * b + i] += Fa[i] * len + D1[i] * sq + D2[i] * cu;",
                                 "row[6 * b + i] += Fa[i] * len + D1[i] * sq - D2[i] * cu;"),
    "quadratic_divided_difference": ("D2[i] = (D1[i] - D0) / (L + h);", "D2[i] = (D1[i] - D0) / L;"),
    # held-previous field: the current sample's field held instead
    "hold_previous_uses_current": ("clipped += FN(deposit_interval)(a, c, Fprev, n_bins, row);",
                                   "clipped += FN(deposit_interval)(a, c, F, n_bins, row);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(tmp_path, name):
    old, new = MUTATIONS[name]
    for d in ("oracle", "tests", "paper_2302_14812_gb300"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_build", "__pycache__", "*.so"))
    core = tmp_path / "oracle" / "rd_oracle_core.h"
    src = core.read_text()
    assert src.count(old) == 1, name
    core.write_text(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py"], cwd=tmp_path, capture_output=True, text=True,
                       timeout=600)
    tail = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else r.stderr[-400:]
    assert r.returncode != 0 and "failed" in tail, f"{name}: pins did not catch it ({tail})"
