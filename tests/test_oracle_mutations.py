"""The oracle's pins must catch plausible mistakes.

Each case compiles a copy of the oracle with ONE planted error (a flipped sign,
a wrong index or width, a dropped factor, a transposed operand) into a temporary
directory, runs the pin suite against it in a subprocess, and requires that the
suite fails.  Nothing here touches the real oracle library or a GPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ram_oracle.c")

MUTANTS = {
    "ppm_w2_sign": ("double w2 = -h0 * (hm + h0)", "double w2 = h0 * (hm + h0)"),
    "ppm_dq_width": ("(2.0 * a + b) / (b + c)", "(2.0 * a + b) / (a + c)"),
    "ppm_face_weight": ("h0 / (h0 + h1) * (q[ip] - q[i])", "h1 / (h0 + h1) * (q[ip] - q[i])"),
    "ppm_constraint_operand": ("L = 3.0 * Q - 2.0 * R;", "L = 3.0 * Q - 2.0 * L;"),
    "ppm_q6_sign": ("6.0 * Q - 3.0 * (L + R)", "6.0 * Q - 3.0 * (L - R)"),
    "ppm_dq_limiter_factor": ("if (2.0 * fabs(dn) < m) m = 2.0 * fabs(dn);",
                              "if (fabs(dn) < m) m = fabs(dn);"),
    "plm_harmonic_factor": ("2.0 * dl * dr / (dl + dr)", "dl * dr / (dl + dr)"),
    "plm_centred_index": ("sigma[i] = (q[ip] - q[im]) / (hl + hr);",
                          "sigma[i] = (q[ip] - q[i]) / (hl + hr);"),
    "plm_cumulative_sign": ("0.5 * r->c1[i] * (d * d - d * h)",
                            "0.5 * r->c1[i] * (d * d + d * h)"),
    "ppm_cumulative_term": ("S * (0.5 * xi * xi - xi * xi * xi / 3.0));",
                            "S * (0.5 * xi * xi - xi * xi * xi / 2.0));"),
    "quartic_degree": ("int lo = side, hi = side + 4;", "int lo = side, hi = side + 3;"),
    "seam_whole_count": ("c->nwhole = pr - pl - 1 + n;", "c->nwhole = pr - pl + n;"),
    "tie_to_left_cell": ("if (x[mid] <= y)", "if (x[mid] < y)"),
    "shift_direction": ("double yy = x[j] - sred;", "double yy = x[j] + sred;"),
    "no_copy_rule": ("c->copy = (dl == 0.0", "c->copy = (dl == 1.0"),
    "vanleer_midpoint_sign": ("qhat += sigma[jm] * 0.5 * (dx[jm] - c);",
                              "qhat += sigma[jm] * 0.5 * (dx[jm] + c);"),
    "residual_flux_index": ("q_next[i] = q[i] - (flux[cyc(i + 1, n)] - flux[i]) / dx[i];",
                            "q_next[i] = q[i] - (flux[cyc(i + 1, n)] - flux[i]) / dx[cyc(i + 1, n)];"),
    "adjoint_quartic_mass": ("gm[cyc(i - 1, n)] += w * (-b[0] - b[1]);",
                             "gm[cyc(i - 1, n)] += w * (-b[1]);"),
    "adjoint_upwind_side": ("int up = (c >= 0.0) ? cyc(j - 1, n) : j;",
                            "int up = (c >= 0.0) ? j : cyc(j - 1, n);"),
    "adjoint_plm_transpose": ("g_in[ip] += l1[i] / span;", "g_in[ip] -= l1[i] / span;"),
    "rows_mesh_offset": ("shared_mesh ? nodes : nodes + b + r;", "shared_mesh ? nodes : nodes + b;"),
    "rows_order_index": ("order[r], limiter, shift[r]", "order[0], limiter, shift[r]"),
    "rows_nsub_index": ("nsub ? nsub[r] : 1", "nsub ? nsub[0] : 1"),
    "rows_dv_offset": ("dv ? dv + b : NULL", "dv ? dv : NULL"),
    "rows_shared_mesh_ignored": ("shared_mesh ? nodes : nodes + b + r;", "nodes + b + r;"),
    "a4_factor": ("2.0 * q[i] + q[cyc(i - 1, n)]) / 24.0;", "2.0 * q[i] + q[cyc(i - 1, n)]) / 12.0;"),
    "a4_inverse_diagonal": ("for (int i = 0; i < n; ++i) b[i] = 22.0;",
                            "for (int i = 0; i < n; ++i) b[i] = 20.0;"),
    "a4_sherman_morrison_sign": ("double f = (y[0] + beta * y[n - 1] / gamma)",
                                 "double f = (y[0] - beta * y[n - 1] / gamma)"),
    "limited4_bound_neighbour": ("if (qp > hi) hi = qp;", "if (qp > hi) hi = Q;"),
    "limited4_blend": ("g = th * g + (1.0 - th) * r->q[i] * d;",
                       "g = th * g + (1.0 - th) * r->q[i] * r->dx[i];"),
    "limited4_theta": ("double t = (hi - Q) / (qmax - Q);", "double t = (hi - Q) / (qmax + Q);"),
    "radial_face_length": ("dt * (rf[j + 1] * F[j + 1] - rf[j] * F[j]) / area;",
                           "dt * (F[j + 1] - F[j]) / area;"),
    "radial_ring_area": ("double area = 0.5 * (rf[j + 1] * rf[j + 1] - rf[j] * rf[j]);",
                         "double area = 0.5 * (rf[j + 1] + rf[j]) * (rf[j + 1] - rf[j]) * 1.01;"),
    "radial_upwind_side": ("qh = col[j - 1] + sig[j - 1] * 0.5 * (dr[j - 1] - c);",
                           "qh = col[j] + sig[j - 1] * 0.5 * (dr[j - 1] - c);"),
    "shear_difference_sign": ("double d = fabs(omega[j + 1] - omega[j]);",
                              "double d = omega[j + 1] - omega[j];"),
    "tangent_minmod_choice": ("if (an.v < m.v) m = an;", "if (an.v > m.v) m = an;"),
    "tangent_vanleer_factor": ("sig = ddiv(dscale(dmul(dl, dr), 2.0), dadd(dl, dr));",
                               "sig = ddiv(dscale(dmul(dl, dr), 1.0), dadd(dl, dr));"),
    "tangent_constraint_operand": ("L = dsub(dscale(Q, 3.0), dscale(R, 2.0));",
                                   "L = dsub(dscale(Q, 3.0), dscale(L, 2.0));"),
    "tangent_mass_derivative": ("dm[i] = vdir[i] * dx[i];", "dm[i] = vdir[i];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor missing: %s" % name
    mutated = tmp_path / "ram_oracle_mutant.c"
    mutated.write_text(src.replace(old, new, 1))  # first occurrence: the forward map
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", str(lib),
                    str(mutated), "-lm"], check=True)
    env = dict(os.environ, RAM_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "planted mistake %s was not caught:\n%s" % (name, r.stdout[-2000:])
