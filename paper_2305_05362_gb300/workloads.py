"""Seeded synthetic inputs for the RAM hot path.

This module only draws inputs: meshes, initial fields, bulk velocities, time
steps and residual velocities.  It holds none of the method's arithmetic (no
reconstruction, no remap, no residual step), so both the CUDA library's tests
and the CPU oracle can take their inputs from it.

Every workload is a set of independent periodic rows packed back to back:
row r owns cells [row_offset[r], row_offset[r+1]).  Nodes are either one shared
mesh (N+1 values) or per-row meshes packed with one extra node per row (row r's
N_r+1 nodes start at row_offset[r] + r).

Recipes (the paper's tests are analytic setups; these stand in for them):
  line_uniform    1D periodic uniform row on [0,1), Q0 = 1 + 0.5 sin(2 pi x) plus a
                  top-hat of height 1 on [0.3, 0.5], exact cell averages.
  line_nonuniform 1D periodic row, widths log-uniform in [0.5, 2] x mean, renormalised
                  to length 1; Q0 = 1 + three periodic Gaussians; dv = 0.05 sin(4 pi x).
  disk            polar disk, rings log-spaced in r, uniform phi mesh shared by all
                  rings, Sigma = r^-1/2 (1 + 0.1 vortex), Keplerian angular rate
                  v0 = r^-3/2, dv = 1% random perturbation at every interface.
  batched         uneven independent rows (lengths log-uniform), own non-uniform
                  meshes, per-row shifts and orders, dv = 0.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass
class Workload:
    name: str
    row_offset: np.ndarray          # int64, n_rows + 1
    nodes: np.ndarray               # float64: shared (N+1) or packed per row
    shared_mesh: bool
    order: np.ndarray               # int8 per row (2, 3 or 4)
    limiter: bool
    q0: np.ndarray                  # float64 packed cell values
    v0: np.ndarray                  # float64 per row: bulk velocity (shift per unit time)
    dt: float
    dv: Optional[np.ndarray]        # float64 packed interface velocities, or None
    scheme: int                     # 0 donor, 1 van Leer
    nsub: np.ndarray                # int32 per row: residual sub-steps
    steps: int
    notes: str = ""

    @property
    def n_rows(self) -> int:
        return int(self.row_offset.size - 1)

    @property
    def n_cells(self) -> int:
        return int(self.row_offset[-1])

    def row_nodes(self, r: int) -> np.ndarray:
        if self.shared_mesh:
            return self.nodes
        b, e = int(self.row_offset[r]), int(self.row_offset[r + 1])
        return self.nodes[b + r: e + r + 1]

    def row_slice(self, r: int) -> slice:
        return slice(int(self.row_offset[r]), int(self.row_offset[r + 1]))

    def period(self, r: int) -> float:
        x = self.row_nodes(r)
        return float(x[-1] - x[0])


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def uniform_nodes(n: int, x0: float = 0.0, length: float = 1.0) -> np.ndarray:
    x = x0 + length * (np.arange(n + 1, dtype=np.float64) / n)
    x[-1] = x0 + length
    return x


def random_nodes(n: int, seed: int, ratio: float = 4.0, length: float = 1.0,
                 x0: float = 0.0) -> np.ndarray:
    """Widths drawn log-uniform in [1/sqrt(ratio), sqrt(ratio)] x mean,
    renormalised so that the row has the given length."""
    rng = np.random.default_rng(seed)
    half = 0.5 * math.log(ratio)
    w = np.exp(rng.uniform(-half, half, n))
    x = np.concatenate([[0.0], np.cumsum(w)])
    x = x0 + length * (x / x[-1])
    x[-1] = x0 + length
    return x


# --------------------------------------------------------------------------
# exact cell averages of the analytic profiles
# --------------------------------------------------------------------------

def sine_averages(x: np.ndarray, k: int = 1, amp: float = 1.0, phase: float = 0.0,
                  period: float = 1.0) -> np.ndarray:
    """Cell averages of amp * sin(2 pi k x / period + phase)."""
    w = TWO_PI * k / period
    a, b = x[:-1], x[1:]
    return amp * (np.cos(w * a + phase) - np.cos(w * b + phase)) / (w * (b - a))


def tophat_averages(x: np.ndarray, lo: float, hi: float, height: float = 1.0) -> np.ndarray:
    a, b = x[:-1], x[1:]
    overlap = np.clip(np.minimum(b, hi) - np.maximum(a, lo), 0.0, None)
    return height * overlap / (b - a)


def gaussian_averages(x: np.ndarray, centre: float, sigma: float, period: float,
                      amp: float = 1.0, images=(-1, 0, 1)) -> np.ndarray:
    """Cell averages of a periodic Gaussian amp * sum_k exp(-(x-c-kP)^2 / 2 s^2)."""
    from scipy.special import erf
    a, b = x[:-1], x[1:]
    out = np.zeros(a.size)
    c = sigma * math.sqrt(math.pi / 2.0)
    s2 = sigma * math.sqrt(2.0)
    for k in images:
        cc = centre + k * period
        out += c * (erf((b - cc) / s2) - erf((a - cc) / s2))
    return amp * out / (b - a)


def three_gaussians(x: np.ndarray, seed: int) -> np.ndarray:
    """1 + three periodic Gaussians (centres U[0,L), widths U[0.02,0.1] L)."""
    rng = np.random.default_rng(seed)
    period = float(x[-1] - x[0])
    q = np.ones(x.size - 1)
    for _ in range(3):
        c = x[0] + period * rng.uniform(0.0, 1.0)
        s = period * rng.uniform(0.02, 0.1)
        q += gaussian_averages(x, c, s, period)
    return q


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def line_uniform(n: int = 256, shift_cells: float = 7.3, steps: int = 100,
                 order: int = 2) -> Workload:
    x = uniform_nodes(n)
    q0 = 1.0 + sine_averages(x, amp=0.5) + tophat_averages(x, 0.3, 0.5)
    dt = 1.0
    v0 = np.array([shift_cells / n / dt])
    return Workload("line_uniform_%d" % n, np.array([0, n], dtype=np.int64), x, True,
                    np.array([order], dtype=np.int8), True, q0, v0, dt, None, 1,
                    np.ones(1, dtype=np.int32), steps,
                    "uniform row, PLM, shift %.1f cells/step" % shift_cells)


def line_nonuniform(n: int = 4096, shift_cells: float = 40.7, steps: int = 1000,
                    seed_mesh: int = 2, seed_q: int = 3, order: int = 3) -> Workload:
    x = random_nodes(n, seed_mesh)
    q0 = three_gaussians(x, seed_q)
    v0_val = 10.0
    dt = shift_cells / n / v0_val
    # dv at the interfaces x_{j-1/2}
    dv = 0.05 * np.sin(4.0 * math.pi * x[:-1])
    return Workload("line_nonuniform_%d" % n, np.array([0, n], dtype=np.int64), x, True,
                    np.array([order], dtype=np.int8), True, q0, np.array([v0_val]), dt,
                    dv, 1, np.ones(1, dtype=np.int32), steps,
                    "non-uniform row, PPM + van Leer residual")


def disk(n_r: int = 1024, n_phi: int = 4096, seed_dv: int = 4, steps: int = 500,
         r_in: float = 0.4, r_out: float = 2.5, inner_shift_cells: float = 150.0,
         ref_n_phi: Optional[int] = None, order: int = 3, limiter: bool = True,
         scheme: int = 1, dv_amp: float = 0.01, cfl_target: float = 0.5,
         dtype=np.float64, with_dv: bool = True) -> Workload:
    """Polar disk: every ring is a periodic row in phi on one shared uniform mesh.

    The time step moves the ring at r = r_in by `inner_shift_cells` cells of a
    mesh with `ref_n_phi` cells (default n_phi).  Residual sub-steps per ring keep
    |dv| dt / (nsub dphi) <= cfl_target."""
    ref = n_phi if ref_n_phi is None else ref_n_phi
    x = uniform_nodes(n_phi, 0.0, TWO_PI)
    k = np.arange(n_r, dtype=np.float64)
    r = r_in * (r_out / r_in) ** ((k + 0.5) / n_r)
    omega = r ** -1.5
    dt = inner_shift_cells * (TWO_PI / ref) / (r_in ** -1.5)
    # vortex: radial Gaussian (width 0.05) times an azimuthal Gaussian (width 0.3)
    radial = np.exp(-((r - 1.0) ** 2) / (2.0 * 0.05 ** 2))
    az = gaussian_averages(x, math.pi, 0.3, TWO_PI)
    q0 = (r[:, None] ** -0.5) * (1.0 + 0.1 * radial[:, None] * az[None, :])
    q0 = np.ascontiguousarray(q0.reshape(-1), dtype=dtype)
    dphi = TWO_PI / n_phi
    if with_dv:
        rng = np.random.default_rng(seed_dv)
        u = rng.uniform(-1.0, 1.0, size=(n_r, n_phi))
        dvm = dv_amp * omega[:, None] * u
        cfl = np.abs(dvm).max(axis=1) * dt / dphi
        nsub = np.maximum(1, np.ceil(cfl / cfl_target)).astype(np.int32)
        dv = np.ascontiguousarray(dvm.reshape(-1), dtype=dtype)
    else:
        dv = None
        nsub = np.ones(n_r, dtype=np.int32)
    ro = (np.arange(n_r + 1, dtype=np.int64) * n_phi)
    return Workload("disk_%dx%d" % (n_r, n_phi), ro, x, True,
                    np.full(n_r, order, dtype=np.int8), limiter, q0, omega, dt, dv,
                    scheme, nsub, steps,
                    "Keplerian disk, r in [%.1f,%.1f], inner ring %.1f cells/step"
                    % (r_in, r_out, inner_shift_cells * n_phi / ref))


def batched(n_rows: int = 512, n_min: int = 64, n_max: int = 65536, seed_len: int = 6,
            seed_mesh0: int = 7, seed_shift: int = 9, seed_order: int = 10,
            seed_q0: int = 11, steps: int = 200, orders=(2, 3, 4),
            limiter: bool = False, with_dv: bool = False, seed_dv: int = 12) -> Workload:
    """Uneven independent rows, each with its own non-uniform mesh of length 1,
    shift exp(U[ln 0.3, ln 200]) mean cells per step, order drawn from `orders`.
    with_dv: a residual velocity at the interfaces, 0.3 dx_min sin(2 pi (3 x + phi_r))
    / dt on row r (phi_r seeded), so its Courant number stays below 0.3; van Leer."""
    rng = np.random.default_rng(seed_len)
    lens = np.round(np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_rows)))
    lens = lens.astype(np.int64)
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nodes = np.empty(int(ro[-1]) + n_rows, dtype=np.float64)
    q0 = np.empty(int(ro[-1]), dtype=np.float64)
    for rr in range(n_rows):
        n = int(lens[rr])
        x = random_nodes(n, seed_mesh0 + rr)
        nodes[ro[rr] + rr: ro[rr + 1] + rr + 1] = x
        q0[ro[rr]:ro[rr + 1]] = three_gaussians(x, seed_q0 + rr)
    rs = np.random.default_rng(seed_shift)
    shift_cells = np.exp(rs.uniform(math.log(0.3), math.log(200.0), n_rows))
    dt = 1.0
    v0 = shift_cells / lens / dt  # every row has length 1
    ro_ = np.random.default_rng(seed_order)
    order = ro_.choice(np.array(orders, dtype=np.int8), size=n_rows)
    dv = None
    if with_dv:
        dv = np.empty(int(ro[-1]), dtype=np.float64)
        ph = np.random.default_rng(seed_dv).random(n_rows)
        for rr in range(n_rows):
            x = nodes[ro[rr] + rr: ro[rr + 1] + rr + 1]
            amp = 0.3 * float(np.diff(x).min()) / dt
            dv[ro[rr]:ro[rr + 1]] = amp * np.sin(2.0 * math.pi * (3.0 * x[:-1] + ph[rr]))
    return Workload("batched_%d_rows%s" % (n_rows, "_dv" if with_dv else ""), ro, nodes, False,
                    order, limiter, q0, v0, dt, dv, 1, np.ones(n_rows, dtype=np.int32), steps,
                    "uneven rows %d..%d cells%s" % (n_min, n_max,
                                                    ", van Leer residual" if with_dv else ""))


# --------------------------------------------------------------------------
# mesh-density meshes (App. B.1): periodic bump on [x_min, x_max], centred at 0
# --------------------------------------------------------------------------

def bump_density(s, a: float, b: float, c: float):
    """Unnormalised periodic-bump density psi(s): 1 + c inside |s| <= a, a cos^2
    transition for a < |s| < b, 1 outside."""
    s = np.abs(np.asarray(s, dtype=np.float64))
    mid = 1.0 + c * np.cos(0.5 * math.pi * (s - a) / (b - a)) ** 2
    return np.where(s <= a, 1.0 + c, np.where(s < b, mid, 1.0))


def bump_norm(x_min: float, x_max: float, a: float, b: float, c: float) -> float:
    """Integral of psi over the domain: (x_max - x_min) + c (a + b)."""
    return (x_max - x_min) + c * (a + b)


def bump_cumulative(x, x_min: float, x_max: float, a: float, b: float, c: float):
    """u(x) = (1/I) * integral of psi from x_min to x, in [0, 1] (Eq. 23)."""
    x = np.asarray(x, dtype=np.float64)
    w = b - a

    def prim_pos(t):
        # integral of psi from 0 to t >= 0
        t = np.asarray(t, dtype=np.float64)
        inner = (1.0 + c) * np.minimum(t, a)
        tt = np.clip(t, a, b)
        trans = (tt - a) + c * (0.5 * (tt - a) + w / (2.0 * math.pi)
                                * np.sin(math.pi * (tt - a) / w))
        outer = np.maximum(t - b, 0.0)
        return inner + trans + outer

    def prim(t):
        return np.sign(t) * prim_pos(np.abs(t))

    return (prim(x) - prim(x_min)) / bump_norm(x_min, x_max, a, b, c)


def bump_nodes(n: int, x_min: float, x_max: float, a: float, b: float, c: float,
               iters: int = 200) -> np.ndarray:
    """Nodes with equal density integral per cell, u(x_{i+1/2}) = (i+1)/n, found by
    bisection (App. B.1, Eq. 22)."""
    target = np.arange(n + 1, dtype=np.float64) / n
    lo = np.full(n + 1, x_min)
    hi = np.full(n + 1, x_max)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        below = bump_cumulative(mid, x_min, x_max, a, b, c) < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    x = 0.5 * (lo + hi)
    x[0], x[-1] = x_min, x_max
    return x


# --------------------------------------------------------------------------
# the radial bump (App. B.2) and the two-dimensional polar disk (Sec. 4.2)
# --------------------------------------------------------------------------

def radial_bump_density(s, s0: float, a: float, b: float, c: float):
    """psi(s) = 1/s + c beta(|s - s0|), beta = 1 inside a, cos^2 transition to b, 0
    outside (unnormalised)."""
    s = np.asarray(s, dtype=np.float64)
    t = np.abs(s - s0)
    beta = np.where(t <= a, 1.0,
                    np.where(t < b, np.cos(0.5 * math.pi * (t - a) / (b - a)) ** 2, 0.0))
    return 1.0 / s + c * beta


def radial_bump_norm(x_min: float, x_max: float, a: float, b: float, c: float) -> float:
    """Integral of psi over [x_min, x_max] for a bump inside the domain:
    log(x_max / x_min) + c (a + b)."""
    return math.log(x_max) - math.log(x_min) + c * (a + b)


def radial_bump_cumulative(x, x_min: float, x_max: float, s0: float, a: float, b: float,
                           c: float):
    """u(x) = (1/I) integral of psi from x_min to x, in [0, 1]."""
    x = np.asarray(x, dtype=np.float64)
    w = b - a

    def bump_from_centre(t):
        # integral of beta from 0 to t >= 0 (distance from s0)
        t = np.asarray(t, dtype=np.float64)
        tt = np.clip(t, a, b)
        return np.minimum(t, a) + 0.5 * (tt - a) + w / (2.0 * math.pi) * np.sin(math.pi * (tt - a) / w)

    def bump_prim(s):
        d = s - s0
        return np.sign(d) * bump_from_centre(np.abs(d))

    num = np.log(x / x_min) + c * (bump_prim(x) - bump_prim(x_min))
    return num / radial_bump_norm(x_min, x_max, a, b, c)


def radial_bump_nodes(n: int, x_min: float, x_max: float, s0: float, a: float, b: float,
                      c: float, iters: int = 200) -> np.ndarray:
    """Faces with equal density integral per ring, u(r_j) = j / n, by bisection."""
    target = np.arange(n + 1, dtype=np.float64) / n
    lo = np.full(n + 1, x_min)
    hi = np.full(n + 1, x_max)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        below = radial_bump_cumulative(mid, x_min, x_max, s0, a, b, c) < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    x = 0.5 * (lo + hi)
    x[0], x[-1] = x_min, x_max
    return x


@dataclasses.dataclass
class Disk2D:
    """A polar disk for the dimensionally split step: rings are rows on one shared
    azimuthal mesh `phi`; `rf` holds the n_r + 1 ring face radii."""
    name: str
    phi: np.ndarray        # n_phi + 1 azimuthal nodes
    rf: np.ndarray         # n_r + 1 radial faces
    omega: np.ndarray      # n_r angular rates of the bulk rotation (the RAM shift per time)
    q0: np.ndarray         # (n_r, n_phi) surface density
    dvphi: np.ndarray      # (n_r, n_phi) residual azimuthal velocity at the phi interfaces
    vr: np.ndarray         # (n_r + 1, n_phi) radial velocity on the ring faces (0 at the ends)
    order: int
    limiter: bool
    scheme: int
    nsub: np.ndarray       # residual sub-steps per ring
    dt: float

    @property
    def n_r(self) -> int:
        return int(self.rf.size - 1)

    @property
    def n_phi(self) -> int:
        return int(self.phi.size - 1)


def polar_disk_2d(n_r: int = 128, n_phi: int = 512, seed: int = 21, nonuniform: bool = True,
                  order: int = 2, scheme: int = 1, beta: float = 0.44,
                  dv_amp: float = 0.01, vr_amp: float = 0.01) -> Disk2D:
    """The mesh of Sec. 4.2: phi in [-pi, pi] on the periodic bump (a = 0.1387,
    b = 0.2773, c = 15) and r in [0.4, 2.1] on the radial bump centred at 1 (same a,
    b, c = 2.5), or a uniform / log-uniform mesh.  Frame co-rotating with r = 1:
    omega = r^-3/2 - 1.  Sigma = r^-1/2 (1 + 0.1 vortex at r = 1), a seeded 1%
    azimuthal residual velocity and a smooth seeded radial velocity that vanishes at
    the walls.  dt is the shear limit (beta) capped by the radial and residual CFL
    conditions."""
    a, b = 0.1387, 0.2773
    if nonuniform:
        phi = bump_nodes(n_phi, -math.pi, math.pi, a, b, 15.0)
        rf = radial_bump_nodes(n_r, 0.4, 2.1, 1.0, a, b, 2.5)
    else:
        phi = uniform_nodes(n_phi, -math.pi, 2.0 * math.pi)
        rf = 0.4 * (2.1 / 0.4) ** (np.arange(n_r + 1) / n_r)
    rc = 0.5 * (rf[1:] + rf[:-1])
    omega = rc ** -1.5 - 1.0
    dphi = np.diff(phi)
    vortex = np.exp(-((rc - 1.0) ** 2) / (2 * 0.05 ** 2))[:, None] * \
        gaussian_averages(phi, 0.5, 0.3, 2.0 * math.pi)[None, :]
    q0 = (rc ** -0.5)[:, None] * (1.0 + 0.1 * vortex)
    rng = np.random.default_rng(seed)
    dvphi = dv_amp * (rc ** -1.5)[:, None] * rng.uniform(-1.0, 1.0, (n_r, n_phi))
    phase = rng.uniform(0.0, 2.0 * math.pi, 3)
    pc = 0.5 * (phi[1:] + phi[:-1])
    shape = (np.sin(pc + phase[0]) + 0.5 * np.sin(2 * pc + phase[1]))[None, :]
    wall = ((rf - rf[0]) * (rf[-1] - rf) / ((rf[-1] - rf[0]) / 2.0) ** 2)[:, None]
    vr = vr_amp * wall * shape
    vr[0] = 0.0
    vr[-1] = 0.0
    dt_shear = beta * dphi.min() / np.max(np.abs(np.diff(omega)))
    dr = np.diff(rf)
    dr_face = np.minimum(np.concatenate([[np.inf], dr]), np.concatenate([dr, [np.inf]]))
    vmax = np.max(np.abs(vr), axis=1)
    dt_r = beta * np.min(dr_face[vmax > 0] / vmax[vmax > 0]) if np.any(vmax > 0) else np.inf
    dt = min(dt_shear, dt_r)
    cfl = np.abs(dvphi).max(axis=1) * dt / dphi.min()
    nsub = np.maximum(1, np.ceil(cfl / 0.5)).astype(np.int32)
    return Disk2D("polar_disk_2d_%dx%d%s" % (n_r, n_phi, "" if nonuniform else "_uniform"),
                  phi, rf, omega, np.ascontiguousarray(q0), np.ascontiguousarray(dvphi),
                  np.ascontiguousarray(vr), order, True, scheme, nsub, float(dt))
