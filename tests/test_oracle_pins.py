"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests re-types the oracle's formulas.  Each checks a property
that a plausible mistake in the oracle (a dropped term, a wrong sign or index,
a transposed operand, a mishandled periodic seam) would break:

  conservation (Eq. 10), constants, exact rolls and full-period identity
  (Sec. 1, Eq. 8), polynomial reproduction, measured convergence order,
  brute-force quadrature of the reconstructed profile (Eqs. 15-18),
  textbook PPM interface values (App. A / Colella & Woodward 1984),
  no new extrema (Sec. 2, Sec. 3.1), the small-shift equivalence with the
  upwind step (Sec. 3.2), the worked example of Fig. 1, and the transpose
  identities of the linear step.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2305_05362_gb300 import workloads as wl

EPS = np.finfo(np.float64).eps


def rel_l1(a, b, x=None):
    w = np.ones(len(a)) if x is None else np.diff(x)
    return float(np.sum(np.abs(a - b) * w) / np.sum(np.abs(b) * w))


# ---------------------------------------------------------------------------
# conservation, constants, rolls
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("order,limiter", [(2, True), (2, False), (3, True),
                                           (3, False), (4, False)])
@pytest.mark.parametrize("s", [0.0, 1e-3, 0.37, -2.71, 5.0, 123.456])
def test_mass_conservation(order, limiter, s):
    """Eq. 10: the remap conserves the total mass to round-off."""
    x = wl.random_nodes(97, seed=11)
    q = 1.0 + np.random.default_rng(3).random(97)
    out = oracle.shift(x, q, s, order, limiter)
    m0, m1 = oracle.mass(x, q), oracle.mass(x, out)
    assert abs(m1 - m0) <= 64 * EPS * m0


@pytest.mark.parametrize("order,limiter", [(2, True), (3, True), (3, False), (4, False)])
def test_constant_field(order, limiter):
    """A constant stays constant.  The only error is the rounding of the shifted
    edge positions (~eps * L absolute) relative to the smallest width."""
    x = wl.random_nodes(128, seed=5)
    c = 3.7
    out = oracle.shift(x, np.full(128, c), 0.4321, order, limiter)
    bound = 8 * EPS * (x[-1] - x[0]) / np.diff(x).min()
    assert np.max(np.abs(out - c)) <= c * bound


@pytest.mark.parametrize("order,limiter", [(2, True), (3, True), (3, False), (4, False)])
@pytest.mark.parametrize("k", [0, 1, 3, 100, 255, 256, 700, -5])
def test_integer_roll_bit_exact(order, limiter, k):
    """Sec. 1 (Eq. 8): a whole-cell shift on a uniform periodic mesh is a cyclic
    permutation with no numerical error (dyadic mesh, so the shifted edges are
    exact)."""
    n = 256
    x = wl.uniform_nodes(n)
    q = np.random.default_rng(7).random(n)
    out = oracle.shift(x, q, k / n, order, limiter)
    assert np.array_equal(out, np.roll(q, k))


@pytest.mark.parametrize("m", [1, 2, -3])
@pytest.mark.parametrize("order", [2, 3, 4])
def test_full_period_identity(m, order):
    """A shift by whole periods returns the input bit for bit, on any mesh."""
    x = wl.random_nodes(200, seed=2, x0=-0.3)
    q = wl.three_gaussians(x, 3)
    L = x[-1] - x[0]
    out = oracle.shift(x, q, m * L, order, order != 4)
    assert np.array_equal(out, q)


def test_config_line_uniform_period_recovery():
    """The uniform 256-cell line: 7.3 cells/step for 2560 steps is 73 periods;
    with a whole-period total the profile returns close to the input, the mass
    is conserved and the top-hat stays within its bounds (limited PLM)."""
    w = wl.line_uniform()
    x = w.row_nodes(0)
    q = w.q0.copy()
    s = oracle.shift_from_velocity(w.v0[0], w.dt)
    for _ in range(w.steps):
        q = oracle.step(x, q, s, 2, True)
    m0 = oracle.mass(x, w.q0)
    assert abs(oracle.mass(x, q) - m0) <= 1e-13 * m0
    assert q.min() >= w.q0.min() - 1e-12 and q.max() <= w.q0.max() + 1e-12


# ---------------------------------------------------------------------------
# accuracy: polynomials and convergence order
# ---------------------------------------------------------------------------

def poly_cell_averages(P, a, b):
    Pi = P.integ()
    return (Pi(b) - Pi(a)) / (b - a)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_polynomial_reproduction(order):
    """Limiter off, cell averages of a polynomial of degree < p: the shifted cell
    averages are exact to round-off (cells whose stencils touch the seam of the
    non-periodic polynomial are excluded)."""
    n = 300
    x = wl.random_nodes(n, seed=21)
    rng = np.random.default_rng(22)
    P = np.polynomial.Polynomial(rng.uniform(-1, 1, order))  # degree order-1
    q = poly_cell_averages(P, x[:-1], x[1:])
    s = 7.77 / n
    out = oracle.shift(x, q, s, order, False)
    lo, hi = x[:-1] - s, x[1:] - s
    keep = (lo >= x[4]) & (hi <= x[n - 4])
    exact = poly_cell_averages(P, lo[keep], hi[keep])
    assert keep.sum() > 250
    np.testing.assert_allclose(out[keep], exact, rtol=0, atol=1e-12)


@pytest.mark.parametrize("order", [2, 3])
def test_linear_profile_kept_with_limiter(order):
    """A linear profile is not touched by the limiters (no extremum, no clipping)."""
    n = 200
    x = wl.random_nodes(n, seed=4)
    P = np.polynomial.Polynomial([0.3, 2.0])
    q = poly_cell_averages(P, x[:-1], x[1:])
    s = 3.3 / n
    out = oracle.shift(x, q, s, order, True)
    lo, hi = x[:-1] - s, x[1:] - s
    keep = (lo >= x[4]) & (hi <= x[n - 4])
    # rounding of the shifted edges: ~eps * L absolute, relative to the width
    tol = 8 * EPS * (x[-1] - x[0]) / np.diff(x).min() * np.abs(q).max()
    np.testing.assert_allclose(out[keep], poly_cell_averages(P, lo[keep], hi[keep]),
                               rtol=0, atol=tol)


def _sine_period_error(n, order, limiter, cells_per_step=7.3):
    x = wl.uniform_nodes(n)
    q0 = wl.sine_averages(x)
    steps = int(round(n / cells_per_step))
    assert abs(steps * cells_per_step - n) < 1e-9  # same sub-cell fraction at every n
    s = 1.0 / steps
    q = q0.copy()
    for _ in range(steps):
        q = oracle.shift(x, q, s, order, limiter)
    return rel_l1(q, q0, x)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_convergence_order_smooth_sine(order):
    """Limiter off, exact initial cell averages, one period at 7.3 cells/step:
    the measured order equals the interpolation order p.  N is a multiple of 73 so
    that every resolution takes the same sub-cell fraction per step."""
    ns = [146, 292, 584, 1168]
    errs = [_sine_period_error(n, order, False) for n in ns]
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert abs(-slope - order) < 0.15, (errs, slope)


# ---------------------------------------------------------------------------
# brute-force quadrature of the reconstructed profile (Eqs. 15-18)
# ---------------------------------------------------------------------------

GL_X, GL_W = np.polynomial.legendre.leggauss(6)


def _q_eval(coef, order, x, i, xx):
    """Evaluate q_i at points xx from the oracle's per-cell coefficients."""
    a, b = x[i], x[i + 1]
    h = b - a
    if order == 2:
        return coef[i, 0] + coef[i, 1] * (xx - 0.5 * (a + b))
    xi = (xx - a) / h
    L, R, S = coef[i]
    return L + xi * (R - L) + S * xi * (1.0 - xi)


def _brute_shift(x, q, s, order, limiter):
    n = q.size
    L = x[-1] - x[0]
    coef = oracle.reconstruct(x, q, order, limiter)
    out = np.empty(n)
    for i in range(n):
        lo, hi = x[i] - s, x[i + 1] - s
        k0 = math.floor((lo - x[0]) / L) - 1
        k1 = math.floor((hi - x[0]) / L) + 1
        brk = [lo, hi]
        for k in range(k0, k1 + 1):
            pts = x[:-1] + k * L
            brk += list(pts[(pts > lo) & (pts < hi)])
        brk = np.sort(np.array(brk))
        tot = 0.0
        for a, b in zip(brk[:-1], brk[1:]):
            if b <= a:
                continue
            mid = 0.5 * (a + b)
            k = math.floor((mid - x[0]) / L)
            p = int(np.searchsorted(x, mid - k * L, side="right") - 1)
            p = min(max(p, 0), n - 1)
            xx = 0.5 * (b - a) * GL_X + 0.5 * (a + b) - k * L
            tot += 0.5 * (b - a) * np.dot(GL_W, _q_eval(coef, order, x, p, xx))
        out[i] = tot / (x[i + 1] - x[i])
    return out


@pytest.mark.parametrize("order,limiter", [(2, True), (2, False), (3, True), (3, False)])
@pytest.mark.parametrize("s", [0.0123, 0.4, 1.77, -0.91, 3.0 + 1e-9])
def test_brute_force_quadrature(order, limiter, s):
    n = 37
    x = wl.random_nodes(n, seed=31, x0=-0.5)
    q = 1.0 + np.random.default_rng(32).random(n)
    out = oracle.shift(x, q, s, order, limiter)
    ref = _brute_shift(x, q, s, order, limiter)
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-13)


def _quartic_pair_G(x, m, i):
    """G_i for order 4 built independently: numpy fits of the two quartics of the
    cumulative mass through nodes {i-5/2..i+3/2} and {i-3/2..i+5/2}."""
    n = m.size
    L = x[-1] - x[0]
    idx = np.arange(i - 2, i + 4)            # node indices i-5/2 .. i+5/2 as x[j]
    pos = np.array([x[j % n] + (j // n) * L for j in idx]) - x[i]
    cum = np.concatenate([[0.0], np.cumsum(m)])
    tot = cum[-1]
    vals = np.array([cum[j % n] + (j // n) * tot for j in idx]) - cum[i]
    scale = x[i + 1] - x[i]
    p1 = np.polynomial.Polynomial.fit(pos[:5] / scale, vals[:5], 4, domain=[-1, 1],
                                      window=[-1, 1])
    p2 = np.polynomial.Polynomial.fit(pos[1:] / scale, vals[1:], 4, domain=[-1, 1],
                                      window=[-1, 1])
    return lambda d: 0.5 * (p1(d / scale) + p2(d / scale))


@pytest.mark.parametrize("s", [0.0123, 0.4, -0.91, 2.5])
def test_brute_force_order4(s):
    n = 29
    x = wl.random_nodes(n, seed=41)
    q = 1.0 + np.random.default_rng(42).random(n)
    m = q * np.diff(x)
    out = oracle.shift(x, q, s, 4, False)
    L = x[-1] - x[0]
    G = [_quartic_pair_G(x, m, i) for i in range(n)]
    ref = np.empty(n)
    for i in range(n):
        lo, hi = x[i] - s, x[i + 1] - s
        brk = [lo, hi]
        for k in range(math.floor((lo - x[0]) / L) - 1, math.floor((hi - x[0]) / L) + 2):
            pts = x[:-1] + k * L
            brk += list(pts[(pts > lo) & (pts < hi)])
        brk = np.sort(brk)
        tot = 0.0
        for a, b in zip(brk[:-1], brk[1:]):
            mid = 0.5 * (a + b)
            k = math.floor((mid - x[0]) / L)
            p = int(np.searchsorted(x, mid - k * L, side="right") - 1)
            base = x[p] + k * L
            tot += G[p](b - base) - G[p](a - base)
        ref[i] = tot / (x[i + 1] - x[i])
    np.testing.assert_allclose(out, ref, rtol=1e-10, atol=1e-11)


# ---------------------------------------------------------------------------
# reconstruction: textbook values and monotonicity
# ---------------------------------------------------------------------------

def test_ppm_uniform_interface_textbook():
    """Uniform mesh, limiter off: <Q>_{i+1/2} = 7/12 (Q_i + Q_{i+1}) - 1/12 (Q_{i-1} +
    Q_{i+2}) (Colella & Woodward 1984, uniform form of App. A)."""
    n = 50
    x = wl.uniform_nodes(n)
    q = np.random.default_rng(8).random(n)
    c = oracle.reconstruct(x, q, 3, False)
    qr = c[:, 1]
    ref = 7 / 12 * (q + np.roll(q, -1)) - 1 / 12 * (np.roll(q, 1) + np.roll(q, -2))
    np.testing.assert_allclose(qr, ref, rtol=0, atol=1e-14)
    np.testing.assert_allclose(c[:, 0], np.roll(qr, 1), rtol=0, atol=0)


def test_ppm_cubic_interface_exact_nonuniform():
    """App. A with sums of widths: for cell averages of a cubic the interface value
    is the cubic's value at the node, on a non-uniform mesh.  (With the printed
    products the error is O(1), which pins that reading.)"""
    n = 80
    x = wl.random_nodes(n, seed=9)
    P = np.polynomial.Polynomial([0.2, -1.0, 3.0, -2.5])
    q = poly_cell_averages(P, x[:-1], x[1:])
    c = oracle.reconstruct(x, q, 3, False)
    inner = slice(3, n - 4)
    np.testing.assert_allclose(c[inner, 1], P(x[1:][inner]), rtol=0, atol=1e-12)


def test_plm_van_leer_cases():
    """Sec. 3.1: zero slope at an extremum, harmonic mean of the one-sided slopes
    otherwise."""
    x = wl.uniform_nodes(4)        # h = 1/4
    q = np.array([0.0, 1.0, 3.0, 1.0])
    c = oracle.reconstruct(x, q, 2, True)
    h = 0.25
    dl, dr = (1.0 - 0.0) / h, (3.0 - 1.0) / h
    assert c[1, 1] == pytest.approx(2 * dl * dr / (dl + dr), rel=1e-15)
    assert c[2, 1] == 0.0           # cell 2 is a maximum
    assert c[0, 1] == 0.0           # cell 0 is a minimum (periodic neighbour 1.0)


@pytest.mark.parametrize("order", [2, 3])
def test_no_new_extrema_in_reconstruction(order):
    """Sec. 2: the limited q_i stays within the range of Q_{i-1}, Q_i, Q_{i+1}.
    PLM is checked on a uniform mesh: with slopes per unit length the harmonic
    mean of Sec. 3.1 can overshoot a neighbour on a strongly non-uniform mesh
    (a property of the stated limiter, recorded with the readings)."""
    n = 300
    x = wl.uniform_nodes(n) if order == 2 else wl.random_nodes(n, seed=12)
    rng = np.random.default_rng(13)
    q = np.where(rng.random(n) < 0.2, 1.0, 0.0) + 0.1 * rng.random(n)
    c = oracle.reconstruct(x, q, order, True)
    lo = np.minimum(np.minimum(np.roll(q, 1), q), np.roll(q, -1))
    hi = np.maximum(np.maximum(np.roll(q, 1), q), np.roll(q, -1))
    for i in range(n):
        xx = np.linspace(x[i], x[i + 1], 33)
        v = _q_eval(c, order, x, i, xx)
        assert v.min() >= lo[i] - 1e-13 and v.max() <= hi[i] + 1e-13


@pytest.mark.parametrize("order", [2, 3])
def test_no_new_extrema_after_shift(order):
    n = 256
    x = wl.uniform_nodes(n) if order == 2 else wl.random_nodes(n, seed=14)
    q = wl.tophat_averages(x, 0.3, 0.55) + 0.25
    out = q
    for _ in range(20):
        out = oracle.shift(x, out, 0.0371, order, True)
    assert out.min() >= q.min() - 1e-13 and out.max() <= q.max() + 1e-13


def test_cumulative_is_conservative():
    """Eq. 13: the in-cell cumulative at the full width is the cell mass."""
    n = 40
    x = wl.random_nodes(n, seed=15)
    q = np.random.default_rng(16).random(n) + 0.5
    cells = np.arange(n)
    for order, lim in [(2, True), (3, True), (3, False), (4, False)]:
        g = oracle.cell_cumulative(x, q, cells, np.diff(x), order, lim)
        np.testing.assert_allclose(g, q * np.diff(x), rtol=1e-13, atol=0)
        g0 = oracle.cell_cumulative(x, q, cells, np.zeros(n), order, lim)
        assert np.all(g0 == 0.0)


# ---------------------------------------------------------------------------
# equivalences stated by the paper
# ---------------------------------------------------------------------------

def test_small_shift_equals_van_leer_upwind_step():
    """Sec. 3.2: for a shift below the smallest cell the remap is a standard upwind
    step; with PLM the upwind flux through the swept region, evaluated at its
    midpoint (exact for a linear profile), is the van Leer residual step with
    dv = s / dt."""
    n = 120
    x = wl.random_nodes(n, seed=17)
    q = wl.three_gaussians(x, 18)
    s = 0.8 * np.diff(x).min()
    dt = 0.37
    a = oracle.shift(x, q, s, 2, True)
    b = oracle.residual(x, q, np.full(n, s / dt), dt, oracle.VANLEER)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-14)


def test_uniform_mesh_shift_splits_into_roll_plus_fraction():
    """Sec. 4.1: on a uniform mesh RAM is FARGO -- an integer roll composed with a
    sub-cell remap."""
    n = 128
    x = wl.uniform_nodes(n)
    q = wl.three_gaussians(x, 19)
    sig = 37.41
    a = oracle.shift(x, q, sig / n, 3, True)
    b = np.roll(oracle.shift(x, q, (sig - 37) / n, 3, True), 37)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-14)


def test_worked_example_fig1():
    """Sec. 3.4 (Fig. 1): an output cell whose shifted interval starts in cell 1,
    covers cell 2 and ends in cell 3 gets the right part of q_1, all of M_2 and
    the left part of q_3.  Structural check on a hand-built 6-cell mesh (the paper
    prints no numbers for this example)."""
    x = np.array([0.0, 0.1, 0.25, 0.33, 0.5, 0.7, 1.0])
    q = np.array([1.0, 2.0, 4.0, 3.0, 1.5, 1.2])
    s = 0.3  # output cell 4 = [0.5, 0.7] comes from [0.2, 0.4]: cells 1, 2, 3
    coef = oracle.reconstruct(x, q, 2, True)
    out = oracle.shift(x, q, s, 2, True)
    lo, hi = x[4] - s, x[5] - s
    assert x[1] <= lo < x[2] and x[3] <= hi < x[4]

    def integ(i, a, b):
        xc = 0.5 * (x[i] + x[i + 1])
        return coef[i, 0] * (b - a) + 0.5 * coef[i, 1] * ((b - xc) ** 2 - (a - xc) ** 2)

    m = integ(1, lo, x[2]) + q[2] * (x[3] - x[2]) + integ(3, x[3], hi)
    assert out[4] == pytest.approx(m / (x[5] - x[4]), rel=1e-14)


# ---------------------------------------------------------------------------
# residual step
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("scheme", [oracle.DONOR, oracle.VANLEER])
def test_residual_zero_velocity_identity(scheme):
    x = wl.random_nodes(64, seed=23)
    q = np.random.default_rng(24).random(64)
    out = oracle.residual(x, q, np.zeros(64), 0.1, scheme)
    assert np.array_equal(out, q)


@pytest.mark.parametrize("scheme", [oracle.DONOR, oracle.VANLEER])
def test_residual_cfl_one_is_a_roll(scheme):
    """Sec. 4.1 footnote: moving exactly one cell per step is exact on a uniform mesh."""
    n = 64
    x = wl.uniform_nodes(n)
    q = np.random.default_rng(25).random(n)
    dt = 0.5
    out = oracle.residual(x, q, np.full(n, (1.0 / n) / dt), dt, scheme)
    np.testing.assert_allclose(out, np.roll(q, 1), rtol=0, atol=1e-14)
    out = oracle.residual(x, q, np.full(n, -(1.0 / n) / dt), dt, scheme)
    np.testing.assert_allclose(out, np.roll(q, -1), rtol=0, atol=1e-14)


@pytest.mark.parametrize("scheme", [oracle.DONOR, oracle.VANLEER])
def test_residual_conserves_and_bounds(scheme):
    n = 200
    x = wl.random_nodes(n, seed=26)
    q = wl.tophat_averages(x, 0.2, 0.4) + 0.5
    dv = 0.3 * np.sin(2 * np.pi * x[:-1]) * np.diff(x).min() / 0.1
    out = q
    for _ in range(10):
        out = oracle.residual(x, out, dv, 0.1, scheme, nsub=2)
    m0 = oracle.mass(x, q)
    assert abs(oracle.mass(x, out) - m0) <= 1e-14 * m0
    # with a constant velocity (no compression) donor cell adds no extrema
    dvc = np.full(n, 0.7 * np.diff(x).min() / 0.1)
    out = q
    for _ in range(10):
        out = oracle.residual(x, out, dvc, 0.1, scheme)
    if scheme == oracle.DONOR:
        assert out.min() >= q.min() - 1e-14 and out.max() <= q.max() + 1e-14


def test_residual_cfl_flag():
    n = 32
    x = wl.uniform_nodes(n)
    q = np.ones(n)
    _, st = oracle.residual(x, q, np.full(n, 2.0), 1.0 / n, oracle.DONOR,
                            return_status=True)
    assert st == 3
    _, st = oracle.residual(x, q, np.full(n, 2.0), 1.0 / n, oracle.DONOR, nsub=2,
                            return_status=True)
    assert st == 0


def test_subcycles_equal_repeated_steps():
    n = 50
    x = wl.random_nodes(n, seed=27)
    q = wl.three_gaussians(x, 28)
    dv = 0.02 * np.cos(2 * np.pi * x[:-1])
    a = oracle.residual(x, q, dv, 0.3, oracle.VANLEER, nsub=3)
    b = q
    for _ in range(3):
        b = oracle.residual(x, b, dv, 0.1, oracle.VANLEER)
    np.testing.assert_allclose(a, b, rtol=1e-14, atol=0)


def test_phase_update():
    L = 2 * np.pi
    ph = 0.0
    for _ in range(1000):
        ph = oracle.phase_update(ph, 3.3, 0.7, L)
        assert 0.0 <= ph < L
    assert ph == pytest.approx(math.fmod(1000 * 3.3 * 0.7, L), abs=1e-9)


# ---------------------------------------------------------------------------
# transpose of the linear step
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("s", [0.013, 0.41, -1.73])
def test_shift_adjoint_dot_product(order, s):
    n = 90
    x = wl.random_nodes(n, seed=51)
    rng = np.random.default_rng(52)
    u, v = rng.standard_normal(n), rng.standard_normal(n)
    Au = oracle.shift(x, u, s, order, False)
    ATv = oracle.shift_adjoint(x, v, s, order)
    lhs, rhs = float(Au @ v), float(u @ ATv)
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(Au) @ np.abs(v))


@pytest.mark.parametrize("order", [2, 3, 4])
def test_shift_adjoint_dense_transpose(order):
    n = 24
    x = wl.random_nodes(n, seed=53)
    s = 0.377
    A = np.stack([oracle.shift(x, e, s, order, False) for e in np.eye(n)], axis=1)
    AT = np.stack([oracle.shift_adjoint(x, e, s, order) for e in np.eye(n)], axis=1)
    np.testing.assert_allclose(AT, A.T, rtol=0, atol=1e-13)


def test_step_adjoint_dense_transpose_with_donor_residual():
    n = 20
    x = wl.random_nodes(n, seed=54)
    rng = np.random.default_rng(55)
    dv = rng.uniform(-1, 1, n) * np.diff(x).min()
    dt, s = 0.6, 0.31
    A = np.stack([oracle.step(x, e, s, 3, False, dv, dt, oracle.DONOR, 2)
                  for e in np.eye(n)], axis=1)
    AT = np.stack([oracle.step_adjoint(x, np.zeros(n), e, s, 3, dv, dt, 2)[0]
                   for e in np.eye(n)], axis=1)
    np.testing.assert_allclose(AT, A.T, rtol=0, atol=1e-13)


def test_step_adjoint_dv_gradient_vs_finite_differences():
    """d loss / d dv of the donor step against central differences; dv is kept
    away from zero so that no upwind side flips under the perturbation."""
    n = 40
    x = wl.random_nodes(n, seed=56)
    rng = np.random.default_rng(57)
    q = wl.three_gaussians(x, 58)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    dv = sign * (0.3 + 0.5 * rng.random(n)) * np.diff(x).min()
    dt, s, nsub = 0.5, 0.123, 2
    g = rng.standard_normal(n)
    _, gdv = oracle.step_adjoint(x, q, g, s, 2, dv, dt, nsub)

    def loss(d):
        return float(g @ oracle.step(x, q, s, 2, False, d, dt, oracle.DONOR, nsub))

    h = 1e-6 * np.diff(x).min()
    for k in range(8):
        e = rng.standard_normal(n)
        fd = (loss(dv + h * e) - loss(dv - h * e)) / (2 * h)
        assert fd == pytest.approx(float(gdv @ e), rel=1e-6, abs=1e-9)


# ---------------------------------------------------------------------------
# the batched driver over packed rows (rows are independent, Sec. 3.5)
# ---------------------------------------------------------------------------

def _packed_rows(lens, seed, uniform=False):
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nodes = np.concatenate([wl.uniform_nodes(n) if uniform else
                            wl.random_nodes(n, seed=seed + r, x0=0.1 * r)
                            for r, n in enumerate(lens)])
    return ro, nodes


def test_step_rows_per_row_meshes_equal_single_rows():
    """The batched driver gives, bit for bit, the single-row step of every row:
    per-row meshes of different lengths, mixed orders, per-row shifts and
    sub-step counts, with a residual."""
    lens = [17, 64, 5, 230, 1, 99]
    ro, nodes = _packed_rows(lens, 60)
    rng = np.random.default_rng(61)
    order = np.array([2, 3, 4, 3, 2, 4], dtype=np.int8)
    nsub = np.array([1, 3, 2, 1, 4, 2], dtype=np.int32)
    shifts = rng.uniform(-3, 3, len(lens))
    q = 1.0 + rng.random(int(ro[-1]))
    dt = 0.05
    dv = np.concatenate([0.4 * (rng.random(n) - 0.5) * np.diff(nodes[ro[r] + r: ro[r + 1] + r + 1]).min() / dt
                         for r, n in enumerate(lens)])
    for limiter in (True, False):
        got = oracle.step_rows(ro, nodes, False, order, limiter, shifts, q, dv=dv, dt=dt,
                               scheme=oracle.VANLEER, nsub=nsub)
        for r, n in enumerate(lens):
            sl = slice(int(ro[r]), int(ro[r + 1]))
            x = nodes[ro[r] + r: ro[r + 1] + r + 1]
            ref = oracle.step(x, q[sl], shifts[r], int(order[r]), limiter, dv[sl], dt,
                              oracle.VANLEER, int(nsub[r]))
            assert np.array_equal(got[sl], ref), (limiter, r)


def test_step_rows_shared_mesh_equal_single_rows():
    """RAM_SHARED_MESH form: every row takes the first row's nodes."""
    n, rows = 48, 5
    x = wl.random_nodes(n, seed=62, x0=-1.0)
    ro = np.arange(rows + 1, dtype=np.int64) * n
    rng = np.random.default_rng(63)
    q = 1.0 + rng.random(rows * n)
    shifts = rng.uniform(-2, 2, rows)
    order = np.array([3, 2, 4, 3, 2], dtype=np.int8)
    got = oracle.step_rows(ro, x, True, order, True, shifts, q)
    for r in range(rows):
        sl = slice(r * n, (r + 1) * n)
        assert np.array_equal(got[sl], oracle.step(x, q[sl], shifts[r], int(order[r]), True))


def test_step_rows_whole_cell_rolls():
    """Independent of the single-row driver: per-row uniform dyadic meshes of
    different lengths, each shifted by its own whole number of cells, give the
    cyclic permutation of each row (Sec. 1, Eq. 8) bit for bit."""
    lens = [8, 32, 16, 64]
    ro, nodes = _packed_rows(lens, 0, uniform=True)
    rng = np.random.default_rng(64)
    q = rng.random(int(ro[-1]))
    ks = [3, -5, 16, 63]
    shifts = np.array([k / n for k, n in zip(ks, lens)])
    got = oracle.step_rows(ro, nodes, False, np.array([2, 3, 4, 3], dtype=np.int8), False,
                           shifts, q)
    for r, (n, k) in enumerate(zip(lens, ks)):
        sl = slice(int(ro[r]), int(ro[r + 1]))
        assert np.array_equal(got[sl], np.roll(q[sl], k)), r


# ---------------------------------------------------------------------------
# the fourth-order cell-average correction (Sec. 3.1) and the limited order 4
# ---------------------------------------------------------------------------

def test_a4_averages_are_exact_for_cubics():
    """Point values of a cubic at the cell centres of a uniform mesh: the A4 formula
    gives the exact cell averages (away from the periodic seam, where the cubic
    itself is not periodic)."""
    n = 40
    x = wl.uniform_nodes(n, -1.0, 2.0)
    c = np.array([0.3, -1.2, 0.7, 2.1])  # c0 + c1 t + c2 t^2 + c3 t^3
    xc = 0.5 * (x[1:] + x[:-1])
    pts = np.polyval(c[::-1], xc)
    prim = np.polyint(c[::-1])
    exact = (np.polyval(prim, x[1:]) - np.polyval(prim, x[:-1])) / np.diff(x)
    avg = oracle.a4_average(pts)
    np.testing.assert_allclose(avg[1:-1], exact[1:-1], rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64])
def test_a4_inverse_round_trip_and_sum(n):
    """The point values recovered from the corrected averages are the original ones,
    and the correction keeps the sum (Eq. 10 on a periodic uniform mesh)."""
    q = 1.0 + np.random.default_rng(n).random(n)
    avg = oracle.a4_average(q)
    np.testing.assert_allclose(oracle.a4_point(avg), q, rtol=0, atol=1e-14)
    assert abs(avg.sum() - q.sum()) <= 1e-14 * q.sum()
    # the inverse is an independent solve: check A4(a4_point(b)) == b for any b
    b = np.random.default_rng(n + 1).standard_normal(n)
    np.testing.assert_allclose(oracle.a4_average(oracle.a4_point(b)), b, rtol=0, atol=1e-14)


@pytest.mark.parametrize("limiter", [True, False])
def test_a4_step_conservation_roll_and_identity(limiter):
    n = 96
    x = wl.uniform_nodes(n)
    q = wl.three_gaussians(x, 7)
    m0 = q.sum()
    for s in (0.0, 0.37, -2.71, 5.0 / n, 123.456):
        out = oracle.step_a4(x, q, s, limiter)
        assert abs(out.sum() - m0) <= 1e-13 * m0, s
    np.testing.assert_allclose(oracle.step_a4(x, q, 0.0, limiter), q, rtol=0, atol=1e-14)
    # a whole-cell shift commutes with the circulant correction: a cyclic roll
    np.testing.assert_allclose(oracle.step_a4(x, q, 7.0 / n, limiter), np.roll(q, 7),
                               rtol=0, atol=1e-13)


def test_a4_interface_values_fourth_order():
    """Sec. 3.1: identifying <Q>_i with the point value Q_i is second order, which
    limits the PPM interface values; with the corrected averages they converge at
    fourth order (smooth periodic function sampled at the cell centres; unlimited
    PPM faces against the exact values at the nodes)."""
    def f(t):
        return np.sin(2 * np.pi * t) + 0.4 * np.cos(6 * np.pi * t + 0.3)

    ns = [32, 64, 128, 256]
    errs = {False: [], True: []}
    for n in ns:
        x = wl.uniform_nodes(n)
        pts = f(0.5 * (x[1:] + x[:-1]))
        for a4 in (False, True):
            avg = oracle.a4_average(pts) if a4 else pts
            qr = oracle.reconstruct(x, avg, order=3, limiter=False)[:, 1]  # QR_i = face i+1/2
            errs[a4].append(np.max(np.abs(qr - f(x[1:]))))
    slope = {k: -np.polyfit(np.log(ns), np.log(v), 1)[0] for k, v in errs.items()}
    assert abs(slope[False] - 2.0) < 0.2, slope
    assert slope[True] > 3.8, slope


def test_limited_order4_keeps_linear_profiles():
    """A linear profile is reproduced by the quartic and already inside the
    neighbours' range: the limiter leaves it alone."""
    n = 60
    x = wl.random_nodes(n, seed=70, ratio=1.5)
    xc = 0.5 * (x[1:] + x[:-1])
    q = 2.0 + 0.5 * xc
    cells = np.arange(5, 55)
    d = 0.37 * np.diff(x)[cells]
    a = oracle.cell_cumulative(x, q, cells, d, order=4, limiter=True)
    b = oracle.cell_cumulative(x, q, cells, d, order=4, limiter=False)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_limited_order4_profile_inside_neighbour_range(seed):
    """Brute force: the limited profile dG/dx, sampled densely in every cell, stays
    within [min, max] of the cell and its two neighbours, and integrates to the
    cell's mass."""
    n = 30
    x = wl.random_nodes(n, seed=80 + seed, ratio=3.0)
    q = np.random.default_rng(seed).random(n)
    q[10:15] = 3.0  # a plateau: the unlimited quartic overshoots next to it
    dx = np.diff(x)
    m = 400
    for i in range(n):
        d = np.linspace(0.0, dx[i], m + 1)
        G = oracle.cell_cumulative(x, q, np.full(m + 1, i), d, order=4, limiter=True)
        # the profile dG/dx at the sample points, by differences of step eps
        eps = 1e-7 * dx[i]
        dl = np.clip(d - eps, 0.0, dx[i])
        dr = np.clip(d + eps, 0.0, dx[i])
        Gl = oracle.cell_cumulative(x, q, np.full(m + 1, i), dl, order=4, limiter=True)
        Gr = oracle.cell_cumulative(x, q, np.full(m + 1, i), dr, order=4, limiter=True)
        prof = (Gr - Gl) / (dr - dl)
        lo = min(q[i - 1], q[i], q[(i + 1) % n])
        hi = max(q[i - 1], q[i], q[(i + 1) % n])
        assert prof.min() >= lo - 1e-7 and prof.max() <= hi + 1e-7, i
        assert abs(G[-1] - q[i] * dx[i]) <= 1e-13 * abs(q[i] * dx[i])
        # where the limiter acts, theta is the largest admissible value: the
        # scaled profile reaches one of the bounds
        Gu = oracle.cell_cumulative(x, q, np.full(m + 1, i), d, order=4, limiter=False)
        if np.max(np.abs(G - Gu)) > 1e-12 * abs(q[i] * dx[i]):
            gap = min(hi - prof.max(), prof.min() - lo)
            assert gap <= 1e-5 * (hi - lo), (i, gap)


def test_limited_order4_no_new_extrema_and_conservation():
    """The limited order 4 creates no new extrema on a square wave over many shifts
    (the unlimited one overshoots) and conserves the mass (Eq. 10)."""
    n = 128
    x = wl.random_nodes(n, seed=90, ratio=2.0)
    xc = 0.5 * (x[1:] + x[:-1])
    q0 = np.where((xc > 0.3) & (xc < 0.6), 1.0, 0.0)
    ql, qu = q0.copy(), q0.copy()
    for _ in range(20):
        ql = oracle.shift(x, ql, 0.0173, 4, True)
        qu = oracle.shift(x, qu, 0.0173, 4, False)
    assert ql.max() <= 1.0 + 1e-12 and ql.min() >= -1e-12
    assert qu.max() > 1.0 + 1e-3 or qu.min() < -1e-3
    assert abs(oracle.mass(x, ql) - oracle.mass(x, q0)) <= 1e-13 * oracle.mass(x, q0)


# ---------------------------------------------------------------------------
# two dimensions by dimensional splitting (Sec. 3.5), the radial bump (App. B.2)
# ---------------------------------------------------------------------------

def _ring_areas(rf):
    return 0.5 * (rf[1:] ** 2 - rf[:-1] ** 2)


@pytest.mark.parametrize("scheme", [oracle.DONOR, oracle.VANLEER])
def test_radial_sweep_conserves_mass(scheme):
    """Closed radial walls: sum over rings of q times ring area is conserved."""
    rf = wl.radial_bump_nodes(40, 0.4, 2.1, 1.0, 0.1387, 0.2773, 2.5)
    rng = np.random.default_rng(1)
    q = 1.0 + rng.random((40, 16))
    vr = 0.2 * (rng.random((41, 16)) - 0.5) * np.diff(rf).min()
    vr[0] = vr[-1] = 0.0
    out = oracle.radial_upwind(rf, q, vr, 1.0, scheme)
    area = _ring_areas(rf)
    np.testing.assert_allclose((out * area[:, None]).sum(axis=0), (q * area[:, None]).sum(axis=0),
                               rtol=1e-14)


def test_radial_sweep_divergence_free_flow_keeps_a_constant():
    """r vr constant on the interior faces: the flux divergence vanishes in every ring
    that has two open faces, so a constant density stays constant there (cylindrical
    geometry; a planar update would not)."""
    rf = np.linspace(0.5, 2.0, 31)
    q = np.full((30, 4), 2.5)
    vr = np.zeros((31, 4))
    vr[1:-1] = 0.01 / rf[1:-1, None]
    for scheme in (oracle.DONOR, oracle.VANLEER):
        out = oracle.radial_upwind(rf, q, vr, 0.7, scheme)
        np.testing.assert_allclose(out[1:-1], 2.5, rtol=1e-14)
        assert out[0, 0] < 2.5 and out[-1, 0] > 2.5  # the walls stop the flow


def test_radial_sweep_planar_limit_is_a_shift():
    """Far from the axis (thin annulus) a donor sweep at Courant number 1 with r vr
    constant moves every ring's value to the next ring, to O(dr / r)."""
    n = 20
    r0 = 1.0e6
    rf = r0 + np.arange(n + 1, dtype=np.float64)
    q = np.random.default_rng(2).random((n, 3))
    vr = np.zeros((n + 1, 3))
    vr[1:-1] = r0 / rf[1:-1, None]  # ~1: one ring width per unit time
    out = oracle.radial_upwind(rf, q, vr, 1.0, oracle.DONOR)
    np.testing.assert_allclose(out[1:-1], q[:-2], atol=1e-4)


def test_radial_sweep_donor_positive_and_cfl_flag():
    rf = np.linspace(0.4, 2.1, 25)
    rng = np.random.default_rng(3)
    q = rng.random((24, 8))
    vr = (rng.random((25, 8)) - 0.5) * 2.0 * np.diff(rf).min()
    vr[0] = vr[-1] = 0.0
    out, st = oracle.radial_upwind(rf, q, vr, 0.45, oracle.DONOR, return_status=True)
    assert st == 0 and out.min() >= 0.0
    _, st = oracle.radial_upwind(rf, q, vr * 4.0, 1.0, oracle.DONOR, return_status=True)
    assert st == 3


def test_shear_limit_bounds_the_relative_shift_of_neighbouring_rings():
    """With the shear limit, no two neighbouring rings move apart by more than beta
    azimuthal cells in one step, and one pair does by exactly that."""
    rf = wl.radial_bump_nodes(64, 0.4, 2.1, 1.0, 0.1387, 0.2773, 2.5)
    rc = 0.5 * (rf[1:] + rf[:-1])
    omega = rc ** -1.5 - 1.0
    dphi = 2 * np.pi / 300
    dt = oracle.shear_dt(omega, dphi, 0.44)
    rel = np.abs(np.diff(omega)) * dt
    assert rel.max() <= 0.44 * dphi * (1 + 1e-14)
    assert abs(rel.max() - 0.44 * dphi) <= 1e-14 * dphi
    assert oracle.shear_dt(np.full(5, 0.7), dphi, 0.44) == np.inf


def test_radial_bump_mesh():
    """App. B.2: the normalisation I = log(x_max / x_min) + c (a + b) by quadrature,
    the faces' density integrals equal, and c = 0 gives the log-uniform mesh."""
    import scipy.integrate as si
    a, b, c = 0.1387, 0.2773, 2.5
    I_q, _ = si.quad(lambda s: wl.radial_bump_density(s, 1.0, a, b, c), 0.4, 2.1,
                     points=[1 - b, 1 - a, 1 + a, 1 + b], limit=200)
    assert abs(I_q - wl.radial_bump_norm(0.4, 2.1, a, b, c)) <= 1e-12 * I_q
    rf = wl.radial_bump_nodes(50, 0.4, 2.1, 1.0, a, b, c)
    pieces = [si.quad(lambda s: wl.radial_bump_density(s, 1.0, a, b, c), rf[j], rf[j + 1],
                      epsabs=0.0, epsrel=1e-13, limit=200)[0] for j in range(50)]
    np.testing.assert_allclose(pieces, I_q / 50, rtol=1e-9)
    logu = wl.radial_bump_nodes(16, 0.4, 2.1, 1.0, a, b, 0.0)
    np.testing.assert_allclose(logu, 0.4 * (2.1 / 0.4) ** (np.arange(17) / 16), rtol=1e-13)


def test_split_step_is_the_ring_steps_then_the_radial_sweep():
    """The split step with no radial flow is the RAM step of every ring; with no
    rotation and no residual it is the radial sweep alone."""
    d = wl.polar_disk_2d(n_r=12, n_phi=64)
    rows = np.stack([oracle.step(d.phi, d.q0[j], oracle.shift_from_velocity(d.omega[j], d.dt),
                                 d.order, True, d.dvphi[j], d.dt, d.scheme, int(d.nsub[j]))
                     for j in range(12)])
    got = oracle.step_2d(d.phi, d.rf, d.omega, d.q0, d.dt, d.order, True, d.dvphi, d.scheme,
                         d.nsub, np.zeros_like(d.vr))
    np.testing.assert_array_equal(got, rows)
    got = oracle.step_2d(d.phi, d.rf, np.zeros(12), d.q0, d.dt, d.order, True, None, d.scheme,
                         None, d.vr)
    np.testing.assert_array_equal(got, oracle.radial_upwind(d.rf, d.q0, d.vr, d.dt, d.scheme))


# ---------------------------------------------------------------------------
# the step linearised at a forward state (limited PLM / PPM)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("order", [2, 3])
def test_linearisation_without_limiter_is_the_linear_transpose(order):
    """With the limiter off the step is linear: the transpose of the tangent equals
    the hand-derived transpose of the linear step."""
    x = wl.random_nodes(48, seed=100 + order)
    rng = np.random.default_rng(order)
    q0, g = 1.0 + rng.random(48), rng.standard_normal(48)
    np.testing.assert_allclose(oracle.shift_vjp(x, q0, g, 0.417, order, False),
                               oracle.shift_adjoint(x, g, 0.417, order), rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_limited_ppm_tangent_is_exact_within_its_branches(seed):
    """The limited PPM is piecewise linear in Q (App. A.2 selects among linear
    expressions): along a direction small enough to keep every branch, the step's
    increment is exactly the tangent times the step length."""
    x = wl.random_nodes(64, seed=110 + seed)
    rng = np.random.default_rng(seed)
    q0 = wl.three_gaussians(x, seed) + 0.3 * rng.random(64)
    v = rng.standard_normal(64)
    eps = 1e-7
    jv = oracle.shift_jvp(x, q0, v, 0.3713, 3, True)
    inc = (oracle.shift(x, q0 + eps * v, 0.3713, 3, True) - oracle.shift(x, q0, 0.3713, 3, True)) / eps
    assert np.max(np.abs(inc - jv)) <= 1e-6 * np.max(np.abs(jv))


@pytest.mark.parametrize("order", [2, 3])
def test_limited_tangent_against_central_differences(order):
    x = wl.random_nodes(50, seed=120 + order)
    rng = np.random.default_rng(120 + order)
    q0 = 1.0 + rng.random(50)
    for s in (0.011, 0.77, -2.3):
        v = rng.standard_normal(50)
        h = 1e-6
        fd = (oracle.shift(x, q0 + h * v, s, order, True) - oracle.shift(x, q0 - h * v, s, order, True)) / (2 * h)
        jv = oracle.shift_jvp(x, q0, v, s, order, True)
        assert np.max(np.abs(fd - jv)) <= 1e-6 * np.max(np.abs(jv)), s


def test_limited_step_adjoint_dot_product_and_dv_gradient():
    """The step linearised at q (limited PPM shift, donor residual): <g, R J v> =
    <J^T R^T g, v> with the donor residual R linear in its input, and d<g, step>/d dv
    against central differences."""
    n = 40
    x = wl.random_nodes(n, seed=130)
    rng = np.random.default_rng(131)
    q = wl.three_gaussians(x, 132)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    dv = sign * (0.3 + 0.5 * rng.random(n)) * np.diff(x).min()
    dt, s, nsub = 0.5, 0.2217, 2
    g = rng.standard_normal(n)
    gi, gdv = oracle.step_adjoint_limited(x, q, g, s, 3, True, dv, dt, nsub)
    v = rng.standard_normal(n)
    rjv = oracle.residual(x, oracle.shift_jvp(x, q, v, s, 3, True), dv, dt, oracle.DONOR, nsub)
    assert abs(g @ rjv - gi @ v) <= 1e-12 * (np.abs(g) @ np.abs(rjv))

    def loss(d):
        return float(g @ oracle.step(x, q, s, 3, True, d, dt, oracle.DONOR, nsub))

    h = 1e-6 * np.diff(x).min()
    for k in range(5):
        e = rng.standard_normal(n)
        fd = (loss(dv + h * e) - loss(dv - h * e)) / (2 * h)
        assert fd == pytest.approx(float(gdv @ e), rel=1e-6, abs=1e-9)
