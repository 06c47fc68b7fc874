"""The paper's 1D advection test (Sec. 4.1, Fig. 2) on the oracle.

The paper prints slopes, not errors: e1 ~ N^-2 for the smooth profile with PLM
and PPM, e1 ~ N^-3/4 for the square profile, on a uniform and on a
periodic-bump mesh.  The fixture in tests/golden/fig2_convergence.json holds the
printed values and the setup."""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from paper_2305_05362_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


FIG2 = _load("fig2_convergence.json")


def _mesh(kind, n):
    lo, hi = FIG2["setup"]["domain"]
    if kind == "uniform":
        return wl.uniform_nodes(n, lo, hi - lo)
    b = FIG2["setup"]["bump_mesh"]
    return wl.bump_nodes(n, lo, hi, b["a"], b["a"] + b["b_minus_a"], b["c"])


def _e1(kind, n, order, profile):
    st = FIG2["setup"]
    x = _mesh(kind, n)
    xc = 0.5 * (x[1:] + x[:-1])
    if profile == "smooth":
        q0 = 2.0 / math.pi * np.exp(-4.0 * xc ** 2 / math.pi)
    else:
        q0 = np.where(np.abs(xc) <= math.pi / 2, 0.75, 0.25) / math.pi
    v0, t_end = st["v0"], st["t_end"]
    dt = st["beta_ram"] * np.diff(x).min() / v0
    q, t = q0.copy(), 0.0
    while t < t_end - 1e-12:
        h = min(dt, t_end - t)
        q = oracle.shift(x, q, v0 * h, order, True)
        t += h
    return float(np.sum(np.abs(q - q0) * np.diff(x)) / np.sum(np.diff(x)))


@pytest.mark.parametrize("kind", ["uniform", "bump"])
@pytest.mark.parametrize("profile", ["smooth", "square"])
def test_fig2_slopes(kind, profile):
    ns = FIG2["setup"]["N"]
    errs = {o: [_e1(kind, n, o, profile) for n in ns] for o in (2, 3)}
    target = FIG2["printed"]["%s_slope" % profile]
    tol = FIG2["tolerance"]["%s_slope" % profile]
    for o in (2, 3):
        slope = np.polyfit(np.log(ns), np.log(errs[o]), 1)[0]
        assert abs(slope - target) <= tol, (kind, profile, o, slope)
    # PLM errors are larger than PPM errors (Sec. 4.1)
    assert all(a > b for a, b in zip(errs[2], errs[3]))


def test_bump_normalisation_and_mesh():
    """App. B.1: the printed normalisation of the bump density matches a
    quadrature of the density, and the bisection mesh puts an equal share of the
    density into every cell (Eq. 22)."""
    for c in _load("bump_normalisation.json")["cases"]:
        args = (c["a"], c["b"], c["c"])
        num = quad(lambda s: float(wl.bump_density(s, *args)), c["x_min"], c["x_max"],
                   points=[-c["b"], -c["a"], c["a"], c["b"]], limit=200)[0]
        assert wl.bump_norm(c["x_min"], c["x_max"], *args) == pytest.approx(num, rel=1e-12)
        x = wl.bump_nodes(64, c["x_min"], c["x_max"], *args)
        share = [quad(lambda s: float(wl.bump_density(s, *args)), x[i], x[i + 1],
                      limit=100)[0] for i in range(64)]
        np.testing.assert_allclose(share, num / 64, rtol=1e-9)
