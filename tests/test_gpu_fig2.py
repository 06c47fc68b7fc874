"""The paper's 1D advection test (Sec. 4.1, Fig. 2) on the GPU, through the C ABI.

All cases run as rows of one plan: uniform and periodic-bump meshes (App. B.1,
the non-uniform path with its tabulated index function), N = 32..512, PLM and
PPM, the smooth and the square profile -- 40 uneven rows with their own meshes,
orders and time steps, advanced with one ram_shift launch per step (a row that
has reached t_end gets a zero shift, which copies it).  Checks: the e1 slopes
the paper prints (e1 ~ N^-2 smooth, N^-3/4 square; tests/golden/
fig2_convergence.json), PLM errors above PPM's, and the final fields against the
FP64 oracle (the last step from the GPU's own input, and the whole trajectory;
FP64: relative L1 <= 1e-12 per row, FP32: <= 1e-5)."""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2305_05362_gb300 import ram, workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
with open(os.path.join(os.path.dirname(__file__), "golden", "fig2_convergence.json")) as f:
    FIG2 = json.load(f)


def _mesh(kind, n):
    lo, hi = FIG2["setup"]["domain"]
    if kind == "uniform":
        return wl.uniform_nodes(n, lo, hi - lo)
    b = FIG2["setup"]["bump_mesh"]
    return wl.bump_nodes(n, lo, hi, b["a"], b["a"] + b["b_minus_a"], b["c"])


def _q0(x, profile):
    xc = 0.5 * (x[1:] + x[:-1])
    if profile == "smooth":
        return 2.0 / math.pi * np.exp(-4.0 * xc ** 2 / math.pi)
    return np.where(np.abs(xc) <= math.pi / 2, 0.75, 0.25) / math.pi


def _cases():
    return [(kind, profile, order, n) for kind in ("uniform", "bump")
            for profile in ("smooth", "square") for order in (2, 3)
            for n in FIG2["setup"]["N"]]


def _schedule(xs):
    """Per-row step lengths (the paper's beta dx_min / v0, the last step cut to
    t_end) as a (steps, rows) array of shifts v0 h, zero once a row is done."""
    st = FIG2["setup"]
    v0, t_end = st["v0"], st["t_end"]
    cols = []
    for x in xs:
        dt = st["beta_ram"] * np.diff(x).min() / v0
        t, hs = 0.0, []
        while t < t_end - 1e-12:
            h = min(dt, t_end - t)
            hs.append(v0 * h)
            t += h
        cols.append(hs)
    steps = max(len(c) for c in cols)
    sh = np.zeros((steps, len(xs)))
    for r, c in enumerate(cols):
        sh[:len(c), r] = c
    return sh, [len(c) for c in cols]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_fig2_on_gpu(dtype):
    cases = _cases()
    xs = [_mesh(kind, n) for kind, _, _, n in cases]
    q0s = [_q0(x, profile) for x, (_, profile, _, _) in zip(xs, cases)]
    lens = [x.size - 1 for x in xs]
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    plan = ram.Plan(ro, np.concatenate(xs), order=np.array([c[2] for c in cases], np.int8),
                    limiter=True)
    sh, n_steps = _schedule(xs)
    shd = torch.tensor(sh, dtype=torch.float64, device=DEV)
    q = torch.tensor(np.concatenate(q0s), dtype=dtype, device=DEV)
    buf = torch.empty_like(q)
    hist = []  # the GPU state before every step
    for k in range(sh.shape[0]):
        hist.append(q.double().cpu().numpy())
        ram.shift(plan, q, buf, shd[k])
        q, buf = buf, q
    torch.cuda.synchronize()
    assert plan.check_errors() == 0
    got = q.double().cpu().numpy()

    # against the oracle: the last step of every row from the GPU's own input, and
    # the whole trajectory from the same (rounded) start, both at the stated
    # tolerance (FP64 1e-12, FP32 1e-5)
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    for r, (x, q0) in enumerate(zip(xs, q0s)):
        sl = slice(int(ro[r]), int(ro[r + 1]))
        g = got[sl]
        w_ = np.diff(x)
        last = n_steps[r] - 1
        one = oracle.shift(x, hist[last][sl], sh[last, r], cases[r][2], True)
        err1 = np.sum(np.abs(g - one) * w_) / np.sum(np.abs(one) * w_)
        assert err1 <= tol, (cases[r], "last step", err1)
        ref = np.asarray(torch.tensor(q0, dtype=dtype).double().numpy())
        for k in range(n_steps[r]):
            ref = oracle.shift(x, ref, sh[k, r], cases[r][2], True)
        err = np.sum(np.abs(g - ref) * w_) / np.sum(np.abs(ref) * w_)
        assert err <= tol, (cases[r], n_steps[r], err)

    # the slopes the paper prints, and PLM above PPM
    e1 = {}
    for r, ((kind, profile, order, n), x, q0) in enumerate(zip(cases, xs, q0s)):
        g = got[ro[r]:ro[r + 1]]
        e1[(kind, profile, order, n)] = float(np.sum(np.abs(g - q0) * np.diff(x)) / np.sum(np.diff(x)))
    ns = FIG2["setup"]["N"]
    for kind in ("uniform", "bump"):
        for profile in ("smooth", "square"):
            target = FIG2["printed"]["%s_slope" % profile]
            tol = FIG2["tolerance"]["%s_slope" % profile]
            errs = {o: [e1[(kind, profile, o, n)] for n in ns] for o in (2, 3)}
            for o in (2, 3):
                slope = np.polyfit(np.log(ns), np.log(errs[o]), 1)[0]
                assert abs(slope - target) <= tol, (kind, profile, o, slope)
            assert all(a > b for a, b in zip(errs[2], errs[3])), (kind, profile)


def _densities(cases):
    """The periodic bump of every bump row (App. B.1); uniform rows take none."""
    lo, hi = FIG2["setup"]["domain"]
    b = FIG2["setup"]["bump_mesh"]
    return [(lo, hi, b["a"], b["a"] + b["b_minus_a"], b["c"]) for _ in cases]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nseg", [False, True])
def test_fig2_with_the_index_function(dtype, nseg):
    """The same runs with the bump rows located by the index function of Sec. 3.2.1
    (p = floor(N u(x~)) from the closed-form cumulative, App. B.1) instead of the
    plan's bucket table: the located cells are exact either way, so the fields are
    identical bit for bit, and the printed slopes hold."""
    if nseg and dtype == torch.float64:
        pytest.skip("the warp-segment kernel is FP32")
    cases = _cases()
    xs = [_mesh(kind, n) for kind, _, _, n in cases]
    q0s = [_q0(x, profile) for x, (_, profile, _, _) in zip(xs, cases)]
    lens = [x.size - 1 for x in xs]
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    sh, n_steps = _schedule(xs)
    shd = torch.tensor(sh, dtype=torch.float64, device=DEV)
    finals = []
    for with_density in (False, True):
        plan = ram.Plan(ro, np.concatenate(xs), order=np.array([c[2] for c in cases], np.int8),
                        limiter=True)
        if nseg:
            t = plan.tuning()
            t.nonuniform_kernel_f32 = 1
            plan.set_tuning(t)
        if with_density:
            plan.set_density(_densities(cases))
            n_bump = sum(1 for c in cases if c[0] == "bump")
            assert plan.info().n_density_rows == n_bump
        q = torch.tensor(np.concatenate(q0s), dtype=dtype, device=DEV)
        buf = torch.empty_like(q)
        for k in range(sh.shape[0]):
            ram.shift(plan, q, buf, shd[k])
            q, buf = buf, q
        torch.cuda.synchronize()
        assert plan.check_errors() == 0
        finals.append(q.double().cpu().numpy())
    assert np.array_equal(finals[0], finals[1])
    got = finals[1]
    e1 = {}
    for r, ((kind, profile, order, n), x, q0) in enumerate(zip(cases, xs, q0s)):
        g = got[ro[r]:ro[r + 1]]
        e1[(kind, profile, order, n)] = float(np.sum(np.abs(g - q0) * np.diff(x)) / np.sum(np.diff(x)))
    ns = FIG2["setup"]["N"]
    for profile in ("smooth", "square"):
        target = FIG2["printed"]["%s_slope" % profile]
        tol = FIG2["tolerance"]["%s_slope" % profile]
        for o in (2, 3):
            slope = np.polyfit(np.log(ns), np.log([e1[("bump", profile, o, n)] for n in ns]), 1)[0]
            assert abs(slope - target) <= tol, (profile, o, slope)


def test_density_refused_for_other_nodes():
    """Nodes that are not the density's are refused (RAM_ERR_MESH), the plan unchanged."""
    n = 64
    lo, hi = FIG2["setup"]["domain"]
    b = FIG2["setup"]["bump_mesh"]
    plan = ram.Plan([0, n], wl.random_nodes(n, seed=3, x0=lo, length=hi - lo), order=3)
    with pytest.raises(ram.RamError) as e:
        plan.set_density([(lo, hi, b["a"], b["a"] + b["b_minus_a"], b["c"])])
    assert e.value.status == 2
    assert plan.info().n_density_rows == 0
