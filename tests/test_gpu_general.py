"""GPU parity of the non-uniform-mesh path against the FP64 oracle, through the C
ABI: FP64 relative L1 <= 1e-12, FP32 <= 1e-5 (per row)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2305_05362_gb300 import ram, workloads as wl
from gpu_common import TOL, oracle_shifts, oracle_step, rel_l1_rows

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
DT = {"float64": torch.float64, "float32": torch.float32}


def _t(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def _use_nseg(plan, on=True):
    """Select the FP32 warp-segment kernel for the plan's rows with their own mesh
    (the default is the per-order kernels)."""
    t = plan.tuning()
    t.nonuniform_kernel_f32 = 1 if on else 0
    plan.set_tuning(t)
    return plan


def _rounded(a, dtype):
    a = np.asarray(a, dtype=np.float64)
    return a.astype(np.float32).astype(np.float64) if dtype == "float32" else a


@pytest.mark.parametrize("dtype,nseg", [("float64", False), ("float32", False),
                                        ("float32", True)])
def test_line_nonuniform_c2(dtype, nseg):
    """4096 cells, log-uniform widths in [0.5, 2] x mean, three Gaussians, 40.7 mean
    cells per step, dv = 0.05 sin(4 pi x), PPM + van Leer, the recipe's 1000 steps.
    At steps 1, 10, 100 and 1000: the GPU step against the oracle step from the
    same (GPU) input, and the whole GPU trajectory against the FP64 oracle's own
    trajectory, both at the stated tolerance."""
    w = wl.line_nonuniform()
    plan = _use_nseg(ram.Plan.from_workload(w), nseg)
    assert plan.info().n_uniform_rows == 0
    q = _t(w.q0, DT[dtype])
    buf = torch.empty_like(q)
    dvd = _t(w.dv, DT[dtype])
    v0 = _t(w.v0, torch.float64)
    ref = q.double().cpu().numpy()
    dvr = dvd.double().cpu().numpy()
    shifts = oracle_shifts(w)
    for k in range(1, w.steps + 1):
        ram.step(plan, q, buf, v0, w.dt, dv=dvd, scheme=ram.VANLEER)
        ref = oracle_step(w, ref, shifts, dv=dvr, nsub=w.nsub)
        if k in (1, 10, 100, w.steps):
            torch.cuda.synchronize()
            got = buf.double().cpu().numpy()
            one = oracle_step(w, q.double().cpu().numpy(), shifts, dv=dvr, nsub=w.nsub)
            assert rel_l1_rows(w, got, one) <= TOL[dtype], (k, rel_l1_rows(w, got, one))
            assert rel_l1_rows(w, got, ref) <= TOL[dtype], (k, rel_l1_rows(w, got, ref))
        q, buf = buf, q
    assert plan.check_errors() == 0


@pytest.mark.parametrize("n", [1, 2, 3, 7, 40, 333, 1500, 4001])
@pytest.mark.parametrize("ratio", [1.5, 16.0])
@pytest.mark.parametrize("order,limiter", [(2, True), (2, False), (3, True), (3, False),
                                           (4, False)])
def test_random_meshes(n, ratio, order, limiter):
    """Random non-uniform rows from a single cell to several windowed tiles, strongly
    varying widths, shifts of many periods both ways, residual included; FP64."""
    x = wl.random_nodes(n, seed=n + int(ratio), ratio=ratio, x0=-0.25)
    rng = np.random.default_rng(n)
    q0 = 1.0 + rng.random(n)
    dxmin = np.diff(x).min()
    dt = 0.1
    dv = (rng.random(n) - 0.5) * 1.2 * dxmin / dt  # |dv| dt <= 0.6 dx_min
    plan = ram.Plan([0, n], x, order=order, limiter=limiter)
    plan.set_tiling(512, 128)  # non-uniform tiles of 256 cells: rows > ~600 are windowed
    qd, dvd = _t(q0, torch.float64), _t(dv, torch.float64)
    for s in (0.0, 0.3 * dxmin, 0.4321, 7.77, -3.1415):
        out = torch.empty_like(qd)
        v0 = _t([s / dt], torch.float64)
        ram.step(plan, qd, out, v0, dt, dv=dvd, scheme=ram.VANLEER)
        torch.cuda.synchronize()
        ref = oracle.step(x, q0, oracle.shift_from_velocity(s / dt, dt), order, limiter, dv, dt,
                          oracle.VANLEER, 1)
        err = np.sum(np.abs(out.cpu().numpy() - ref)) / np.sum(np.abs(ref))
        assert err <= 1e-12, (s, err)
    assert plan.check_errors() == 0


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("order", [2, 3, 4])
def test_long_row_windowed_tiles(dtype, order):
    """A 20000-cell row in tiles of 256 output cells: every tile locates its own source
    window through the bucket table; shift only and full step."""
    n = 20000
    x = wl.random_nodes(n, seed=77)
    q0 = _rounded(wl.three_gaussians(x, 78), dtype)
    plan = ram.Plan([0, n], x, order=order, limiter=(order != 4))
    plan.set_tiling(512, 256)
    assert plan.info().n_tiles_general > 20
    qd = _t(q0, DT[dtype])
    out = torch.empty_like(qd)
    for s in (123.4 / n, 0.5, 2.0 + 17.3 / n):
        ram.shift(plan, qd, out, _t([s], torch.float64))
        torch.cuda.synchronize()
        ref = oracle.shift(x, q0, s, order, order != 4)
        err = np.sum(np.abs(out.double().cpu().numpy() - ref)) / np.sum(np.abs(ref))
        assert err <= TOL[dtype], (s, err)
    assert plan.check_errors() == 0


def test_full_period_identity_nonuniform():
    """A shift by whole periods returns the input bit for bit on a non-uniform mesh
    (every shifted edge lands exactly on its own node: the exact-cover copy)."""
    for n in (5, 600, 3000):
        x = wl.random_nodes(n, seed=n)
        plan = ram.Plan([0, n], x, order=3)
        for dtype in (torch.float64, torch.float32):
            q = torch.rand(n, dtype=dtype, device=DEV) + 0.5
            out = torch.empty_like(q)
            for m in (1.0, 3.0, -2.0):
                ram.shift(plan, q, out, _t([m], torch.float64))
                torch.cuda.synchronize()
                assert torch.equal(out, q), (n, dtype, m)


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_mixed_uniform_and_nonuniform_rows(dtype):
    """One plan with uniform and non-uniform rows of assorted lengths and orders."""
    lens = [700, 64, 2048, 9, 1500, 4096]
    uni = [True, False, True, False, False, True]
    orders = np.array([3, 2, 4, 3, 4, 2], dtype=np.int8)
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nodes = np.concatenate([wl.uniform_nodes(n) if u else wl.random_nodes(n, seed=r)
                            for r, (n, u) in enumerate(zip(lens, uni))])
    rng = np.random.default_rng(9)
    q0 = _rounded(1.0 + rng.random(int(ro[-1])), dtype)
    dt = 0.2
    dv = np.concatenate([(rng.random(n) - 0.5) * 0.5 / n / dt for n in lens])
    dv = _rounded(dv, dtype)
    v0 = rng.uniform(-5, 5, len(lens)) / dt
    plan = ram.Plan(ro, nodes, order=orders, limiter=False)
    info = plan.info()
    assert info.n_uniform_rows == 3
    qd, dvd = _t(q0, DT[dtype]), _t(dv, DT[dtype])
    out = torch.empty_like(qd)
    ram.step(plan, qd, out, _t(v0, torch.float64), dt, dv=dvd, scheme=ram.DONOR)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    for r, n in enumerate(lens):
        sl = slice(int(ro[r]), int(ro[r + 1]))
        x = nodes[ro[r] + r: ro[r + 1] + r + 1]
        ref = oracle.step(x, q0[sl], oracle.shift_from_velocity(v0[r], dt), int(orders[r]), False,
                          dv[sl], dt, oracle.DONOR, 1)
        err = np.sum(np.abs(got[sl] - ref)) / np.sum(np.abs(ref))
        assert err <= TOL[dtype], (r, err)


@pytest.mark.parametrize("dtype,nseg", [("float32", False), ("float32", True),
                                        ("float64", False)])
def test_batched_uneven_rows(dtype, nseg):
    """The batched recipe (uneven rows with their own meshes, per-row shifts of
    0.3-200 mean cells, orders 2/3/4, limiter off), reduced to 40 rows of up to 8192
    cells, 20 steps: at steps 1, 5 and 20 the step from the GPU's own input and the
    trajectory against the FP64 oracle's, both at the stated tolerance."""
    w = wl.batched(n_rows=40, n_max=8192, steps=20)
    plan = _use_nseg(ram.Plan.from_workload(w), nseg)
    q = _t(w.q0, DT[dtype])
    buf = torch.empty_like(q)
    v0 = _t(w.v0, torch.float64)
    ref = q.double().cpu().numpy()
    shifts = oracle_shifts(w)
    for k in range(1, w.steps + 1):
        ram.step(plan, q, buf, v0, w.dt)
        ref = oracle_step(w, ref, shifts)
        if k in (1, 5, w.steps):
            torch.cuda.synchronize()
            got = buf.double().cpu().numpy()
            one = oracle_step(w, q.double().cpu().numpy(), shifts)
            assert rel_l1_rows(w, got, one) <= TOL[dtype], (k, rel_l1_rows(w, got, one))
            assert rel_l1_rows(w, got, ref) <= TOL[dtype], (k, rel_l1_rows(w, got, ref))
        q, buf = buf, q
    assert plan.check_errors() == 0


def test_row_mass_compensated_scan():
    """ram_row_mass uses the kernels' compensated scan: for FP32 cells its total
    matches the exact sum of the stored FP32 masses to 1e-12 relative; FP64 to 1e-13."""
    w = wl.batched(n_rows=24, n_min=1000, n_max=65536, seed_len=3)
    plan = ram.Plan.from_workload(w)
    q32 = w.q0.astype(np.float32)
    out = torch.empty(w.n_rows, dtype=torch.float64, device=DEV)
    ram.row_mass(plan, _t(q32, torch.float32), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for r in range(w.n_rows):
        sl = w.row_slice(r)
        dx32 = np.diff(w.row_nodes(r)).astype(np.float32).astype(np.float64)
        exact = math.fsum((q32[sl].astype(np.float64) * dx32).tolist())
        assert abs(got[r] - exact) <= 1e-12 * abs(exact), (r, got[r], exact)
    ram.row_mass(plan, _t(w.q0, torch.float64), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for r in range(w.n_rows):
        exact = oracle.mass(w.row_nodes(r), w.q0[w.row_slice(r)])
        assert abs(got[r] - exact) <= 1e-13 * abs(exact)


def test_step_scan_is_compensated():
    """The step's own prefix sum (the tiled kernel's block scan, FP32 cells): one row
    of 65536 cells on a log-uniform mesh (width ratio 4), PPM + van Leer with a
    residual (which takes the tiled kernel), a shift of ~300 cells, tiles of 2048
    cells.  Every output mass is a difference of two window prefix sums over up to
    ~2400 cells; with a plain FP32 running sum their rounding (about 2^-24 of the
    prefix, i.e. up to ~1e-4 of a cell's mass) would dominate, while the two-float
    scan leaves the FP32 rounding of the reconstruction and of the output (~1e-7).
    Relative L1 against the FP64 oracle <= 1e-6."""
    n = 65536
    rng = np.random.default_rng(41)
    w = np.exp(rng.uniform(math.log(0.5), math.log(2.0), n))
    x = np.concatenate([[0.0], np.cumsum(w / w.sum())])
    xc = 0.5 * (x[1:] + x[:-1])
    q0 = (1.0 + 0.5 * np.sin(2 * math.pi * 3 * xc) + np.exp(-((xc - 0.4) / 0.05) ** 2))
    q0 = q0.astype(np.float32).astype(np.float64)
    dv = (0.002 * np.sin(2 * math.pi * 5 * x[:-1])).astype(np.float32).astype(np.float64)
    plan = ram.Plan([0, n], x, order=3, limiter=True)
    plan.set_tiling(2048, 512)
    assert plan.info().n_uniform_rows == 0
    dt = 1e-3
    v0 = 300.0 / n / dt
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    ram.step(plan, _t(q0, torch.float32), out, _t([v0], torch.float64), dt,
             dv=_t(dv, torch.float32), scheme=ram.VANLEER)
    torch.cuda.synchronize()
    assert plan.check_errors() == 0
    ref = oracle.step(x, q0, oracle.shift_from_velocity(v0, dt), 3, True, dv, dt,
                      oracle.VANLEER, 1)
    got = out.double().cpu().numpy()
    err = float(np.abs(got - ref).sum() / np.abs(ref).sum())
    assert err <= 1e-6, err


def test_step_conserves_mass_fp64():
    """Eq. 10 on the GPU: the FP64 step conserves every row's mass to round-off."""
    w = wl.batched(n_rows=16, n_max=20000, seed_len=12)
    plan = ram.Plan.from_workload(w)
    q = _t(w.q0, torch.float64)
    out = torch.empty_like(q)
    m0 = torch.empty(w.n_rows, dtype=torch.float64, device=DEV)
    m1 = torch.empty_like(m0)
    ram.row_mass(plan, q, m0)
    ram.step(plan, q, out, _t(w.v0, torch.float64), w.dt)
    ram.row_mass(plan, out, m1)
    torch.cuda.synchronize()
    rel = ((m1 - m0).abs() / m0.abs()).max().item()
    assert rel <= 1e-13, rel


@pytest.mark.parametrize("n", [34, 35, 64, 127, 129, 300, 2049, 5000, 40000])
@pytest.mark.parametrize("order,limiter", [(2, True), (2, False), (3, True), (3, False),
                                           (4, False)])
def test_fp32_warp_segment_rows(n, order, limiter):
    """FP32 rows with their own mesh on the warp-segment kernel: rows from the
    shortest it takes to many tiles, shifts of many periods both ways, shift alone
    and with donor / van Leer residuals of 1..8 sub-steps (the widest halo)."""
    x = wl.random_nodes(n, seed=3 * n + order, ratio=4.0, x0=0.3)
    plan = _use_nseg(ram.Plan([0, n], x, order=order, limiter=limiter))
    assert plan.info().n_nseg_rows == 1
    rng = np.random.default_rng(n + order)
    q0 = _rounded(1.0 + rng.random(n), "float32")
    dxmin = np.diff(x).min()
    dt = 0.1
    qd = _t(q0, torch.float32)
    out = torch.empty_like(qd)
    for s in (0.0, 0.3 * dxmin, 0.4321, 7.77, -3.1415):
        ram.shift(plan, qd, out, _t([s], torch.float64))
        torch.cuda.synchronize()
        ref = oracle.shift(x, q0, s, order, limiter)
        err = np.sum(np.abs(out.double().cpu().numpy() - ref) * np.diff(x)) / np.sum(np.abs(ref) * np.diff(x))
        assert err <= TOL["float32"], ("shift", s, err)
    for scheme, nsub in ((ram.DONOR, 1), (ram.VANLEER, 1), (ram.VANLEER, 8), (ram.DONOR, 5)):
        dv = _rounded((rng.random(n) - 0.5) * 1.6 * nsub * dxmin / dt, "float32")
        v0 = _t([7.3 * (1.0 - x[0]) / dt], torch.float64)
        ram.step(plan, qd, out, v0, dt, dv=_t(dv, torch.float32), scheme=scheme,
                 nsub=_t([nsub], torch.int32))
        torch.cuda.synchronize()
        ref = oracle.step(x, q0, oracle.shift_from_velocity(v0.item(), dt), order, limiter, dv, dt,
                          scheme, nsub)
        err = np.sum(np.abs(out.double().cpu().numpy() - ref) * np.diff(x)) / np.sum(np.abs(ref) * np.diff(x))
        assert err <= TOL["float32"], (scheme, nsub, err)
    assert plan.check_errors() == 0


def test_fp32_warp_segment_full_period_and_zero_shift_bit_exact():
    """Whole periods and a zero shift return the input bit for bit on the FP32
    warp-segment kernel (every shifted edge on its own node: the exact-cover copy)."""
    for n in (34, 600, 3000, 70000):
        x = wl.random_nodes(n, seed=n + 1)
        plan = _use_nseg(ram.Plan([0, n], x, order=3))
        assert plan.info().n_nseg_rows == 1
        q = torch.rand(n, dtype=torch.float32, device=DEV) + 0.5
        out = torch.empty_like(q)
        for m in (0.0, 1.0, 3.0, -2.0):
            ram.shift(plan, q, out, _t([m], torch.float64))
            torch.cuda.synchronize()
            assert torch.equal(out, q), (n, m)


def test_fp32_rows_the_warp_segment_kernel_does_not_take():
    """Rows shorter than its minimum or with a source window above its cap run the
    tiled kernels in the same FP32 step; every row matches the oracle."""
    lens = [5, 33, 34, 2000, 1500]
    ratios = [4.0, 4.0, 4.0, 4.0, 4000.0]
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nodes = np.concatenate([wl.random_nodes(n, seed=40 + r, ratio=ra)
                            for r, (n, ra) in enumerate(zip(lens, ratios))])
    plan = _use_nseg(ram.Plan(ro, nodes, order=3))
    assert plan.info().n_nseg_rows == 2 or plan.info().n_nseg_rows == 3
    rng = np.random.default_rng(41)
    q0 = _rounded(1.0 + rng.random(int(ro[-1])), "float32")
    v0 = rng.uniform(-3, 3, len(lens))
    qd = _t(q0, torch.float32)
    out = torch.empty_like(qd)
    ram.step(plan, qd, out, _t(v0, torch.float64), 1.0)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    for r in range(len(lens)):
        sl = slice(int(ro[r]), int(ro[r + 1]))
        x = nodes[ro[r] + r: ro[r + 1] + r + 1]
        ref = oracle.step(x, q0[sl], oracle.shift_from_velocity(v0[r], 1.0), 3, True)
        err = np.sum(np.abs(got[sl] - ref) * np.diff(x)) / np.sum(np.abs(ref) * np.diff(x))
        assert err <= TOL["float32"], (r, err)
    assert plan.check_errors() == 0
