"""GPU parity of the streaming-warp kernel (FP32 uniform rows) against the FP64
oracle through the C ABI: per-row relative L1 <= 1e-5 (the FP32 bar), over the
orders, limiters, schemes, sub-step counts, row lengths that leave ragged last
segments, shift-only and residual-only launches, and whole-cell shifts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2305_05362_gb300 import ram, workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL32 = 1e-5


def _t(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def _stream_plan(lens, order, limiter, v):
    """Uniform rows of the given lengths (period 1 each) on their own meshes."""
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nodes = np.concatenate([wl.uniform_nodes(n) for n in lens])
    plan = ram.Plan(ro, nodes, order=order, limiter=limiter)
    t = plan.tuning()
    t.uniform_kernel_f32 = 2
    t.stream_cells_per_lane_f32 = v
    plan.set_tuning(t)
    return plan, ro, nodes


def _rows(ro, nodes, got, refs):
    errs = []
    for r in range(len(ro) - 1):
        sl = slice(int(ro[r]), int(ro[r + 1]))
        errs.append(np.sum(np.abs(got[sl] - refs[r])) / np.sum(np.abs(refs[r])))
    return max(errs)


@pytest.mark.parametrize("v", [4, 8])
@pytest.mark.parametrize("order,limiter", [(3, True), (3, False), (2, True), (2, False),
                                           (4, False)])
@pytest.mark.parametrize("scheme", [ram.VANLEER, ram.DONOR])
def test_stream_step_matches_oracle(v, order, limiter, scheme):
    """Rows of 512 .. 4100 cells (ragged last segments, rows shorter than the
    longest: empty segment slots), shifts of many cells both ways, nsub 1..8."""
    lens = [520, 1000, 4096, 4100, 2052, 768]
    plan, ro, nodes = _stream_plan(lens, order, limiter, v)
    rng = np.random.default_rng(order * 10 + v + scheme)
    n_tot = int(ro[-1])
    q0 = (1.0 + rng.random(n_tot)).astype(np.float32).astype(np.float64)
    dt = 0.25
    nsub = np.array([1, 2, 3, 8, 5, 1], dtype=np.int32)
    dv = np.concatenate([(rng.random(n) - 0.5) * 1.6 / n / dt * nsub[r] / 8
                         for r, n in enumerate(lens)])
    dv = dv.astype(np.float32).astype(np.float64)
    v0 = rng.uniform(-300.0, 300.0, len(lens)) / 1000.0 / dt
    out = torch.empty(n_tot, dtype=torch.float32, device=DEV)
    ram.step(plan, _t(q0, torch.float32), out, _t(v0, torch.float64), dt,
             dv=_t(dv, torch.float32), scheme=scheme, nsub=_t(nsub, torch.int32))
    torch.cuda.synchronize()
    refs = []
    for r, n in enumerate(lens):
        sl = slice(int(ro[r]), int(ro[r + 1]))
        x = nodes[ro[r] + r: ro[r + 1] + r + 1]
        refs.append(oracle.step(x, q0[sl], oracle.shift_from_velocity(v0[r], dt), order, limiter,
                                dv[sl], dt, scheme, int(nsub[r])))
    assert _rows(ro, nodes, out.double().cpu().numpy(), refs) <= TOL32
    assert plan.check_errors() == 0


@pytest.mark.parametrize("v", [4, 8])
def test_stream_shift_only_and_residual_only(v):
    lens = [4096, 524]
    plan, ro, nodes = _stream_plan(lens, 3, True, v)
    rng = np.random.default_rng(5)
    q0 = (1.0 + rng.random(int(ro[-1]))).astype(np.float32).astype(np.float64)
    qd = _t(q0, torch.float32)
    out = torch.empty_like(qd)
    shifts = np.array([0.3337, -2.71])
    ram.shift(plan, qd, out, _t(shifts, torch.float64))
    torch.cuda.synchronize()
    refs = [oracle.shift(nodes[ro[r] + r: ro[r + 1] + r + 1], q0[int(ro[r]):int(ro[r + 1])],
                         shifts[r], 3, True) for r in range(2)]
    assert _rows(ro, nodes, out.double().cpu().numpy(), refs) <= TOL32
    dt = 0.5
    dv = np.concatenate([(rng.random(n) - 0.5) * 0.8 / n / dt for n in lens])
    dv = dv.astype(np.float32).astype(np.float64)
    ram.residual_upwind(plan, qd, out, _t(dv, torch.float32), dt, ram.VANLEER, None)
    torch.cuda.synchronize()
    refs = [oracle.residual(nodes[ro[r] + r: ro[r + 1] + r + 1], q0[int(ro[r]):int(ro[r + 1])],
                            dv[int(ro[r]):int(ro[r + 1])], dt, oracle.VANLEER, 1)
            for r in range(2)]
    assert _rows(ro, nodes, out.double().cpu().numpy(), refs) <= TOL32
    assert plan.check_errors() == 0


@pytest.mark.parametrize("v", [4, 8])
def test_stream_whole_cell_shift_is_exact(v):
    """A shift by a whole number of cells (no residual) moves the row bit for bit."""
    n = 4096
    plan, ro, nodes = _stream_plan([n], 3, True, v)
    q = torch.rand(n, dtype=torch.float32, device=DEV) + 0.5
    out = torch.empty_like(q)
    for k in (0, 1, 3, 4093, -5):
        ram.shift(plan, q, out, _t([k / n], torch.float64))
        torch.cuda.synchronize()
        assert torch.equal(out, torch.roll(q, k)), k


def test_stream_disk_matches_other_kernels():
    """The benchmark disk recipe (reduced to 64 rings): the streaming kernel agrees
    with the persistent whole-row kernel to FP32 round-off, and with the oracle."""
    w = wl.disk(n_r=64, n_phi=4096, dtype=np.float32)
    plan = ram.Plan.from_workload(w)
    q = _t(w.q0, torch.float32)
    dvd = _t(w.dv, torch.float32)
    v0 = _t(w.v0, torch.float64)
    ns = _t(w.nsub, torch.int32)
    outs = {}
    for kern, sv in ((0, 8), (2, 4), (2, 8)):
        t = plan.tuning()
        t.uniform_kernel_f32 = kern
        t.stream_cells_per_lane_f32 = sv
        plan.set_tuning(t)
        o = torch.empty_like(q)
        ram.step(plan, q, o, v0, w.dt, dv=dvd, scheme=w.scheme, nsub=ns)
        outs[(kern, sv)] = o
    torch.cuda.synchronize()
    base = outs[(0, 8)].double()
    for key, o in outs.items():
        rel = float((o.double() - base).abs().sum() / base.abs().sum())
        assert rel <= 2e-6, (key, rel)
    got = outs[(2, 4)].double().cpu().numpy()
    q0 = q.double().cpu().numpy()
    dvr = dvd.double().cpu().numpy()
    for r in range(0, 64, 9):
        sl = w.row_slice(r)
        ref = oracle.step(w.row_nodes(r), q0[sl], oracle.shift_from_velocity(w.v0[r], w.dt),
                          3, True, dvr[sl], w.dt, w.scheme, int(w.nsub[r]))
        assert np.sum(np.abs(got[sl] - ref)) / np.sum(np.abs(ref)) <= TOL32
    assert plan.check_errors() == 0


def test_stream_short_rows_fall_back_to_narrow_pairs():
    """Rows of 512 cells are shorter than the 8-cells-per-lane window: the plan
    still runs them (4 cells per lane) and matches the oracle."""
    lens = [512, 512, 516]
    plan, ro, nodes = _stream_plan(lens, 3, True, 8)
    rng = np.random.default_rng(8)
    q0 = (1.0 + rng.random(int(ro[-1]))).astype(np.float32).astype(np.float64)
    dt = 0.5
    dv = np.concatenate([(rng.random(n) - 0.5) * 0.8 / n / dt for n in lens])
    dv = dv.astype(np.float32).astype(np.float64)
    v0 = np.array([0.123, -7.77, 3.3]) / dt
    out = torch.empty(int(ro[-1]), dtype=torch.float32, device=DEV)
    ram.step(plan, _t(q0, torch.float32), out, _t(v0, torch.float64), dt,
             dv=_t(dv, torch.float32), scheme=ram.VANLEER)
    torch.cuda.synchronize()
    refs = []
    for r, n in enumerate(lens):
        sl = slice(int(ro[r]), int(ro[r + 1]))
        x = nodes[ro[r] + r: ro[r + 1] + r + 1]
        refs.append(oracle.step(x, q0[sl], oracle.shift_from_velocity(v0[r], dt), 3, True,
                                dv[sl], dt, ram.VANLEER, 1))
    assert _rows(ro, nodes, out.double().cpu().numpy(), refs) <= TOL32
    assert plan.check_errors() == 0
