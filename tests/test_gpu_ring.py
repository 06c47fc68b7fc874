"""The FP32 warp-segment kernel with shared-memory rings (tuning variant 2), which
forms each row's shift parameters itself in two-float arithmetic, so that no
parameter kernel runs before it when every row of the plan takes it.  Checked
against the FP64 oracle (FP32 tolerance) in every mode: shift, residual alone and
the full step, with the phase, the error flags, shifts of many periods, and plans
or arrays that need the parameter kernel after all."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2305_05362_gb300 import ram, workloads as wl
from gpu_common import TOL, oracle_shifts, oracle_step, rel_l1_rows

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def _ring(plan, warps=4):
    t = plan.tuning()
    t.uniform_kernel_f32 = 1
    t.seg_variant_f32 = 2
    t.seg_warps = warps
    plan.set_tuning(t)
    return plan


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("warps", [3, 4, 6, 8])
def test_step_matches_oracle(warps):
    w = wl.disk(n_r=24, n_phi=2048)
    plan = _ring(ram.Plan.from_workload(w), warps)
    q0, dv = _f32(w.q0), _f32(w.dv)
    out = torch.empty(w.n_cells, dtype=torch.float32, device=DEV)
    ram.step(plan, _t(q0, torch.float32), out, _t(w.v0, torch.float64), w.dt,
             dv=_t(dv, torch.float32), scheme=w.scheme, nsub=_t(w.nsub, torch.int32))
    torch.cuda.synchronize()
    ref = oracle_step(w, q0, oracle_shifts(w), dv=dv, nsub=w.nsub)
    assert rel_l1_rows(w, out.double().cpu().numpy(), ref) <= TOL["float32"]
    assert plan.check_errors() == 0


def test_shifts_of_many_periods_and_both_signs():
    """ram_shift with shifts from -1e4 to +1e4 periods, just below and above whole
    cells, and exactly zero."""
    n_r, n = 12, 1024
    x = wl.uniform_nodes(n, 0.0, 2 * np.pi)
    rng = np.random.default_rng(3)
    q0 = _f32(1.0 + rng.random(n_r * n))
    L, dx = 2 * np.pi, 2 * np.pi / n
    sh = np.array([0.0, 0.37 * dx, -0.37 * dx, 5 * dx - 1e-9, 5 * dx + 1e-9, -1e4 * L + 0.3 * dx,
                   1e4 * L - 0.7 * dx, 123.456, -98.765, 17 * L, 3.5 * dx, -1e-12])
    plan = _ring(ram.Plan(np.arange(n_r + 1, dtype=np.int64) * n, x, order=3, shared_mesh=True))
    out = torch.empty(n_r * n, dtype=torch.float32, device=DEV)
    ram.shift(plan, _t(q0, torch.float32), out, _t(sh, torch.float64))
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    for r in range(n_r):
        sl = slice(r * n, (r + 1) * n)
        ref = oracle.shift(x, q0[sl], sh[r], 3, True)
        err = np.sum(np.abs(got[sl] - ref)) / np.sum(np.abs(ref))
        # a shift of 1e4 periods carries ~1e4 L 2^-52 of FP64 round-off in the
        # oracle itself; the two-float shift is as close
        assert err <= TOL["float32"], (r, sh[r], err)
    assert plan.check_errors() == 0


def test_residual_alone_and_orders():
    w = wl.disk(n_r=9, n_phi=1536)
    for order in (2, 3, 4):
        plan = _ring(ram.Plan(w.row_offset, w.nodes, order=order, shared_mesh=True))
        q0, dv = _f32(w.q0), _f32(w.dv)
        out = torch.empty(w.n_cells, dtype=torch.float32, device=DEV)
        ram.residual_upwind(plan, _t(q0, torch.float32), out, _t(dv, torch.float32), w.dt,
                            ram.VANLEER, _t(w.nsub, torch.int32))
        torch.cuda.synchronize()
        ref = np.concatenate([oracle.residual(w.nodes, q0[w.row_slice(r)], dv[w.row_slice(r)],
                                              w.dt, oracle.VANLEER, int(w.nsub[r]))
                              for r in range(w.n_rows)])
        assert rel_l1_rows(w, out.double().cpu().numpy(), ref) <= TOL["float32"], order
        v0 = _t(w.v0, torch.float64)
        ram.step(plan, _t(q0, torch.float32), out, v0, w.dt, dv=_t(dv, torch.float32),
                 scheme=ram.DONOR, nsub=_t(w.nsub, torch.int32))
        torch.cuda.synchronize()
        ref = np.concatenate([oracle.step(w.nodes, q0[w.row_slice(r)],
                                          oracle.shift_from_velocity(w.v0[r], w.dt), order,
                                          True, dv[w.row_slice(r)], w.dt, oracle.DONOR,
                                          int(w.nsub[r]))
                              for r in range(w.n_rows)])
        assert rel_l1_rows(w, out.double().cpu().numpy(), ref) <= TOL["float32"], order
        assert plan.check_errors() == 0


def test_phase_advanced_once_per_step():
    """With no parameter kernel the ring kernel advances the phase (FP64)."""
    w = wl.disk(n_r=5, n_phi=1024)
    plan = _ring(ram.Plan.from_workload(w))
    q = _t(w.q0, torch.float32)
    out = torch.empty_like(q)
    phase = torch.zeros(w.n_rows, dtype=torch.float64, device=DEV)
    ref = np.zeros(w.n_rows)
    v0 = _t(w.v0, torch.float64)
    for _ in range(7):
        ram.step(plan, q, out, v0, w.dt, phase=phase)
        ref = np.array([oracle.phase_update(ref[r], w.v0[r], w.dt, w.period(r))
                        for r in range(w.n_rows)])
    torch.cuda.synchronize()
    np.testing.assert_allclose(phase.cpu().numpy(), ref, rtol=0, atol=1e-13)


def test_mixed_plan_runs_the_parameter_kernel_once():
    """Rows too short for the warp segments go to the tiled kernel, so the
    parameter kernel runs; the ring rows form their own parameters and leave the
    phase to it (advanced once per step, not twice)."""
    lens = [2048, 100, 1024]
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nodes = np.concatenate([wl.uniform_nodes(n, 0.0, 1.0) for n in lens])
    rng = np.random.default_rng(8)
    q0 = _f32(1.0 + rng.random(int(ro[-1])))
    v0 = np.array([3.3, -7.1, 0.45])
    dt = 0.01
    plan = _ring(ram.Plan(ro, nodes, order=3))
    q = _t(q0, torch.float32)
    out = torch.empty_like(q)
    phase = torch.zeros(3, dtype=torch.float64, device=DEV)
    ram.step(plan, q, out, _t(v0, torch.float64), dt, phase=phase)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    for r, n in enumerate(lens):
        sl = slice(int(ro[r]), int(ro[r + 1]))
        x = nodes[ro[r] + r: ro[r + 1] + r + 1]
        ref = oracle.shift(x, q0[sl], oracle.shift_from_velocity(v0[r], dt), 3, True)
        err = np.sum(np.abs(got[sl] - ref)) / np.sum(np.abs(ref))
        assert err <= TOL["float32"], (n, err)
    ref_phase = [oracle.phase_update(0.0, v0[r], dt, 1.0) for r in range(3)]
    np.testing.assert_allclose(phase.cpu().numpy(), ref_phase, rtol=0, atol=1e-13)
    assert plan.check_errors() == 0


def test_error_flags():
    w = wl.disk(n_r=4, n_phi=1024)
    plan = _ring(ram.Plan.from_workload(w))
    q = _t(w.q0, torch.float32)
    out = torch.empty_like(q)
    dvd = _t(w.dv, torch.float32)
    v0 = w.v0.copy()
    v0[2] = math.nan
    ram.step(plan, q, out, _t(v0, torch.float64), w.dt, dv=dvd, nsub=_t(w.nsub, torch.int32))
    assert plan.check_errors() == 8  # non-finite shift
    ns = w.nsub.copy()
    ns[1] = 99
    ram.step(plan, q, out, _t(w.v0, torch.float64), w.dt, dv=dvd, nsub=_t(ns, torch.int32))
    assert plan.check_errors() == 1  # sub-step count out of range
    ram.step(plan, q, out, _t(w.v0, torch.float64), w.dt, dv=dvd * 50.0,
             nsub=_t(w.nsub, torch.int32))
    assert plan.check_errors() == 3  # CFL above 1
    assert plan.check_errors() == 0


def test_misaligned_arrays_fall_back_to_the_parameter_kernel():
    w = wl.disk(n_r=4, n_phi=1024)
    plan = _ring(ram.Plan.from_workload(w))
    base = torch.zeros(w.n_cells + 1, dtype=torch.float32, device=DEV)
    qa = base[1:]
    qa.copy_(_t(w.q0, torch.float32))
    qb = _t(w.q0, torch.float32)
    dvd = _t(w.dv, torch.float32)
    v0 = _t(w.v0, torch.float64)
    ns = _t(w.nsub, torch.int32)
    oa, ob = torch.empty_like(qb), torch.empty_like(qb)
    ram.step(plan, qa, oa, v0, w.dt, dv=dvd, scheme=ram.VANLEER, nsub=ns)
    ram.step(plan, qb, ob, v0, w.dt, dv=dvd, scheme=ram.VANLEER, nsub=ns)
    torch.cuda.synchronize()
    err = float((oa.double() - ob.double()).abs().sum() / ob.double().abs().sum())
    assert err <= 1e-6
    assert plan.check_errors() == 0
