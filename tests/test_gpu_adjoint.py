"""GPU adjoint of the linear RAM step (limiter off, donor residual) against the FP64
oracle's hand-derived transpose, the dot-product identity, and finite differences
of a checkpointed rollout through torch.autograd."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2305_05362_gb300 import ram, workloads as wl
from paper_2305_05362_gb300.autograd import rollout
from gpu_common import TOL

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def _disk(n_r, n_phi, order, seed=4):
    return wl.disk(n_r=n_r, n_phi=n_phi, order=order, limiter=False, scheme=0, seed_dv=seed,
                   ref_n_phi=4096)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("order", [2, 3, 4])
def test_adjoint_matches_oracle(dtype, order):
    w = _disk(6, 1024, order)
    plan = ram.Plan.from_workload(w)
    rng = np.random.default_rng(order)
    q = _t(w.q0, dtype)
    g = _t(rng.standard_normal(w.n_cells), dtype)
    dv = _t(w.dv, dtype)
    gin = torch.empty_like(q)
    gdv = torch.zeros_like(dv)
    v0 = _t(w.v0, torch.float64)
    ns = _t(w.nsub, torch.int32)
    ram.step_adjoint(plan, q, g, gin, v0, w.dt, dv=dv, g_dv=gdv, nsub=ns)
    torch.cuda.synchronize()
    gi, gd = gin.double().cpu().numpy(), gdv.double().cpu().numpy()
    qr, gr, dvr = q.double().cpu().numpy(), g.double().cpu().numpy(), dv.double().cpu().numpy()
    tol = TOL["float64" if dtype == torch.float64 else "float32"]
    for r in range(w.n_rows):
        sl = w.row_slice(r)
        ref_gi, ref_gd = oracle.step_adjoint(w.nodes, qr[sl], gr[sl],
                                             oracle.shift_from_velocity(w.v0[r], w.dt), order,
                                             dvr[sl], w.dt, int(w.nsub[r]))
        e1 = np.abs(gi[sl] - ref_gi).sum() / np.abs(ref_gi).sum()
        e2 = np.abs(gd[sl] - ref_gd).sum() / np.abs(ref_gd).sum()
        assert e1 <= tol and e2 <= tol, (r, e1, e2)
    assert plan.check_errors() == 0


def test_dot_product_identity():
    """<J x, y> = <x, J^T y> for the full step (shift + donor residual), FP64."""
    w = _disk(8, 2048, 3)
    plan = ram.Plan.from_workload(w)
    rng = np.random.default_rng(3)
    x = _t(rng.standard_normal(w.n_cells), torch.float64)
    y = _t(rng.standard_normal(w.n_cells), torch.float64)
    dv = _t(w.dv, torch.float64)
    v0 = _t(w.v0, torch.float64)
    ns = _t(w.nsub, torch.int32)
    jx = torch.empty_like(x)
    jty = torch.empty_like(y)
    ram.step(plan, x, jx, v0, w.dt, dv=dv, scheme=ram.DONOR, nsub=ns)
    ram.step_adjoint(plan, x, y, jty, v0, w.dt, dv=dv, nsub=ns)
    torch.cuda.synchronize()
    lhs, rhs = float((jx * y).sum()), float((x * jty).sum())
    assert abs(lhs - rhs) <= 1e-13 * float((jx.abs() * y.abs()).sum())


def test_limited_plan_is_refused():
    w = wl.disk(n_r=2, n_phi=512)
    plan = ram.Plan.from_workload(w)  # limiter on
    q = _t(w.q0, torch.float64)
    with pytest.raises(ram.RamError) as e:
        ram.step_adjoint(plan, q, q.clone(), torch.empty_like(q), _t(w.v0, torch.float64), w.dt)
    assert e.value.status == 7


def _loss_fn(plan, v0, dt, steps, nsub, target, k):
    def f(q0, dv):
        qt = rollout(plan, q0, v0, dt, steps, dv=dv, nsub=nsub, checkpoint_every=k)
        return ((qt - target) ** 2).sum()
    return f


@pytest.mark.parametrize("n_r,n_phi,steps,k", [(16, 512, 30, 7), (512, 2048, 200, 20)])
def test_rollout_gradients_finite_differences(n_r, n_phi, steps, k):
    """Disk rollout with checkpoints every k steps; loss = sum (Sigma_T - target)^2 with
    target = Sigma_0 (1 + 0.05 N(0,1)).  The autograd gradient with respect to Q0 and
    dv matches central finite differences along random directions (FP64) and the
    FP32 gradient matches the FP64 one."""
    w = _disk(n_r, n_phi, 3, seed=4)
    plan = ram.Plan.from_workload(w)
    rng = np.random.default_rng(5)
    target = _t(w.q0 * (1.0 + 0.05 * rng.standard_normal(w.n_cells)), torch.float64)
    v0 = _t(w.v0, torch.float64)
    ns = _t(w.nsub, torch.int32)
    f = _loss_fn(plan, v0, w.dt, steps, ns, target, k)
    q0 = _t(w.q0, torch.float64).requires_grad_(True)
    dv = _t(w.dv, torch.float64).requires_grad_(True)
    loss = f(q0, dv)
    gq, gdv = torch.autograd.grad(loss, (q0, dv))
    rd = np.random.default_rng(8)
    n_dir = 8 if n_r < 100 else 64
    with torch.no_grad():
        for d in range(n_dir):
            eq = _t(rd.standard_normal(w.n_cells), torch.float64)
            ev = _t(rd.standard_normal(w.n_cells), torch.float64) * dv.abs().mean()
            # dv directions small enough that no upwind side flips
            h = 1e-4
            lp = float(f(q0 + h * eq, dv + h * 1e-3 * ev))
            lm = float(f(q0 - h * eq, dv - h * 1e-3 * ev))
            fd = (lp - lm) / (2 * h)
            an = float((gq * eq).sum() + 1e-3 * (gdv * ev).sum())
            assert fd == pytest.approx(an, rel=1e-6, abs=1e-9 * abs(float(loss))), d
    # FP32 forward and adjoint against the FP64 gradient
    q32 = _t(w.q0, torch.float32).requires_grad_(True)
    dv32 = _t(w.dv, torch.float32).requires_grad_(True)
    qt32 = rollout(plan, q32, v0, w.dt, steps, dv=dv32, nsub=ns, checkpoint_every=k)
    loss32 = ((qt32 - target.float()) ** 2).sum()
    g32q, g32dv = torch.autograd.grad(loss32, (q32, dv32))
    rel_q = float((g32q.double() - gq).abs().sum() / gq.abs().sum())
    assert rel_q <= 1e-3, rel_q
