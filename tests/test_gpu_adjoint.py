"""GPU adjoint of the linear RAM step (limiter off, donor residual) against the FP64
oracle's hand-derived transpose, the dot-product identity, and finite differences
of a checkpointed rollout through torch.autograd; the adjoint of the limited step
linearised at its input (RAM_ADJOINT plans) against the oracle's linearisation."""
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


def _rel(got, ref):
    return float(np.abs(got - ref).sum() / np.abs(ref).sum())


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


def _nonuniform_batch(n_rows=7, seed=30, n_max=3000):
    lens = np.random.default_rng(seed).integers(5, n_max, n_rows)
    lens[0] = 3  # a row shorter than the stencil
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nodes = np.concatenate([wl.random_nodes(int(n), seed=seed + r, ratio=4.0, x0=0.2 * r)
                            for r, n in enumerate(lens)])
    orders = np.array([(2, 3, 4)[r % 3] for r in range(n_rows)], dtype=np.int8)
    return ro, nodes, orders


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("with_dv", [False, True])
def test_adjoint_nonuniform_rows_match_oracle(dtype, with_dv):
    """Rows with their own mesh (orders 2/3/4, one shorter than the stencil), per-row
    shifts of many cells both ways, donor residual with 1-3 sub-steps: g_in and
    dL/d dv against the oracle's transpose."""
    ro, nodes, orders = _nonuniform_batch()
    n_rows = ro.size - 1
    plan = ram.Plan(ro, nodes, order=orders, limiter=False, adjoint=True)
    assert plan.info().n_uniform_rows == 0
    rng = np.random.default_rng(31)
    n = int(ro[-1])
    q = _t(1.0 + rng.random(n), dtype)
    g = _t(rng.standard_normal(n), dtype)
    dt = 0.5
    v0 = rng.uniform(-40, 40, n_rows) / np.diff(ro) / dt
    nsub = np.array([1 + r % 3 for r in range(n_rows)], dtype=np.int32)
    dvh = None
    if with_dv:
        dvh = np.concatenate([
            (rng.random(int(ro[r + 1] - ro[r])) - 0.5) * 1.6 * nsub[r] *
            np.diff(nodes[ro[r] + r: ro[r + 1] + r + 1]).min() / dt for r in range(n_rows)])
    dv = None if dvh is None else _t(dvh, dtype)
    gin = torch.empty_like(q)
    gdv = None if dv is None else torch.zeros_like(dv)
    ram.step_adjoint(plan, q, g, gin, _t(v0, torch.float64), dt, dv=dv, g_dv=gdv,
                     nsub=_t(nsub, torch.int32))
    torch.cuda.synchronize()
    tol = TOL["float64" if dtype == torch.float64 else "float32"]
    gi = gin.double().cpu().numpy()
    qr, gr = q.double().cpu().numpy(), g.double().cpu().numpy()
    dvr = None if dv is None else dv.double().cpu().numpy()
    gd = None if gdv is None else gdv.double().cpu().numpy()
    for r in range(n_rows):
        sl = slice(int(ro[r]), int(ro[r + 1]))
        x = nodes[ro[r] + r: ro[r + 1] + r + 1]
        ref_gi, ref_gd = oracle.step_adjoint(x, qr[sl], gr[sl],
                                             oracle.shift_from_velocity(v0[r], dt), int(orders[r]),
                                             None if dvr is None else dvr[sl], dt, int(nsub[r]))
        e1 = np.abs(gi[sl] - ref_gi).sum() / np.abs(ref_gi).sum()
        assert e1 <= tol, (r, int(orders[r]), e1)
        if gd is not None:
            e2 = np.abs(gd[sl] - ref_gd).sum() / np.abs(ref_gd).sum()
            assert e2 <= tol, (r, e2)
    assert plan.check_errors() == 0


def test_adjoint_nonuniform_dot_product_and_scratch_flag():
    """<J x, y> = <x, J^T y> on rows with their own mesh (FP64); without the
    RAM_ADJOINT flag a step with a residual is refused (no scratch), one without
    a residual is not."""
    ro, nodes, orders = _nonuniform_batch(n_rows=5, seed=40)
    n_rows = ro.size - 1
    rng = np.random.default_rng(41)
    n = int(ro[-1])
    x = _t(rng.standard_normal(n), torch.float64)
    y = _t(rng.standard_normal(n), torch.float64)
    dt = 0.3
    v0 = _t(rng.uniform(-9, 9, n_rows), torch.float64)
    dv = _t(np.concatenate([(rng.random(int(ro[r + 1] - ro[r])) - 0.5) * 0.5 *
                            np.diff(nodes[ro[r] + r: ro[r + 1] + r + 1]).min() / dt
                            for r in range(n_rows)]), torch.float64)
    plan = ram.Plan(ro, nodes, order=orders, limiter=False, adjoint=True)
    jx, jty = torch.empty_like(x), torch.empty_like(y)
    ram.step(plan, x, jx, v0, dt, dv=dv, scheme=ram.DONOR)
    ram.step_adjoint(plan, x, y, jty, v0, dt, dv=dv)
    torch.cuda.synchronize()
    lhs, rhs = float((jx * y).sum()), float((x * jty).sum())
    assert abs(lhs - rhs) <= 1e-13 * float((jx.abs() * y.abs()).sum())
    bare = ram.Plan(ro, nodes, order=orders, limiter=False)
    with pytest.raises(ram.RamError) as e:
        ram.step_adjoint(bare, x, y, jty, v0, dt, dv=dv)
    assert e.value.status == 7
    ram.step_adjoint(bare, x, y, jty, v0, dt)
    torch.cuda.synchronize()


def test_rollout_gradients_nonuniform_finite_differences():
    """Checkpointed rollout on rows with their own mesh (FP64): the autograd gradient
    with respect to Q0 and dv against central differences on random directions."""
    ro, nodes, orders = _nonuniform_batch(n_rows=4, seed=50, n_max=800)
    n_rows = ro.size - 1
    plan = ram.Plan(ro, nodes, order=orders, limiter=False, adjoint=True)
    rng = np.random.default_rng(51)
    n = int(ro[-1])
    dt = 0.2
    v0 = _t(rng.uniform(-20, 20, n_rows), torch.float64)
    q0 = _t(1.0 + rng.random(n), torch.float64).requires_grad_(True)
    dvh = np.concatenate([(0.3 + 0.4 * rng.random(int(ro[r + 1] - ro[r]))) *
                          np.where(rng.random(int(ro[r + 1] - ro[r])) < 0.5, -1, 1) *
                          np.diff(nodes[ro[r] + r: ro[r + 1] + r + 1]).min() / dt
                          for r in range(n_rows)])
    dv = _t(dvh, torch.float64).requires_grad_(True)
    target = _t(1.0 + rng.random(n), torch.float64)
    ns = _t(np.ones(n_rows), torch.int32)

    def f(q, d):
        return ((rollout(plan, q, v0, dt, 12, dv=d, nsub=ns, checkpoint_every=5) - target) ** 2).sum()

    loss = f(q0, dv)
    gq, gdv = torch.autograd.grad(loss, (q0, dv))
    with torch.no_grad():
        for d in range(6):
            eq = _t(rng.standard_normal(n), torch.float64)
            ev = _t(rng.standard_normal(n), torch.float64) * dv.abs().mean() * 1e-3
            h = 1e-5
            fd = (float(f(q0 + h * eq, dv + h * ev)) - float(f(q0 - h * eq, dv - h * ev))) / (2 * h)
            an = float((gq * eq).sum() + (gdv * ev).sum())
            assert fd == pytest.approx(an, rel=1e-6, abs=1e-9 * abs(float(loss))), d


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("uniform", [True, False])
def test_limited_adjoint_matches_the_oracle_linearisation(dtype, order, uniform):
    """RAM_ADJOINT plans with the limiter on: the transpose of the step linearised at
    its input (limited PLM / PPM, donor residual) against the oracle's, on uniform
    rows (a disk) and on rows with their own mesh."""
    lens = [40, 200, 7, 300] if not uniform else [256] * 4
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    if uniform:
        nodes = wl.uniform_nodes(256, 0.0, 2 * np.pi)
        plan = ram.Plan(ro, nodes, order=order, limiter=True, shared_mesh=True, adjoint=True)
        xs = [nodes] * 4
    else:
        xs = [wl.random_nodes(n, seed=60 + r, ratio=3.0) for r, n in enumerate(lens)]
        nodes = np.concatenate(xs)
        plan = ram.Plan(ro, nodes, order=order, limiter=True, adjoint=True)
    rng = np.random.default_rng(61 + order)
    n = int(ro[-1])
    # smooth rows with a few extrema each: the limiters act, away from ties
    qh = np.concatenate([1.5 + 0.4 * wl.sine_averages(x, k=2 + r, phase=0.7 * r, period=x[-1] - x[0])
                         + 0.2 * wl.sine_averages(x, k=5, phase=1.3 + r, period=x[-1] - x[0])
                         for r, x in enumerate(xs)])
    q = _t(qh, dtype)
    g = _t(rng.standard_normal(n), dtype)
    dt = 0.4
    v0 = rng.uniform(-30, 30, 4) * np.array([x[-1] - x[0] for x in xs]) / np.array(lens) / dt
    nsub = np.array([1, 2, 1, 3], dtype=np.int32)
    dvh = np.concatenate([(rng.random(lens[r]) - 0.5) * 1.6 * nsub[r] * np.diff(xs[r]).min() / dt
                          for r in range(4)])
    dv = _t(dvh, dtype)
    gin = torch.empty_like(q)
    gdv = torch.zeros_like(dv)
    ram.step_adjoint(plan, q, g, gin, _t(v0, torch.float64), dt, dv=dv, g_dv=gdv,
                     nsub=_t(nsub, torch.int32))
    torch.cuda.synchronize()
    tol = TOL["float64" if dtype == torch.float64 else "float32"]
    gi, gd = gin.double().cpu().numpy(), gdv.double().cpu().numpy()
    qr, gr, dvr = q.double().cpu().numpy(), g.double().cpu().numpy(), dv.double().cpu().numpy()
    alike = np.ones(n, dtype=bool)
    if dtype == torch.float32:
        # A limiter branch near a tie may be decided differently by FP32 and FP64
        # arithmetic; there both one-sided linearisations are valid.  Compare the
        # cells where the FP32 kernel decided as its FP64 run did (the same inputs),
        # and require nearly all of them to be such cells.
        g64 = torch.empty(n, dtype=torch.float64, device=DEV)
        ram.step_adjoint(plan, q.double(), g.double(), g64, _t(v0, torch.float64), dt,
                         dv=dv.double(), nsub=_t(nsub, torch.int32))
        torch.cuda.synchronize()
        g64 = g64.cpu().numpy()
        alike = np.abs(gi - g64) <= 1e-3 * np.abs(g64).max()
        assert alike.mean() >= 0.97, alike.mean()
    for r in range(4):
        sl = slice(int(ro[r]), int(ro[r + 1]))
        ref_gi, ref_gd = oracle.step_adjoint_limited(
            xs[r], qr[sl], gr[sl], oracle.shift_from_velocity(v0[r], dt), order, True, dvr[sl], dt,
            int(nsub[r]))
        m = alike[sl]
        e1 = np.abs(gi[sl] - ref_gi)[m].sum() / np.abs(ref_gi)[m].sum()
        assert e1 <= tol, (r, e1)
        if dtype == torch.float64:
            e2 = np.abs(gd[sl] - ref_gd).sum() / np.abs(ref_gd).sum()
            assert e2 <= tol, (r, e2)
    assert plan.check_errors() == 0


def test_limited_adjoint_refusals():
    n = 128
    x = wl.uniform_nodes(n)
    q = _t(np.ones(n), torch.float64)
    v0 = _t([1.0], torch.float64)
    for plan in (ram.Plan([0, n], x, order=3, limiter=True),            # no RAM_ADJOINT
                 ram.Plan([0, n], x, order=4, limiter=True, adjoint=True)):  # limited order 4
        with pytest.raises(ram.RamError) as e:
            ram.step_adjoint(plan, q, q.clone(), torch.empty_like(q), v0, 0.1)
        assert e.value.status == 7


@pytest.mark.parametrize("order", [2, 3])
def test_limited_rollout_gradients(order):
    """A checkpointed rollout of the limited step (FP64): the autograd gradient with
    respect to Q0 and dv against the oracle's chain of step linearisations (its own
    forward states, its transposes), element by element; for PLM also against
    central differences.  The limited PPM step is piecewise smooth with many
    branches: after a few steps some branch boundary comes within 1e-8 of the
    state, so a central difference of any practical step straddles a kink (the
    oracle's own differences do the same there)."""
    w = wl.disk(n_r=8, n_phi=256, order=order, limiter=True, scheme=0, seed_dv=9, ref_n_phi=4096)
    plan = ram.Plan.from_workload(w, adjoint=True)
    rng = np.random.default_rng(70)
    # rings with structure of their own (the disk's rings are flat far from the
    # vortex, where every limiter sits on its kink); phases off the grid's symmetry,
    # so that no two neighbouring differences tie (the nearest tie is ~1e-6 away,
    # far beyond the 1e-8 steps below)
    x = w.nodes
    w.q0 = np.concatenate([w.q0[w.row_slice(r)] * (1.0 + 0.3 * wl.sine_averages(
        x, k=2 + r % 3, phase=0.37 + 0.9 * r, period=x[-1] - x[0])) for r in range(w.n_rows)])
    v0 = _t(w.v0, torch.float64)
    ns = _t(w.nsub, torch.int32)
    th = w.q0 * (1.0 + 0.05 * rng.standard_normal(w.n_cells))
    target = _t(th, torch.float64)
    steps = 9

    def f(q0, dv):
        return ((rollout(plan, q0, v0, w.dt, steps, dv=dv, nsub=ns, checkpoint_every=4) - target) ** 2).sum()

    q0 = _t(w.q0, torch.float64).requires_grad_(True)
    dv = _t(w.dv, torch.float64).requires_grad_(True)
    loss = f(q0, dv)
    gq, gdv = torch.autograd.grad(loss, (q0, dv))
    assert plan.check_errors() == 0

    # the oracle: forward states, then the transposed linearised steps in reverse
    states = [w.q0]
    for _ in range(steps):
        states.append(np.concatenate([
            oracle.step(x, states[-1][w.row_slice(r)], oracle.shift_from_velocity(w.v0[r], w.dt),
                        order, True, w.dv[w.row_slice(r)], w.dt, 0, int(w.nsub[r]))
            for r in range(w.n_rows)]))
    g = 2.0 * (states[-1] - th)
    ref_gdv = np.zeros(w.n_cells)
    for i in reversed(range(steps)):
        gi = np.empty_like(g)
        for r in range(w.n_rows):
            sl = w.row_slice(r)
            gi[sl], gd = oracle.step_adjoint_limited(
                x, states[i][sl], g[sl], oracle.shift_from_velocity(w.v0[r], w.dt), order, True,
                w.dv[sl], w.dt, int(w.nsub[r]))
            ref_gdv[sl] += gd
        g = gi
    assert _rel(gq.cpu().numpy(), g) <= TOL["float64"]
    assert _rel(gdv.cpu().numpy(), ref_gdv) <= TOL["float64"]
    if order != 2:
        return
    with torch.no_grad():
        for d in range(6):
            eq = _t(rng.standard_normal(w.n_cells), torch.float64)
            ev = _t(rng.standard_normal(w.n_cells), torch.float64) * dv.abs().mean() * 1e-3
            h = 1e-8
            fd = (float(f(q0 + h * eq, dv + h * ev)) - float(f(q0 - h * eq, dv - h * ev))) / (2 * h)
            an = float((gq * eq).sum() + (gdv * ev).sum())
            assert fd == pytest.approx(an, rel=1e-5, abs=1e-8 * abs(float(loss))), d
