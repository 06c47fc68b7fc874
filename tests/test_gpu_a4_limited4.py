"""GPU parity, through the C ABI, of the fourth-order cell-average correction of
Sec. 3.1 (RAM_A4 plans: point values in and out, PPM on the corrected averages) and
of the limited order 4 (the quartic cumulative scaled toward the cell mean within
the range of the cell and its neighbours) against the FP64 oracle: relative L1
<= 1e-12 (FP64), <= 1e-5 (FP32)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2305_05362_gb300 import ram, workloads as wl
from gpu_common import TOL

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
DT = {"float64": torch.float64, "float32": torch.float32}


def _t(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def _rounded(a, dtype):
    a = np.asarray(a, dtype=np.float64)
    return a.astype(np.float32).astype(np.float64) if dtype == "float32" else a


def _rel(got, ref, w=None):
    w = np.ones(len(ref)) if w is None else w
    return float(np.sum(np.abs(got - ref) * w) / np.sum(np.abs(ref) * w))


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("limiter", [True, False])
@pytest.mark.parametrize("scheme", [ram.DONOR, ram.VANLEER])
def test_a4_step_matches_oracle(dtype, limiter, scheme):
    """Uniform rows of 7 .. 4100 cells (the short ones take the exact periodic
    inverse), per-row shifts of many cells both ways and residual sub-steps."""
    lens = [7, 24, 25, 600, 4096, 4100]
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nodes = np.concatenate([wl.uniform_nodes(n, -0.5, 1.0 + 0.25 * r) for r, n in enumerate(lens)])
    plan = ram.Plan(ro, nodes, order=3, limiter=limiter, a4=True)
    rng = np.random.default_rng(11)
    q0 = _rounded(1.0 + rng.random(int(ro[-1])), dtype)
    dt = 0.05
    v0 = rng.uniform(-60, 60, len(lens)) * (1.0 + 0.25 * np.arange(len(lens))) / np.array(lens) / dt
    nsub = np.array([1 + r % 3 for r in range(len(lens))], dtype=np.int32)
    dv = np.concatenate([(rng.random(n) - 0.5) * 1.6 * nsub[r] * (1.0 + 0.25 * r) / n / dt
                         for r, n in enumerate(lens)])
    dv = _rounded(dv, dtype)
    qd = _t(q0, DT[dtype])
    out = torch.empty_like(qd)
    for with_dv in (False, True):
        ram.step(plan, qd, out, _t(v0, torch.float64), dt,
                 dv=_t(dv, DT[dtype]) if with_dv else None, scheme=scheme,
                 nsub=_t(nsub, torch.int32))
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        for r, n in enumerate(lens):
            sl = slice(int(ro[r]), int(ro[r + 1]))
            x = nodes[ro[r] + r: ro[r + 1] + r + 1]
            ref = oracle.step_a4(x, q0[sl], oracle.shift_from_velocity(v0[r], dt), limiter,
                                 dv[sl] if with_dv else None, dt, scheme, int(nsub[r]))
            assert _rel(got[sl], ref) <= TOL[dtype], (with_dv, r, _rel(got[sl], ref))
    assert plan.check_errors() == 0


def test_a4_shift_conserves_and_rolls():
    """FP64: the corrected step conserves sum Q dx (Eq. 10 on a periodic uniform mesh)
    and a whole-cell shift is a roll (to round-off: the inverse is a solve)."""
    n = 1024
    x = wl.uniform_nodes(n)
    plan = ram.Plan([0, n], x, order=3, limiter=True, a4=True)
    q = _t(wl.three_gaussians(x, 5), torch.float64)
    out = torch.empty_like(q)
    ram.shift(plan, q, out, _t([0.3123], torch.float64))
    torch.cuda.synchronize()
    assert abs(float(out.sum()) - float(q.sum())) <= 1e-13 * float(q.sum())
    ram.shift(plan, q, out, _t([37.0 / n], torch.float64))
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), np.roll(q.cpu().numpy(), 37), rtol=0,
                               atol=1e-13)


def test_a4_refused_off_its_domain():
    """The correction is the uniform-mesh formula on the PPM remap: other orders or
    rows with their own mesh are refused at planning."""
    with pytest.raises(ram.RamError) as e:
        ram.Plan([0, 64], wl.uniform_nodes(64), order=2, a4=True)
    assert e.value.status == 7
    with pytest.raises(ram.RamError) as e:
        ram.Plan([0, 64], wl.random_nodes(64, seed=1), order=3, a4=True)
    assert e.value.status == 7


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("uniform", [True, False])
def test_limited_order4_matches_oracle(dtype, uniform):
    """Order 4 with the limiter on, on uniform and non-uniform rows (both go to the
    general kernels), a square wave and random data, shifts and steps with a van
    Leer residual."""
    lens = [5, 64, 700, 3000]
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nodes = np.concatenate([wl.uniform_nodes(n) if uniform else wl.random_nodes(n, seed=r)
                            for r, n in enumerate(lens)])
    plan = ram.Plan(ro, nodes, order=4, limiter=True)
    assert plan.info().n_uniform_rows == 0
    rng = np.random.default_rng(12)
    q0 = rng.random(int(ro[-1]))
    q0[ro[2]: ro[2] + 200] = 3.0
    q0 = _rounded(q0, dtype)
    qd = _t(q0, DT[dtype])
    out = torch.empty_like(qd)
    dt = 0.1
    for s in (0.0123, 0.4321, -7.77):
        ram.shift(plan, qd, out, _t(np.full(len(lens), s), torch.float64))
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        for r, n in enumerate(lens):
            sl = slice(int(ro[r]), int(ro[r + 1]))
            x = nodes[ro[r] + r: ro[r + 1] + r + 1]
            ref = oracle.shift(x, q0[sl], s, 4, True)
            assert _rel(got[sl], ref, np.diff(x)) <= TOL[dtype], (s, r)
    dv = np.concatenate([(rng.random(n) - 0.5) * 0.8 * np.diff(nodes[ro[r] + r: ro[r + 1] + r + 1]).min() / dt
                         for r, n in enumerate(lens)])
    dv = _rounded(dv, dtype)
    v0 = rng.uniform(-3, 3, len(lens)) / dt
    ram.step(plan, qd, out, _t(v0, torch.float64), dt, dv=_t(dv, DT[dtype]), scheme=ram.VANLEER)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    for r, n in enumerate(lens):
        sl = slice(int(ro[r]), int(ro[r + 1]))
        x = nodes[ro[r] + r: ro[r + 1] + r + 1]
        ref = oracle.step(x, q0[sl], oracle.shift_from_velocity(v0[r], dt), 4, True, dv[sl], dt,
                          oracle.VANLEER, 1)
        assert _rel(got[sl], ref, np.diff(x)) <= TOL[dtype], ("step", r)
    assert plan.check_errors() == 0


def test_limited_order4_on_the_warp_segment_kernel():
    """FP32 rows with their own mesh, order 4 limited, on the warp-segment kernel:
    oracle parity, and no new extrema over repeated shifts of a square wave."""
    n = 5000
    x = wl.random_nodes(n, seed=13, ratio=3.0)
    plan = ram.Plan([0, n], x, order=4, limiter=True)
    t = plan.tuning()
    t.nonuniform_kernel_f32 = 1
    plan.set_tuning(t)
    assert plan.info().n_nseg_rows == 1
    xc = 0.5 * (x[1:] + x[:-1])
    q0 = np.where((xc > 0.2) & (xc < 0.5), 1.0, 0.0)
    q = _t(q0, torch.float32)
    buf = torch.empty_like(q)
    ref = q0.copy()
    for _ in range(10):
        ram.shift(plan, q, buf, _t([0.01234], torch.float64))
        q, buf = buf, q
        ref = oracle.shift(x, ref, 0.01234, 4, True)
    torch.cuda.synchronize()
    got = q.double().cpu().numpy()
    assert got.max() <= 1.0 + 1e-6 and got.min() >= -1e-6
    assert _rel(got, ref, np.diff(x)) <= TOL["float32"]
