"""GPU parity at the benchmark's full sizes, in the launch configurations the
benchmark times, on sampled rows that the FP64 oracle computes one by one:

  - the batched recipe: 512 and 8192 uneven rows of 64..65536 cells with their
    own non-uniform meshes, per-row shifts of 0.3-200 mean cells, orders 2/3/4,
    launch shapes chosen by the autotuner;
  - the large disk: 8192 rings x 16384 cells (134 M cells), PPM + van Leer
    residual, in both warp-count shapes the benchmark picks between.

FP64 relative L1 <= 1e-12, FP32 <= 1e-5, per row."""
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


def _rel(got, ref):
    return float(np.sum(np.abs(got - ref)) / np.sum(np.abs(ref)))


def _sample_rows(w, k, seed):
    """The longest and shortest rows, the rows of every order, and random others."""
    lens = np.diff(w.row_offset)
    rng = np.random.default_rng(seed)
    rows = {int(np.argmax(lens)), int(np.argmin(lens))}
    for o in (2, 3, 4):
        idx = np.nonzero(np.asarray(w.order) == o)[0]
        if idx.size:
            rows.add(int(idx[np.argmax(lens[idx])]))
    rows.update(int(r) for r in rng.choice(w.n_rows, size=k, replace=False))
    return sorted(rows)


@pytest.fixture(scope="module")
def batched_512():
    return wl.batched(n_rows=512)


@pytest.mark.parametrize("dtype,nseg", [("float32", None), ("float32", 1), ("float64", None)])
def test_batched_512_rows_autotuned(batched_512, dtype, nseg):
    """Autotuned launch shapes (nseg None), and the FP32 warp-segment kernel forced."""
    w = batched_512
    assert int(np.diff(w.row_offset).max()) > 60000
    plan = ram.Plan.from_workload(w)
    q = _t(w.q0, DT[dtype])
    out = torch.empty_like(q)
    v0 = _t(w.v0, torch.float64)
    ram.autotune(plan, q, out, v0, w.dt, reps=3)
    if nseg is not None:
        t = plan.tuning()
        t.nonuniform_kernel_f32 = nseg
        plan.set_tuning(t)
        assert plan.info().n_nseg_rows == w.n_rows
    ram.step(plan, q, out, v0, w.dt)
    torch.cuda.synchronize()
    assert plan.check_errors() == 0
    got = out.double().cpu().numpy()
    q64 = q.double().cpu().numpy()
    for r in _sample_rows(w, 24, seed=1):
        sl = w.row_slice(r)
        ref = oracle.step(w.row_nodes(r), q64[sl], oracle.shift_from_velocity(w.v0[r], w.dt),
                          int(w.order[r]), w.limiter)
        assert _rel(got[sl], ref) <= TOL[dtype], (r, int(w.order[r]), _rel(got[sl], ref))


def test_batched_8192_rows_autotuned_sampled():
    """The 8192-row batch the benchmark times (76 M cells, rows of 64-65536 cells
    with their own meshes, orders 2/3/4), FP32, in the autotuner's launch shapes:
    sampled rows against the oracle."""
    w = wl.batched(n_rows=8192)
    assert w.n_cells > 70_000_000
    plan = ram.Plan.from_workload(w)
    q = _t(w.q0, torch.float32)
    out = torch.empty_like(q)
    v0 = _t(w.v0, torch.float64)
    ram.autotune(plan, q, out, v0, w.dt, reps=2)
    ram.step(plan, q, out, v0, w.dt)
    torch.cuda.synchronize()
    assert plan.check_errors() == 0
    q64 = q.double().cpu().numpy()
    for r in _sample_rows(w, 24, seed=2):
        sl = w.row_slice(r)
        got = out[sl].double().cpu().numpy()
        ref = oracle.step(w.row_nodes(r), q64[sl], oracle.shift_from_velocity(w.v0[r], w.dt),
                          int(w.order[r]), w.limiter)
        assert _rel(got, ref) <= TOL["float32"], (r, int(w.order[r]), _rel(got, ref))
    del plan


def test_large_disk_sampled_rings():
    w = wl.disk(n_r=8192, n_phi=16384, dtype=np.float32)
    plan = ram.Plan.from_workload(w)
    q = _t(w.q0, torch.float32)
    dv = _t(w.dv, torch.float32)
    out = torch.empty_like(q)
    v0 = _t(w.v0, torch.float64)
    ns = _t(w.nsub, torch.int32)
    rows = [0, 1, 2047, 4096, 6000, 8191]
    q64 = w.q0.astype(np.float64)
    dv64 = w.dv.astype(np.float64)
    x = w.nodes
    for warps in (3, 4):
        t = plan.tuning()
        t.uniform_kernel_f32, t.seg_variant_f32, t.seg_warps = 1, 2, warps
        plan.set_tuning(t)
        ram.step(plan, q, out, v0, w.dt, dv=dv, scheme=w.scheme, nsub=ns)
        torch.cuda.synchronize()
        assert plan.check_errors() == 0
        for r in rows:
            sl = w.row_slice(r)
            got = out[sl].double().cpu().numpy()
            ref = oracle.step(x, q64[sl], oracle.shift_from_velocity(w.v0[r], w.dt),
                              int(w.order[r]), w.limiter, dv64[sl], w.dt, w.scheme,
                              int(w.nsub[r]))
            assert _rel(got, ref) <= TOL["float32"], (warps, r, _rel(got, ref))
