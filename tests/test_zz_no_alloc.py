"""The no-allocation step entry point, for callers that cannot call cudaMalloc
(for example code running inside an allocator callback or beside a fixed
device-memory budget): it must give the same result as the planned ram_step
through the C ABI, on two calls in a row, with no device allocation of its own.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2305_05362_gb300 import ram, workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _rel(a, b):
    a, b = a.double(), b.double()
    return float((a - b).abs().sum() / b.abs().sum())


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_step_matches_planned_step_twice(dtype):
    w = wl.disk(n_r=48, n_phi=1024)
    plan = ram.Plan.from_workload(w)
    v0 = torch.tensor(w.v0, dtype=torch.float64, device=DEV)
    dv = torch.tensor(w.dv, dtype=dtype, device=DEV)
    ns = torch.tensor(w.nsub, dtype=torch.int32, device=DEV)
    errs = torch.zeros(1, dtype=torch.int32, device=DEV)
    q = torch.tensor(w.q0, dtype=dtype, device=DEV)
    for call in range(2):
        # a different input and velocity on the second call: nothing may carry over
        qi = q if call == 0 else torch.flip(q, [0]).contiguous()
        vi = v0 if call == 0 else 0.5 * v0
        ref = torch.empty_like(qi)
        ram.step(plan, qi, ref, vi, w.dt, dv=dv, scheme=ram.VANLEER, nsub=ns)
        out = torch.empty_like(qi)
        ram.step_uniform_noalloc(qi, out, w.n_rows, w.period(0), 3, vi, w.dt, dv=dv,
                                 scheme=ram.VANLEER, nsub=ns, device_errors=errs)
        torch.cuda.synchronize()
        assert _rel(out, ref) <= TOL[dtype], (call, _rel(out, ref))
    assert int(errs.item()) == 0
    assert plan.check_errors() == 0


def test_noalloc_rejects_sizes_beyond_its_static_array():
    n_rows = ram.STATIC_MAX_ROWS + 1
    q = torch.zeros(n_rows * 512, dtype=torch.float32, device=DEV)
    out = torch.empty_like(q)
    v0 = torch.zeros(n_rows, dtype=torch.float64, device=DEV)
    with pytest.raises(ram.RamError) as e:
        ram.step_uniform_noalloc(q, out, n_rows, 1.0, 3, v0, 0.1)
    assert e.value.status == 1
