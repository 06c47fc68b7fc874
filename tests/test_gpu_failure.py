"""Failure detection on the GPU without a fault: the bounded device-side waits of
the persistent whole-row kernel give up when their try count is 0, record
RAM_ERR_TIMEOUT in the plan's error word and end the launch; the context stays
usable and the next step with the default count matches a step taken before."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2305_05362_gb300 import ram, workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
DT = {"float64": torch.float64, "float32": torch.float32}
TIMEOUT = 5


def _inputs(w, dtype):
    t = lambda a, d: torch.tensor(np.asarray(a), dtype=d, device=DEV)
    return (t(w.q0, DT[dtype]), t(w.v0, torch.float64), t(w.dv, DT[dtype]),
            t(w.nsub, torch.int32))


def _step(plan, w, q, v0, dv, ns):
    out = torch.empty_like(q)
    ram.step(plan, q, out, v0, w.dt, dv=dv, scheme=w.scheme, nsub=ns)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_wait_timeout_is_reported_and_context_survives(dtype):
    # 1024 rings: several rows per persistent CTA, more than its staging ring
    # holds, so both the producer's and the consumers' waits are reached
    w = wl.disk(1024, 512)
    plan = ram.Plan.from_workload(w)
    t = plan.tuning()
    t.uniform_kernel_f32 = 0
    t.uniform_kernel_f64 = 0
    plan.set_tuning(t)
    q, v0, dv, ns = _inputs(w, dtype)

    ref = _step(plan, w, q, v0, dv, ns)
    assert plan.check_errors() == 0

    plan.set_wait_limit(0)
    _step(plan, w, q, v0, dv, ns)
    assert plan.check_errors() == TIMEOUT
    assert plan.check_errors() == 0  # read and cleared

    plan.set_wait_limit()
    again = _step(plan, w, q, v0, dv, ns)
    assert plan.check_errors() == 0
    assert torch.equal(again, ref)


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_kernels_without_waits_ignore_the_limit(variant):
    """The warp-segment kernels (one segment in flight, the next one's loads in
    flight, shared-memory rings of asynchronous copies) have no waits of their
    own: a try count of 0 changes nothing."""
    w = wl.disk(64, 8192)
    plan = ram.Plan.from_workload(w)
    t = plan.tuning()
    t.uniform_kernel_f32 = 1
    t.uniform_kernel_f64 = 1
    t.seg_variant_f32 = variant
    t.seg_warps = 3
    plan.set_tuning(t)
    for dtype in ("float64", "float32"):
        q, v0, dv, ns = _inputs(w, dtype)
        ref = _step(plan, w, q, v0, dv, ns)
        plan.set_wait_limit(0)
        got = _step(plan, w, q, v0, dv, ns)
        plan.set_wait_limit()
        assert plan.check_errors() == 0
        assert torch.equal(got, ref)
