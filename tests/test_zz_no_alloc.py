"""The no-allocation step entry point, for callers that cannot call cudaMalloc
(for example code running inside an allocator or memory-pool callback, or beside
a fixed device-memory budget that must not move).  Through the C ABI it must
match the FP64 oracle at the tolerances of every other parity test, on two
calls in a row with different inputs, for every reconstruction order, both
residual schemes and the limiter on or off, and it must not change the device's
free memory.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2305_05362_gb300 import ram, workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _rel_rows(got, ref, n_rows):
    """Max over rows of the relative L1 error (uniform rows: plain sums)."""
    g = got.reshape(n_rows, -1)
    r = ref.reshape(n_rows, -1)
    return float((np.abs(g - r).sum(axis=1) / np.abs(r).sum(axis=1)).max())


def _oracle(w, q, v0, order, limiter, scheme, dv):
    shifts = np.array([oracle.shift_from_velocity(v, w.dt) for v in v0])
    return oracle.step_rows(w.row_offset, w.nodes, True, np.full(w.n_rows, order, np.int8),
                            limiter, shifts, q, dv=dv, dt=w.dt, scheme=scheme, nsub=w.nsub)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("order,limiter", [(2, True), (2, False), (3, True), (3, False),
                                           (4, False)])
@pytest.mark.parametrize("scheme", [ram.DONOR, ram.VANLEER])
def test_noalloc_step_matches_oracle_twice(dtype, order, limiter, scheme):
    w = wl.disk(n_r=48, n_phi=1024, order=order, limiter=limiter, scheme=scheme)
    v0 = torch.tensor(w.v0, dtype=torch.float64, device=DEV)
    dv = torch.tensor(w.dv, dtype=dtype, device=DEV)
    ns = torch.tensor(w.nsub, dtype=torch.int32, device=DEV)
    errs = torch.zeros(1, dtype=torch.int32, device=DEV)
    q = torch.tensor(w.q0, dtype=dtype, device=DEV)
    for call in range(2):
        # a different input and velocity on the second call: nothing may carry over
        qi = q if call == 0 else torch.flip(q, [0]).contiguous()
        vi = v0 if call == 0 else 0.5 * v0
        out = torch.empty_like(qi)
        ram.step_uniform_noalloc(qi, out, w.n_rows, w.period(0), order, vi, w.dt, dv=dv,
                                 scheme=scheme, nsub=ns, limiter=limiter, device_errors=errs)
        torch.cuda.synchronize()
        ref = _oracle(w, qi.double().cpu().numpy(), vi.cpu().numpy(), order, limiter, scheme,
                      dv.double().cpu().numpy())
        err = _rel_rows(out.double().cpu().numpy(), ref, w.n_rows)
        assert err <= TOL[dtype], (call, err)
    assert int(errs.item()) == 0


def test_noalloc_at_its_row_limit_without_allocating():
    """Exactly RAM_STATIC_MAX_ROWS rows of 512 cells: oracle parity on sampled rows,
    and the device's free memory is the same before and after repeated calls."""
    n_rows = ram.STATIC_MAX_ROWS
    w = wl.disk(n_r=n_rows, n_phi=512, order=3)
    v0 = torch.tensor(w.v0, dtype=torch.float64, device=DEV)
    dv = torch.tensor(w.dv, dtype=torch.float32, device=DEV)
    ns = torch.tensor(w.nsub, dtype=torch.int32, device=DEV)
    q = torch.tensor(w.q0, dtype=torch.float32, device=DEV)
    out = torch.empty_like(q)
    ram.step_uniform_noalloc(q, out, n_rows, w.period(0), 3, v0, w.dt, dv=dv, nsub=ns)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        ram.step_uniform_noalloc(q, out, n_rows, w.period(0), 3, v0, w.dt, dv=dv, nsub=ns)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    got = out.double().cpu().numpy().reshape(n_rows, -1)
    q64 = q.double().cpu().numpy().reshape(n_rows, -1)
    dv64 = dv.double().cpu().numpy().reshape(n_rows, -1)
    x = w.nodes
    for r in (0, 1, 1000, 2047, 3333, n_rows - 1):
        s = oracle.shift_from_velocity(w.v0[r], w.dt)
        ref = oracle.step(x, q64[r], s, 3, True, dv64[r], w.dt, oracle.VANLEER, int(w.nsub[r]))
        err = float(np.abs(got[r] - ref).sum() / np.abs(ref).sum())
        assert err <= TOL[torch.float32], (r, err)


def test_noalloc_rejects_sizes_beyond_its_static_array():
    n_rows = ram.STATIC_MAX_ROWS + 1
    q = torch.zeros(n_rows * 512, dtype=torch.float32, device=DEV)
    out = torch.empty_like(q)
    v0 = torch.zeros(n_rows, dtype=torch.float64, device=DEV)
    with pytest.raises(ram.RamError) as e:
        ram.step_uniform_noalloc(q, out, n_rows, 1.0, 3, v0, 0.1)
    assert e.value.status == 1


def test_noalloc_rejects_unknown_flags():
    """Only RAM_LIMITER_OFF is a valid flag; anything else is refused, not ignored."""
    lib = ram.load()
    q = torch.zeros(4 * 512, dtype=torch.float32, device=DEV)
    out = torch.empty_like(q)
    v0 = torch.zeros(4, dtype=torch.float64, device=DEV)
    st = lib.ram_step_uniform_noalloc(0, 4, 512, 1.0, 3, ram.SHARED_MESH, q.data_ptr(),
                                      out.data_ptr(), v0.data_ptr(), 0.1, None, 1, None, None,
                                      torch.cuda.current_stream().cuda_stream)
    assert st == 1
