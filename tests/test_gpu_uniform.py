"""GPU parity of the uniform-row path (disks, uniform lines) against the FP64
oracle, through the C ABI.  FP64: relative L1 <= 1e-12; FP32: <= 1e-5."""
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


def _run_step(plan, w, q, dtype, dv=True, scheme=None, phase=None):
    v0 = _t(w.v0, torch.float64)
    qd = _t(q, dtype)
    out = torch.empty_like(qd)
    dvd = _t(w.dv, dtype) if (dv and w.dv is not None) else None
    ns = _t(w.nsub, torch.int32)
    ram.step(plan, qd, out, v0, w.dt, dv=dvd, scheme=w.scheme if scheme is None else scheme,
             nsub=ns, phase=phase)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_line_uniform_c1(dtype):
    """256-cell uniform line, PLM, 7.3 cells/step, 100 steps: parity after 1, 10 and
    100 steps; mass conserved; a whole-period shift returns the input."""
    w = wl.line_uniform()
    plan = ram.Plan.from_workload(w)
    q = _t(w.q0, DT[dtype])
    ref = w.q0.copy()
    shifts = oracle_shifts(w)
    v0 = _t(w.v0, torch.float64)
    buf = torch.empty_like(q)
    for k in range(1, w.steps + 1):
        ram.step(plan, q, buf, v0, w.dt)
        ref = oracle_step(w, ref, shifts)
        if k in (1, 10, 100):
            # the step from the GPU's own input, and the trajectory against the
            # FP64 oracle's, both at the stated tolerance
            torch.cuda.synchronize()
            got = buf.double().cpu().numpy()
            one = oracle_step(w, q.double().cpu().numpy(), shifts)
            assert rel_l1_rows(w, got, one) <= TOL[dtype], (k, rel_l1_rows(w, got, one))
            assert rel_l1_rows(w, got, ref) <= TOL[dtype], (k, rel_l1_rows(w, got, ref))
        q, buf = buf, q
    x = w.row_nodes(0)
    m0 = oracle.mass(x, w.q0)
    assert abs(oracle.mass(x, q.double().cpu().numpy()) - m0) <= (1e-13 if dtype == "float64"
                                                                   else 1e-6) * m0
    # full-period shift is the identity, bit for bit
    out = torch.empty_like(q)
    ram.shift(plan, q, out, _t([3.0], torch.float64))
    torch.cuda.synchronize()
    assert torch.equal(out, q)
    assert plan.check_errors() == 0


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("order,limiter", [(2, True), (2, False), (3, True), (3, False),
                                           (4, False)])
@pytest.mark.parametrize("scheme", [ram.DONOR, ram.VANLEER])
def test_disk_single_step(dtype, order, limiter, scheme):
    """Small disk (rows of 600 cells, tiles of 150: several tiles per row) with the
    residual step sub-cycled per ring."""
    w = wl.disk(n_r=12, n_phi=600, order=order, limiter=limiter, scheme=scheme)
    plan = ram.Plan.from_workload(w)
    plan.set_tiling(150, 128)
    q0 = w.q0.astype(np.float32).astype(np.float64) if dtype == "float32" else w.q0
    dv = w.dv.astype(np.float32).astype(np.float64) if dtype == "float32" else w.dv
    out = _run_step(plan, w, q0, DT[dtype])
    ref = oracle_step(w, q0, oracle_shifts(w), dv=dv, nsub=w.nsub)
    err = rel_l1_rows(w, out.double().cpu().numpy(), ref)
    assert err <= TOL[dtype], err
    assert plan.check_errors() == 0


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_disk_multi_step(dtype):
    """20 steps of the disk recipe (PPM + van Leer): the last step from the GPU's
    own input and the trajectory against the FP64 oracle's, both at the stated
    tolerance."""
    w = wl.disk(n_r=8, n_phi=1024)
    plan = ram.Plan.from_workload(w)
    q = _t(w.q0, DT[dtype])
    buf = torch.empty_like(q)
    v0 = _t(w.v0, torch.float64)
    dvd = _t(w.dv, DT[dtype])
    ns = _t(w.nsub, torch.int32)
    dvr = dvd.double().cpu().numpy()
    ref = q.double().cpu().numpy()
    shifts = oracle_shifts(w)
    for _ in range(20):
        prev = q.double().cpu().numpy()
        ram.step(plan, q, buf, v0, w.dt, dv=dvd, scheme=w.scheme, nsub=ns)
        q, buf = buf, q
        ref = oracle_step(w, ref, shifts, dv=dvr, nsub=w.nsub)
    torch.cuda.synchronize()
    got = q.double().cpu().numpy()
    one = oracle_step(w, prev, shifts, dv=dvr, nsub=w.nsub)
    assert rel_l1_rows(w, got, one) <= TOL[dtype], rel_l1_rows(w, got, one)
    assert rel_l1_rows(w, got, ref) <= TOL[dtype], rel_l1_rows(w, got, ref)


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("k", [0, 1, 37, 255, 256, 1000, -3])
def test_integer_roll_bit_exact(dtype, k):
    """Sec. 1: a whole-cell shift on a uniform periodic mesh is a cyclic
    permutation (dyadic mesh: s = k dx exactly)."""
    n = 256
    x = wl.uniform_nodes(n)
    plan = ram.Plan([0, n], x, order=3)
    q = torch.rand(n, dtype=DT[dtype], device=DEV)
    out = torch.empty_like(q)
    ram.shift(plan, q, out, _t([k / n], torch.float64))
    torch.cuda.synchronize()
    assert torch.equal(out, torch.roll(q, k))


@pytest.mark.parametrize("n,tile", [(1, 64), (2, 64), (3, 64), (5, 64), (17, 64),
                                    (1023, 256), (1025, 256), (4097, 1024), (300, 64)])
@pytest.mark.parametrize("order", [2, 3, 4])
def test_ragged_and_tiny_rows(n, tile, order):
    """Rows shorter than the stencil plus halo, rows one cell off a tile multiple,
    shifts of many periods in both directions; FP64 parity."""
    x = wl.uniform_nodes(n, -1.0, 2.0)
    rng = np.random.default_rng(n)
    q0 = 1.0 + rng.random(n)
    dv = 0.3 * (rng.random(n) - 0.5)
    plan = ram.Plan([0, n], x, order=order, limiter=(order != 4))
    plan.set_tiling(tile, 64)
    qd = _t(q0, torch.float64)
    dvd = _t(dv, torch.float64)
    for s in (0.0, 0.37, 2.0 * 13.0 + 0.001, -5.5, 1234.5678):
        dt = 0.5 * (2.0 / n) / 0.15  # |dv| dt / dx <= 0.5
        out = torch.empty_like(qd)
        v0 = _t([s / dt], torch.float64)
        ram.step(plan, qd, out, v0, dt, dv=dvd, scheme=ram.VANLEER)
        torch.cuda.synchronize()
        ref = oracle.step(x, q0, oracle.shift_from_velocity(s / dt, dt), order, order != 4,
                          dv, dt, oracle.VANLEER, 1)
        got = out.cpu().numpy()
        err = np.sum(np.abs(got - ref)) / np.sum(np.abs(ref))
        assert err <= 1e-12, (s, err)
    assert plan.check_errors() == 0


def test_shift_only_and_residual_only():
    w = wl.disk(n_r=6, n_phi=700)
    plan = ram.Plan.from_workload(w)
    q = _t(w.q0, torch.float64)
    out = torch.empty_like(q)
    sh = np.linspace(-3.0, 50.0, w.n_rows)
    ram.shift(plan, q, out, _t(sh, torch.float64))
    torch.cuda.synchronize()
    ref = np.concatenate([oracle.shift(w.nodes, w.q0[w.row_slice(r)], sh[r], 3, True)
                          for r in range(w.n_rows)])
    assert rel_l1_rows(w, out.cpu().numpy(), ref) <= 1e-12
    dvd = _t(w.dv, torch.float64)
    ns = _t(w.nsub, torch.int32)
    ram.residual_upwind(plan, q, out, dvd, w.dt, ram.VANLEER, ns)
    torch.cuda.synchronize()
    ref = np.concatenate([oracle.residual(w.nodes, w.q0[w.row_slice(r)], w.dv[w.row_slice(r)],
                                          w.dt, oracle.VANLEER, int(w.nsub[r]))
                          for r in range(w.n_rows)])
    assert rel_l1_rows(w, out.cpu().numpy(), ref) <= 1e-12


def test_phase_bookkeeping():
    w = wl.disk(n_r=5, n_phi=256)
    plan = ram.Plan.from_workload(w)
    q = _t(w.q0, torch.float64)
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


def test_device_error_flags():
    n = 64
    x = wl.uniform_nodes(n)
    plan = ram.Plan([0, n], x, order=2)
    q = torch.ones(n, dtype=torch.float64, device=DEV)
    out = torch.empty_like(q)
    # CFL above 1
    ram.residual_upwind(plan, q, out, torch.full_like(q, 3.0), 1.0 / n)
    assert plan.check_errors() == 3
    assert plan.check_errors() == 0  # cleared
    # non-finite shift
    ram.shift(plan, q, out, _t([math.nan], torch.float64))
    assert plan.check_errors() == 8
    # sub-step count out of range
    ram.residual_upwind(plan, q, out, torch.zeros_like(q), 0.1, ram.VANLEER,
                        _t([99], torch.int32))
    assert plan.check_errors() == 1
    # aliasing is refused on the host
    with pytest.raises(ram.RamError) as e:
        ram.shift(plan, q, q, _t([0.1], torch.float64))
    assert e.value.status == 1


def test_full_size_disk_sampled():
    """The 1024 x 4096 disk recipe at full size, FP32 and FP64, one step in the
    launch configuration the benchmark uses; sampled rings against the oracle."""
    w = wl.disk()
    plan = ram.Plan.from_workload(w)
    rows = [0, 1, 200, 511, 777, 1023]
    shifts = oracle_shifts(w)
    for dtype in ("float32", "float64"):
        q0 = w.q0.astype(np.float32).astype(np.float64) if dtype == "float32" else w.q0
        dv = w.dv.astype(np.float32).astype(np.float64) if dtype == "float32" else w.dv
        out = _run_step(plan, w, q0, DT[dtype]).double().cpu().numpy()
        ref = oracle_step(w, q0, shifts, dv=dv, nsub=w.nsub, rows=rows)
        for r in rows:
            sl = w.row_slice(r)
            err = np.sum(np.abs(out[sl] - ref[sl])) / np.sum(np.abs(ref[sl]))
            assert err <= TOL[dtype], (dtype, r, err)
    assert plan.check_errors() == 0


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_uniform_rows_of_mixed_lengths(dtype):
    """Uniform rows of different lengths in one plan: lengths that the persistent
    whole-row kernel takes (16-byte aligned, up to its shared-memory cap, partial
    last groups) and lengths that go to the tiled kernel, with per-row shifts and
    sub-step counts."""
    lens = [16, 20, 64, 1000, 1024, 4096, 5000, 12288, 13000, 7]
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nodes = np.concatenate([wl.uniform_nodes(n, -0.5, 1.0 + 0.1 * r) for r, n in enumerate(lens)])
    rng = np.random.default_rng(5)
    q0 = 1.0 + rng.random(int(ro[-1]))
    dv = 0.2 * (rng.random(int(ro[-1])) - 0.5)
    plan = ram.Plan(ro, nodes, order=3, limiter=True)
    dt = 0.01
    v0 = rng.uniform(-30.0, 30.0, len(lens))
    nsub = np.array([1 + (r % 3) for r in range(len(lens))], dtype=np.int32)
    # keep |dv| dt / (nsub dx) <= 1: dx = L / n
    for r, n in enumerate(lens):
        L = 1.0 + 0.1 * r
        dv[ro[r]:ro[r + 1]] *= min(1.0, 0.9 * nsub[r] * (L / n) / (0.1 * dt))
    qd = _t(q0, DT[dtype])
    out = torch.empty_like(qd)
    dvd = _t(dv, DT[dtype])
    ram.step(plan, qd, out, _t(v0, torch.float64), dt, dv=dvd, scheme=ram.VANLEER,
             nsub=_t(nsub, torch.int32))
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    qr = qd.double().cpu().numpy()
    dvr = dvd.double().cpu().numpy()
    for r, n in enumerate(lens):
        sl = slice(int(ro[r]), int(ro[r + 1]))
        x = nodes[ro[r] + r: ro[r + 1] + r + 1]
        ref = oracle.step(x, qr[sl], oracle.shift_from_velocity(v0[r], dt), 3, True, dvr[sl],
                          dt, oracle.VANLEER, int(nsub[r]))
        err = np.sum(np.abs(got[sl] - ref)) / np.sum(np.abs(ref))
        assert err <= TOL[dtype], (n, err)
    assert plan.check_errors() == 0


def test_misaligned_arrays_take_the_tiled_path():
    """Arrays that are not 16-byte aligned cannot be read with TMA; the launcher
    falls back to the tiled kernel and the result is the same."""
    w = wl.disk(n_r=4, n_phi=512)
    plan = ram.Plan.from_workload(w)
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


def test_autotune_and_tuning_roundtrip():
    """The autotuner keeps a valid candidate; every launch shape gives the same
    result within round-off."""
    w = wl.disk(n_r=16, n_phi=2048)
    plan = ram.Plan.from_workload(w)
    q = _t(w.q0, torch.float32)
    dvd = _t(w.dv, torch.float32)
    v0 = _t(w.v0, torch.float64)
    ns = _t(w.nsub, torch.int32)
    outs = []
    for v in (5, 7, 9, 11, 15):
        t = plan.tuning()
        t.rows_cells_per_thread_f32 = v
        plan.set_tuning(t)
        o = torch.empty_like(q)
        ram.step(plan, q, o, v0, w.dt, dv=dvd, scheme=ram.VANLEER, nsub=ns)
        outs.append(o)
    torch.cuda.synchronize()
    for o in outs[1:]:
        assert torch.allclose(o, outs[0], rtol=1e-6, atol=1e-7)
    t = ram.autotune(plan, q, torch.empty_like(q), v0, w.dt, dv=dvd, scheme=ram.VANLEER,
                     nsub=ns, reps=3)
    assert t.rows_cells_per_thread_f32 in (5, 7, 9, 11, 15)
    assert plan.check_errors() == 0


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("scheme,nsub_max", [(ram.VANLEER, 8), (ram.DONOR, 8), (ram.VANLEER, 1)])
def test_both_uniform_kernels_match_oracle(dtype, scheme, nsub_max):
    """The warp-segment, persistent whole-row and streaming-warp kernels against the
    oracle, with sub-step counts up to the maximum (widest warp halos) and rows
    long enough for several warp segments."""
    n_r, n_phi = 6, 2048
    x = wl.uniform_nodes(n_phi, 0.0, 2 * np.pi)
    rng = np.random.default_rng(21)
    q0 = 1.0 + rng.random(n_r * n_phi)
    nsub = np.array([1 + (r * 3) % nsub_max for r in range(n_r)], dtype=np.int32)
    dt = 0.5
    dxc = 2 * np.pi / n_phi
    dv = (rng.random(n_r * n_phi) - 0.5) * 1.6 * dxc / dt
    dv *= np.repeat(nsub, n_phi) / nsub_max  # |dv| dt / (nsub dx) <= 0.8 / nsub_max
    v0 = rng.uniform(-400.0, 400.0, n_r) * dxc / dt
    ro = np.arange(n_r + 1, dtype=np.int64) * n_phi
    plan = ram.Plan(ro, x, order=3, shared_mesh=True)
    qd, dvd = _t(q0, DT[dtype]), _t(dv, DT[dtype])
    qr, dvr = qd.double().cpu().numpy(), dvd.double().cpu().numpy()
    refs = np.concatenate([oracle.step(x, qr[r * n_phi:(r + 1) * n_phi],
                                       oracle.shift_from_velocity(v0[r], dt), 3, True,
                                       dvr[r * n_phi:(r + 1) * n_phi], dt, scheme, int(nsub[r]))
                           for r in range(n_r)])
    # kernels: 0 whole-row, 1 warp segments (FP32: one segment in flight, the next
    # one's loads in flight, shared-memory rings with the shift parameters formed
    # in the kernel; 3-8 warps per row CTA), 2 streaming warps (FP32; V = 4, 8)
    for kern, sv, gw in ((0, 8, 8), (1, 0, 8), (1, 0, 3), (1, 1, 6), (1, 1, 4), (1, 2, 3),
                         (1, 2, 8), (2, 4, 8), (2, 8, 8)):
        if kern == 2 and dtype == "float64":
            continue
        t = plan.tuning()
        t.uniform_kernel_f32 = kern
        t.uniform_kernel_f64 = min(kern, 1)
        t.seg_warps = gw
        if kern == 2:
            t.stream_cells_per_lane_f32 = sv
        elif kern == 1:
            t.seg_variant_f32 = sv
        plan.set_tuning(t)
        out = torch.empty_like(qd)
        ram.step(plan, qd, out, _t(v0, torch.float64), dt, dv=dvd, scheme=scheme,
                 nsub=_t(nsub, torch.int32))
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        for r in range(n_r):
            sl = slice(r * n_phi, (r + 1) * n_phi)
            err = np.sum(np.abs(got[sl] - refs[sl])) / np.sum(np.abs(refs[sl]))
            assert err <= TOL[dtype], (kern, sv, gw, r, err)
    assert plan.check_errors() == 0
