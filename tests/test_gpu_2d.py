"""The dimensionally split two-dimensional step (Sec. 3.5) on the GPU through the C
ABI: the RAM step of every ring of a polar disk, then the radial sweep
(ram_radial_upwind), on the mesh of Sec. 4.2 (periodic bump in phi, radial bump
in r, App. B) and on a uniform / log-uniform one, against the FP64 oracle
(relative L1 <= 1e-12 FP64, <= 1e-5 FP32, per ring)."""
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


def _rel_rings(got, ref):
    return float(np.max(np.abs(got - ref).sum(axis=1) / np.abs(ref).sum(axis=1)))


def _plan(d):
    n = d.n_phi
    ro = np.arange(d.n_r + 1, dtype=np.int64) * n
    return ram.Plan(ro, d.phi, order=d.order, limiter=d.limiter, shared_mesh=True)


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("nonuniform", [True, False])
@pytest.mark.parametrize("order,scheme", [(2, ram.VANLEER), (3, ram.DONOR)])
def test_split_step_matches_oracle(dtype, nonuniform, order, scheme):
    d = wl.polar_disk_2d(n_r=96, n_phi=384, nonuniform=nonuniform, order=order, scheme=scheme)
    plan = _plan(d)
    q0 = d.q0.astype(np.float32).astype(np.float64) if dtype == "float32" else d.q0
    dvp = d.dvphi.astype(np.float32).astype(np.float64) if dtype == "float32" else d.dvphi
    vr = d.vr.astype(np.float32).astype(np.float64) if dtype == "float32" else d.vr
    q = _t(q0.reshape(-1), DT[dtype])
    out = torch.empty_like(q)
    scratch = torch.empty_like(q)
    om = _t(d.omega, torch.float64)
    rf = _t(d.rf, torch.float64)
    vrd = _t(vr.reshape(-1), DT[dtype])
    dvd = _t(dvp.reshape(-1), DT[dtype])
    ns = _t(d.nsub, torch.int32)
    ref = q0.copy()
    for k in range(1, 11):
        prev = q.double().cpu().numpy().reshape(d.n_r, d.n_phi)
        ram.step_2d(plan, q, out, om, d.dt, rf, vrd, dvphi=dvd, scheme=scheme, nsub=ns,
                    scratch=scratch)
        ref = oracle.step_2d(d.phi, d.rf, d.omega, ref, d.dt, order, True, dvp, scheme, d.nsub, vr)
        if k in (1, 10):
            torch.cuda.synchronize()
            got = out.double().cpu().numpy().reshape(d.n_r, d.n_phi)
            one = oracle.step_2d(d.phi, d.rf, d.omega, prev, d.dt, order, True, dvp, scheme,
                                 d.nsub, vr)
            assert _rel_rings(got, one) <= TOL[dtype], (k, _rel_rings(got, one))
            assert _rel_rings(got, ref) <= TOL[dtype], (k, _rel_rings(got, ref))
        q, out = out, q
    assert plan.check_errors() == 0


@pytest.mark.parametrize("scheme", [ram.DONOR, ram.VANLEER])
def test_radial_sweep_alone_and_conservation(scheme):
    d = wl.polar_disk_2d(n_r=200, n_phi=256)
    plan = _plan(d)
    q = _t(d.q0.reshape(-1), torch.float64)
    out = torch.empty_like(q)
    ram.radial_upwind(plan, q, out, _t(d.rf, torch.float64), _t(d.vr.reshape(-1), torch.float64),
                      d.dt, scheme)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(d.n_r, d.n_phi)
    ref = oracle.radial_upwind(d.rf, d.q0, d.vr, d.dt, scheme)
    assert _rel_rings(got, ref) <= 1e-12
    area = 0.5 * (d.rf[1:] ** 2 - d.rf[:-1] ** 2)
    np.testing.assert_allclose((got * area[:, None]).sum(axis=0),
                               (d.q0 * area[:, None]).sum(axis=0), rtol=1e-13)
    assert plan.check_errors() == 0


def test_radial_cfl_flag_and_refusals():
    d = wl.polar_disk_2d(n_r=32, n_phi=128)
    plan = _plan(d)
    q = _t(d.q0.reshape(-1), torch.float64)
    out = torch.empty_like(q)
    vr = _t((d.vr * 1e4).reshape(-1), torch.float64)
    ram.radial_upwind(plan, q, out, _t(d.rf, torch.float64), vr, d.dt)
    assert plan.check_errors() == 3
    # rows with their own meshes are not rings of one disk
    lens = [128, 128]
    ro = np.array([0, 128, 256], dtype=np.int64)
    nodes = np.concatenate([wl.random_nodes(128, seed=1), wl.random_nodes(128, seed=2)])
    own = ram.Plan(ro, nodes, order=2)
    q2 = torch.ones(256, dtype=torch.float64, device=DEV)
    with pytest.raises(ram.RamError) as e:
        ram.radial_upwind(own, q2, torch.empty_like(q2), _t([0.5, 1.0, 1.5], torch.float64),
                          torch.zeros(384, dtype=torch.float64, device=DEV), 0.1)
    assert e.value.status == 7
