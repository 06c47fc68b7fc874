"""The Python binding refuses tensors whose size, dtype or device does not match
what the C ABI will read or write through them, before any pointer reaches the
library (a short or mistyped buffer would otherwise be read or written past its
end on the GPU).  CPU only: the plan is a stand-in with the sizes of a real one
and the checks run against CPU tensors."""
import types

import pytest

torch = pytest.importorskip("torch")

from paper_2305_05362_gb300 import ram


@pytest.fixture
def plan(monkeypatch):
    p = ram.Plan.__new__(ram.Plan)
    p.n_rows, p.n_cells, p.device, p.handle = 4, 40, 0, None
    # a library that must never be reached with CPU tensors
    p._lib = types.SimpleNamespace(**{n: (lambda *a: pytest.fail("library called"))
                                      for n in ram.EXPORTS})
    # the checks compare devices with the plan's; point it at the CPU tensors here
    monkeypatch.setattr(ram, "_plan_device", lambda plan: torch.device("cpu"))
    return p


def _f32(n):
    return torch.zeros(n, dtype=torch.float32)


def _f64(n):
    return torch.zeros(n, dtype=torch.float64)


def test_step_refusals(plan):
    q, out, v0 = _f32(40), _f32(40), _f64(4)
    bad = [
        dict(q_in=_f32(39)),                         # short input
        dict(q_out=_f32(41)),                        # output of another size
        dict(q_out=_f64(40)),                        # output of another dtype
        dict(v0=_f64(3)),                            # one velocity missing
        dict(v0=_f32(4)),                            # FP32 velocities
        dict(dv=_f32(20)),                           # short dv
        dict(dv=_f64(40)),                           # dv of another dtype than q
        dict(nsub=torch.ones(4, dtype=torch.int64)), # nsub not int32
        dict(nsub=torch.ones(5, dtype=torch.int32)),
        dict(phase=_f64(2)),
    ]
    for kw in bad:
        args = dict(q_in=q, q_out=out, v0=v0, dv=None, nsub=None, phase=None)
        args.update(kw)
        with pytest.raises(ValueError):
            ram.step(plan, args["q_in"], args["q_out"], args["v0"], 0.1, dv=args["dv"],
                     nsub=args["nsub"], phase=args["phase"])
    with pytest.raises(TypeError):
        ram.step(plan, torch.zeros(40, dtype=torch.int32), out, v0, 0.1)


def test_valid_arguments_reach_the_pointer_stage(plan):
    """Arguments of the right sizes pass the checks; CPU tensors are then refused
    as not being CUDA tensors (the library is never called with them)."""
    with pytest.raises(ValueError, match="CUDA"):
        ram.step(plan, _f32(40), _f32(40), _f64(4), 0.1, dv=_f32(40),
                 nsub=torch.ones(4, dtype=torch.int32), phase=_f64(4))


def test_shift_residual_adjoint_mass_refusals(plan):
    with pytest.raises(ValueError):
        ram.shift(plan, _f32(40), _f32(40), _f64(5))
    with pytest.raises(ValueError):
        ram.residual_upwind(plan, _f32(40), _f32(40), None, 0.1)
    with pytest.raises(ValueError):
        ram.residual_upwind(plan, _f32(40), _f32(40), _f32(39), 0.1)
    with pytest.raises(ValueError):
        ram.step_adjoint(plan, _f32(40), _f32(40), _f32(40), _f64(4), 0.1, g_dv=_f32(7))
    with pytest.raises(ValueError):
        ram.step_adjoint(plan, _f32(30), _f32(40), _f32(40), _f64(4), 0.1)
    with pytest.raises(ValueError):
        ram.row_mass(plan, _f32(40), _f32(4))
    with pytest.raises(ValueError):
        ram.row_mass(plan, _f32(40), _f64(3))


def test_noalloc_refusals():
    q, out = _f32(8 * 512), _f32(8 * 512)
    v0 = _f64(8)
    cases = [
        dict(q_in=_f32(8 * 512 + 4)),               # not a multiple of n_rows
        dict(q_out=_f32(8 * 512 - 4)),
        dict(q_out=_f64(8 * 512)),
        dict(v0=_f32(8)),
        dict(v0=_f64(7)),
        dict(dv=_f32(100)),
        dict(nsub=torch.ones(8, dtype=torch.int64)),
        dict(device_errors=torch.zeros(1, dtype=torch.int64)),
    ]
    for kw in cases:
        args = dict(q_in=q, q_out=out, v0=v0, dv=None, nsub=None, device_errors=None)
        args.update(kw)
        with pytest.raises(ValueError):
            ram.step_uniform_noalloc(args["q_in"], args["q_out"], 8, 1.0, 3, args["v0"], 0.1,
                                     dv=args["dv"], nsub=args["nsub"],
                                     device_errors=args["device_errors"])
    with pytest.raises(ValueError):
        ram.step_uniform_noalloc(q, out, 0, 1.0, 3, v0, 0.1)


def test_shear_dt_host_helper_matches_the_oracle():
    import numpy as np
    import oracle
    from paper_2305_05362_gb300 import workloads as wl
    rf = wl.radial_bump_nodes(80, 0.4, 2.1, 1.0, 0.1387, 0.2773, 2.5)
    rc = 0.5 * (rf[1:] + rf[:-1])
    om = rc ** -1.5 - 1.0
    assert ram.shear_dt(om, 0.013, 0.44) == oracle.shear_dt(om, 0.013, 0.44)
    assert ram.shear_dt(np.ones(4), 0.013) == float("inf")
