"""ctypes binding of libram_gb300.so (include/ram.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Cell, velocity, shift and gradient arrays are torch CUDA tensors (the
binding passes their device pointers and the current CUDA stream); meshes are
host arrays.  If the library has not been built the first call raises -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libram_gb300.so")

RAM_OK = 0
STATUS = {0: "RAM_OK", 1: "RAM_ERR_ARG", 2: "RAM_ERR_MESH", 3: "RAM_ERR_CFL",
          4: "RAM_ERR_CUDA", 5: "RAM_ERR_TIMEOUT", 6: "RAM_ERR_NOMEM",
          7: "RAM_ERR_UNSUPPORTED", 8: "RAM_ERR_NONFINITE"}
RAM_F32, RAM_F64 = 0, 1
DONOR, VANLEER = 0, 1
LIMITER_OFF = 1
SHARED_MESH = 2
ADJOINT = 4
A4 = 8
MAX_NSUB = 8

EXPORTS = ["ram_plan_mesh", "ram_plan_destroy", "ram_shift", "ram_residual_upwind",
           "ram_step", "ram_step_adjoint", "ram_row_mass", "ram_plan_check_errors",
           "ram_plan_query", "ram_plan_set_tiling", "ram_plan_set_wait_limit",
           "ram_plan_get_tuning", "ram_plan_set_tuning", "ram_plan_autotune", "ram_step_uniform_noalloc",
           "ram_radial_upwind", "ram_plan_set_density",
           "ram_status_string", "ram_version"]
STATIC_MAX_ROWS = 4096


class RamError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__("%s: %s (%d)" % (where, STATUS.get(status, "?"), status))


class Density(ctypes.Structure):
    """ram_density: the periodic bump of App. B.1 on [x_min, x_max]."""
    _fields_ = [("x_min", ctypes.c_double), ("x_max", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double)]


class _MeshDesc(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32),
                ("row_offset", ctypes.POINTER(ctypes.c_int64)),
                ("nodes", ctypes.POINTER(ctypes.c_double)),
                ("order", ctypes.POINTER(ctypes.c_int8)),
                ("default_order", ctypes.c_int8),
                ("flags", ctypes.c_uint32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("n_cells", ctypes.c_int64),
                ("n_uniform_rows", ctypes.c_int32), ("n_tiles_uniform", ctypes.c_int32),
                ("n_tiles_general", ctypes.c_int32), ("tile_cells", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("device", ctypes.c_int32),
                ("n_nseg_rows", ctypes.c_int32), ("n_density_rows", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("rows_cells_per_thread_f32", ctypes.c_int32),
                ("rows_cells_per_thread_f64", ctypes.c_int32),
                ("tile_cells", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("uniform_kernel_f32", ctypes.c_int32), ("uniform_kernel_f64", ctypes.c_int32),
                ("rows_ctas_per_sm_f32", ctypes.c_int32), ("rows_ctas_per_sm_f64", ctypes.c_int32),
                ("stream_cells_per_lane_f32", ctypes.c_int32),
                ("seg_variant_f32", ctypes.c_int32), ("seg_warps", ctypes.c_int32),
                ("nonuniform_kernel_f32", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None


def load(path: Optional[str] = None):
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libram_gb300.so not found at %s; build it with "
                           "`python -m paper_2305_05362_gb300.build`" % path)
    lib = ctypes.CDLL(path)
    vp, i32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    lib.ram_plan_mesh.argtypes = [ctypes.POINTER(_MeshDesc), ctypes.c_int,
                                  ctypes.POINTER(vp)]
    lib.ram_plan_destroy.argtypes = [vp]
    lib.ram_shift.argtypes = [vp, i32, vp, vp, vp, vp]
    lib.ram_residual_upwind.argtypes = [vp, i32, vp, vp, vp, f64, i32, vp, vp]
    lib.ram_step.argtypes = [vp, i32, vp, vp, vp, vp, f64, vp, i32, vp, vp]
    lib.ram_step_adjoint.argtypes = [vp, i32, vp, vp, vp, vp, f64, vp, vp, vp, vp]
    lib.ram_row_mass.argtypes = [vp, i32, vp, vp, vp]
    lib.ram_plan_check_errors.argtypes = [vp]
    lib.ram_plan_query.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    lib.ram_plan_set_tiling.argtypes = [vp, i32, i32]
    lib.ram_plan_set_wait_limit.argtypes = [vp, ctypes.c_uint32]
    lib.ram_plan_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    lib.ram_plan_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    lib.ram_plan_autotune.argtypes = [vp, i32, vp, vp, vp, f64, vp, i32, vp, i32, vp]
    lib.ram_step_uniform_noalloc.argtypes = [i32, i32, i32, f64, i32, ctypes.c_uint32, vp, vp,
                                             vp, f64, vp, i32, vp, vp, vp]
    lib.ram_radial_upwind.argtypes = [vp, i32, vp, vp, vp, vp, f64, i32, vp]
    lib.ram_plan_set_density.argtypes = [vp, ctypes.POINTER(Density)]
    lib.ram_status_string.argtypes = [i32]
    lib.ram_status_string.restype = ctypes.c_char_p
    lib.ram_version.restype = i32
    for name in EXPORTS:
        getattr(lib, name).restype = getattr(lib, name).restype or ctypes.c_int
    lib.ram_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != RAM_OK:
        raise RamError(st, where)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return RAM_F32
    if t.dtype == torch.float64:
        return RAM_F64
    raise TypeError("cell arrays must be float32 or float64, got %s" % t.dtype)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _need(t, name: str, numel: int, dtype=None, device=None, optional: bool = False):
    """Refuse, before any pointer reaches the library, a tensor whose size, dtype
    or device does not match what the C ABI will read or write through it (a short
    buffer would be read or written past its end on the GPU)."""
    if t is None:
        if optional:
            return
        raise ValueError("%s is required" % name)
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s has dtype %s, expected %s" % (name, t.dtype, dtype))
    if device is not None and t.device != device:
        raise ValueError("%s is on %s, expected %s" % (name, t.device, device))


def _plan_device(plan: "Plan"):
    import torch
    return torch.device("cuda", plan.device)


def _check_step_args(plan: "Plan", q_in, q_out, per_row=(), dv=None, nsub=None,
                     extra_cells=()):
    """Sizes, dtypes and devices of a planned call's tensors (ValueError)."""
    import torch
    dev = _plan_device(plan)
    _need(q_in, "q_in", plan.n_cells, device=dev)
    _dtype_code(q_in)
    _need(q_out, "q_out", plan.n_cells, q_in.dtype, dev)
    for name, t, optional in per_row:
        _need(t, name, plan.n_rows, torch.float64, dev, optional)
    _need(dv, "dv", plan.n_cells, q_in.dtype, dev, optional=True)
    _need(nsub, "nsub", plan.n_rows, torch.int32, dev, optional=True)
    for name, t, optional in extra_cells:
        _need(t, name, plan.n_cells, q_in.dtype, dev, optional)


def _stream(device: int, stream=None) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return stream.cuda_stream


class Plan:
    """A mesh plan (ram_plan_mesh).  Rows are packed: row r owns cells
    [row_offset[r], row_offset[r+1]).  nodes: per-row meshes packed with one
    extra node per row, or the single shared mesh when shared_mesh=True."""

    def __init__(self, row_offset: Sequence[int], nodes, order=3, limiter: bool = True,
                 shared_mesh: bool = False, device: int = 0, adjoint: bool = False,
                 a4: bool = False):
        lib = load()
        self._lib = lib
        self.row_offset = np.ascontiguousarray(row_offset, dtype=np.int64)
        self.nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        self.n_rows = int(self.row_offset.size - 1)
        self.n_cells = int(self.row_offset[-1])
        self.device = int(device)
        self.limiter = bool(limiter)
        order_arr = np.asarray(order)
        if order_arr.ndim == 0:
            self.order = None
            default = int(order_arr)
        else:
            self.order = np.ascontiguousarray(order_arr, dtype=np.int8)
            default = 0
        desc = _MeshDesc()
        desc.n_rows = self.n_rows
        desc.row_offset = self.row_offset.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        desc.nodes = self.nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        desc.order = (self.order.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
                      if self.order is not None else None)
        desc.default_order = default
        desc.flags = ((0 if limiter else LIMITER_OFF) | (SHARED_MESH if shared_mesh else 0) |
                      (ADJOINT if adjoint else 0) | (A4 if a4 else 0))
        h = ctypes.c_void_p()
        _check(lib.ram_plan_mesh(ctypes.byref(desc), self.device, ctypes.byref(h)),
               "ram_plan_mesh")
        self.handle = h

    @classmethod
    def from_workload(cls, w, device: int = 0, limiter: Optional[bool] = None,
                      adjoint: bool = False, a4: bool = False):
        return cls(w.row_offset, w.nodes, order=w.order,
                   limiter=w.limiter if limiter is None else limiter,
                   shared_mesh=w.shared_mesh, device=device, adjoint=adjoint, a4=a4)

    def destroy(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.ram_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def info(self) -> PlanInfo:
        out = PlanInfo()
        _check(self._lib.ram_plan_query(self.handle, ctypes.byref(out)), "ram_plan_query")
        return out

    def set_tiling(self, tile_cells: int, threads: int):
        _check(self._lib.ram_plan_set_tiling(self.handle, int(tile_cells), int(threads)),
               "ram_plan_set_tiling")

    def tuning(self) -> Tuning:
        out = Tuning()
        _check(self._lib.ram_plan_get_tuning(self.handle, ctypes.byref(out)),
               "ram_plan_get_tuning")
        return out

    def set_tuning(self, t: Tuning):
        _check(self._lib.ram_plan_set_tuning(self.handle, ctypes.byref(t)),
               "ram_plan_set_tuning")

    def set_density(self, densities):
        """ram_plan_set_density: locate the edges of rows generated by the periodic
        bump (App. B.1) with the index function of Sec. 3.2.1.  `densities`: one
        (x_min, x_max, a, b, c) per row (one for a shared mesh), or None."""
        if densities is None:
            _check(self._lib.ram_plan_set_density(self.handle, None), "ram_plan_set_density")
            return
        arr = (Density * len(densities))(*[Density(*map(float, d)) for d in densities])
        _check(self._lib.ram_plan_set_density(self.handle, arr), "ram_plan_set_density")

    def set_wait_limit(self, limit: int = 1 << 20):
        """Tries of every bounded device-side wait (test hook; 0: give up at once,
        so a step on the whole-row kernel records a timeout)."""
        _check(self._lib.ram_plan_set_wait_limit(self.handle, int(limit)),
               "ram_plan_set_wait_limit")

    def check_errors(self) -> int:
        """Synchronise and return (and clear) the device error status (0 = ok)."""
        return int(self._lib.ram_plan_check_errors(self.handle))


def shift(plan: Plan, q_in, q_out, shift_per_row, stream=None):
    """ram_shift: remap every row by +shift[r]."""
    _check_step_args(plan, q_in, q_out, per_row=[("shift", shift_per_row, False)])
    _check(plan._lib.ram_shift(plan.handle, _dtype_code(q_in), _ptr(q_in), _ptr(q_out),
                               _ptr(shift_per_row), _stream(plan.device, stream)),
           "ram_shift")


def residual_upwind(plan: Plan, q_in, q_out, dv, dt: float, scheme: int = VANLEER,
                    nsub=None, stream=None):
    """ram_residual_upwind: nsub upwind sub-steps with the interface velocity dv."""
    _check_step_args(plan, q_in, q_out, nsub=nsub)
    _need(dv, "dv", plan.n_cells, q_in.dtype, _plan_device(plan))
    _check(plan._lib.ram_residual_upwind(plan.handle, _dtype_code(q_in), _ptr(q_in),
                                         _ptr(q_out), _ptr(dv), float(dt), int(scheme),
                                         _ptr(nsub), _stream(plan.device, stream)),
           "ram_residual_upwind")


def step(plan: Plan, q_in, q_out, v0, dt: float, dv=None, scheme: int = VANLEER,
         nsub=None, phase=None, stream=None):
    """ram_step: shift by v0*dt then the residual step (dv=None: no residual)."""
    _check_step_args(plan, q_in, q_out, per_row=[("v0", v0, False), ("phase", phase, True)],
                     dv=dv, nsub=nsub)
    _check(plan._lib.ram_step(plan.handle, _dtype_code(q_in), _ptr(q_in), _ptr(q_out),
                              _ptr(phase), _ptr(v0), float(dt), _ptr(dv), int(scheme),
                              _ptr(nsub), _stream(plan.device, stream)),
           "ram_step")


def step_adjoint(plan: Plan, q_in, g_out, g_in, v0, dt: float, dv=None, g_dv=None,
                 nsub=None, stream=None):
    """ram_step_adjoint: g_in = J^T g_out of the linear step; adds into g_dv."""
    _check_step_args(plan, g_out, g_in, per_row=[("v0", v0, False)], dv=dv, nsub=nsub,
                     extra_cells=[("q_in", q_in, False), ("g_dv", g_dv, True)])
    _check(plan._lib.ram_step_adjoint(plan.handle, _dtype_code(g_out), _ptr(q_in),
                                      _ptr(g_out), _ptr(g_in), _ptr(v0), float(dt),
                                      _ptr(dv), _ptr(g_dv), _ptr(nsub),
                                      _stream(plan.device, stream)),
           "ram_step_adjoint")


def autotune(plan: Plan, q_in, q_out, v0, dt: float, dv=None, scheme: int = VANLEER,
             nsub=None, reps: int = 20, stream=None) -> Tuning:
    """ram_plan_autotune: time the candidate launch shapes on these buffers and keep
    the fastest in the plan."""
    _check_step_args(plan, q_in, q_out, per_row=[("v0", v0, False)], dv=dv, nsub=nsub)
    _check(plan._lib.ram_plan_autotune(plan.handle, _dtype_code(q_in), _ptr(q_in), _ptr(q_out),
                                       _ptr(v0), float(dt), _ptr(dv), int(scheme), _ptr(nsub),
                                       int(reps), _stream(plan.device, stream)),
           "ram_plan_autotune")
    return plan.tuning()


def row_mass(plan: Plan, q, out, stream=None):
    """ram_row_mass: per-row mass (FP64) into out."""
    import torch
    dev = _plan_device(plan)
    _need(q, "q", plan.n_cells, device=dev)
    _dtype_code(q)
    _need(out, "out", plan.n_rows, torch.float64, dev)
    _check(plan._lib.ram_row_mass(plan.handle, _dtype_code(q), _ptr(q), _ptr(out),
                                  _stream(plan.device, stream)), "ram_row_mass")


def step_uniform_noalloc(q_in, q_out, n_rows: int, period: float, order: int, v0, dt: float,
                         dv=None, scheme: int = VANLEER, nsub=None, limiter: bool = True,
                         device_errors=None, stream=None):
    """ram_step_uniform_noalloc: one step of n_rows equal uniform rows without any
    device allocation (the library's static scratch array holds its tables).
    Runs with q_in's device current, on that device's current stream unless
    `stream` is given."""
    import torch
    n_rows = int(n_rows)
    if n_rows < 1:
        raise ValueError("n_rows must be positive")
    if q_in.numel() % n_rows:
        raise ValueError("q_in has %d elements, not a multiple of n_rows = %d"
                         % (q_in.numel(), n_rows))
    n_cells = q_in.numel() // n_rows
    dev = q_in.device
    _dtype_code(q_in)
    _need(q_out, "q_out", q_in.numel(), q_in.dtype, dev)
    _need(v0, "v0", n_rows, torch.float64, dev)
    _need(dv, "dv", q_in.numel(), q_in.dtype, dev, optional=True)
    _need(nsub, "nsub", n_rows, torch.int32, dev, optional=True)
    if device_errors is not None:
        _need(device_errors, "device_errors", 1, torch.int32, dev)
    lib = load()
    with torch.cuda.device(dev):
        _check(lib.ram_step_uniform_noalloc(_dtype_code(q_in), n_rows, int(n_cells),
                                            float(period), int(order),
                                            0 if limiter else LIMITER_OFF, _ptr(q_in),
                                            _ptr(q_out), _ptr(v0), float(dt), _ptr(dv),
                                            int(scheme), _ptr(nsub), _ptr(device_errors),
                                            _stream(dev.index, stream)),
               "ram_step_uniform_noalloc")


def radial_upwind(plan: Plan, q_in, q_out, rf, vr, dt: float, scheme: int = VANLEER,
                  stream=None):
    """ram_radial_upwind: one radial flux-form upwind step of a polar disk whose rings
    are the plan's rows (shared azimuthal mesh); rf: FP64 ring faces (n_rows + 1), vr:
    radial velocity on the faces, (n_rows + 1) x N in q's dtype."""
    import torch
    dev = _plan_device(plan)
    _need(q_in, "q_in", plan.n_cells, device=dev)
    _dtype_code(q_in)
    _need(q_out, "q_out", plan.n_cells, q_in.dtype, dev)
    _need(rf, "rf", plan.n_rows + 1, torch.float64, dev)
    _need(vr, "vr", plan.n_cells + plan.n_cells // plan.n_rows, q_in.dtype, dev)
    _check(plan._lib.ram_radial_upwind(plan.handle, _dtype_code(q_in), _ptr(q_in), _ptr(q_out),
                                       _ptr(rf), _ptr(vr), float(dt), int(scheme),
                                       _stream(plan.device, stream)), "ram_radial_upwind")


def shear_dt(omega, dphi_min: float, beta: float = 0.44) -> float:
    """The shear limit of the split step: the largest dt for which neighbouring rings
    turning at the angular rates omega shear by at most beta times the smallest
    azimuthal cell, beta dphi_min / max |omega_{j+1} - omega_j| (host arithmetic)."""
    om = np.asarray(omega, dtype=np.float64)
    m = float(np.max(np.abs(np.diff(om)))) if om.size > 1 else 0.0
    return beta * float(dphi_min) / m if m > 0.0 else float("inf")


def step_2d(plan: Plan, q_in, q_out, omega, dt: float, rf, vr, dvphi=None,
            scheme: int = VANLEER, nsub=None, scratch=None, phase=None, stream=None):
    """One dimensionally split step of a polar disk (Sec. 3.5): the RAM step of every
    ring (shift by omega dt along the azimuth, residual dvphi), then the radial sweep.
    `scratch` (q's shape and dtype) holds the intermediate field; allocated when
    not given."""
    import torch
    mid = torch.empty_like(q_in) if scratch is None else scratch
    step(plan, q_in, mid, omega, dt, dv=dvphi, scheme=scheme, nsub=nsub, phase=phase,
         stream=stream)
    radial_upwind(plan, mid, q_out, rf, vr, dt, scheme=scheme, stream=stream)


def version() -> int:
    return int(load().ram_version())
