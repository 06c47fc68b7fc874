"""FP64 CPU oracle for the RAM shift step and the residual upwind step.

TEST INFRASTRUCTURE.  This package is the slow, plain, obviously-correct
reference (plain C in ``ram_oracle.c``, loaded through ctypes) that the CUDA
library is checked against.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA path and the product never calls it.

Every function takes numpy arrays for ONE periodic row:
  x   -- the N+1 nodes x_{-1/2} < ... < x_{N-1/2} (Sec. 2)
  q   -- the N cell values Q_i (cell averages, Eq. 2)
  dv  -- the residual velocity at the N interfaces; dv[j] sits on node x_{j-1/2}
and returns new arrays.  Status codes mirror the C file (0 ok, 1 bad argument,
2 bad mesh, 3 CFL exceeded -- the result is still returned with a flag).
"""
import ctypes
import os

import numpy as np

from . import build as _build

DONOR = 0
VANLEER = 1

_lib = None


class OracleError(RuntimeError):
    pass


def _load():
    global _lib
    if _lib is None:
        # RAM_ORACLE_LIB lets the mutation test load a deliberately broken copy
        path = os.environ.get("RAM_ORACLE_LIB") or _build.build()
        lib = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        lib.oracle_shift.argtypes = [i, d, d, i, i, ctypes.c_double, d]
        lib.oracle_reconstruct.argtypes = [i, d, d, i, i, d]
        lib.oracle_cell_cumulative.argtypes = [i, d, d, i, i, i,
                                               ctypes.POINTER(ctypes.c_int), d, d]
        lib.oracle_residual.argtypes = [i, d, d, d, ctypes.c_double, i, i, d]
        lib.oracle_step.argtypes = [i, d, d, i, i, ctypes.c_double, d,
                                    ctypes.c_double, i, i, d]
        lib.oracle_shift_adjoint.argtypes = [i, d, i, ctypes.c_double, d, d]
        lib.oracle_residual_adjoint_donor.argtypes = [i, d, d, d, ctypes.c_double,
                                                      i, d, d, d]
        lib.oracle_step_adjoint.argtypes = [i, d, d, i, ctypes.c_double, d,
                                            ctypes.c_double, i, d, d, d]
        lib.oracle_shift_from_velocity.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.oracle_shift_from_velocity.restype = ctypes.c_double
        lib.oracle_phase_update.argtypes = [ctypes.c_double] * 4
        lib.oracle_phase_update.restype = ctypes.c_double
        lib.oracle_step_rows.argtypes = [
            i, ctypes.POINTER(ctypes.c_longlong), d, i,
            ctypes.POINTER(ctypes.c_byte), i, d, d, ctypes.c_double, i,
            ctypes.POINTER(ctypes.c_int), d, d]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_radial_upwind.argtypes = [i, i, d, d, d, ctypes.c_double, i, d]
        lib.oracle_shear_dt.argtypes = [i, d, ctypes.c_double, ctypes.c_double]
        lib.oracle_shear_dt.restype = ctypes.c_double
        lib.oracle_step_2d.argtypes = [i, i, d, d, d, d, i, i, d, i,
                                       ctypes.POINTER(ctypes.c_int), d, ctypes.c_double, d]
        lib.oracle_shift_jvp.argtypes = [i, d, d, i, i, ctypes.c_double, d, d]
        lib.oracle_shift_vjp.argtypes = [i, d, d, i, i, ctypes.c_double, d, d]
        lib.oracle_step_adjoint_limited.argtypes = [i, d, d, i, i, ctypes.c_double, d,
                                                    ctypes.c_double, i, d, d, d]
        lib.oracle_a4_average.argtypes = [i, d, d]
        lib.oracle_a4_point.argtypes = [i, d, d]
        lib.oracle_step_a4.argtypes = [i, d, d, i, ctypes.c_double, d, ctypes.c_double, i, i, d]
        _lib = lib
    return _lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(st, allow_cfl=False):
    if st == 0 or (allow_cfl and st == 3):
        return
    raise OracleError("oracle status %d" % st)


def shift(x, q, s, order=2, limiter=True):
    """Remap one periodic row by +s (Eqs. 15-18, 26)."""
    lib = _load()
    x, xp = _f64(x)
    q, qp = _f64(q)
    n = q.size
    assert x.size == n + 1
    out, op = _f64(np.empty(n))
    _check(lib.oracle_shift(n, xp, qp, int(order), int(bool(limiter)), float(s), op))
    return out


def reconstruct(x, q, order=2, limiter=True):
    """Per-cell coefficients: order 2 -> (Q, sigma, 0); order 3 -> (QL, QR, Q6)."""
    lib = _load()
    x, xp = _f64(x)
    q, qp = _f64(q)
    n = q.size
    out, op = _f64(np.empty(3 * n))
    _check(lib.oracle_reconstruct(n, xp, qp, int(order), int(bool(limiter)), op))
    return out.reshape(n, 3)


def cell_cumulative(x, q, cells, d, order=2, limiter=True):
    """G_i(d): integral of q_i over [x_{i-1/2}, x_{i-1/2} + d]."""
    lib = _load()
    x, xp = _f64(x)
    q, qp = _f64(q)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    d, dp = _f64(d)
    out, op = _f64(np.empty(cells.size))
    _check(lib.oracle_cell_cumulative(
        q.size, xp, qp, int(order), int(bool(limiter)), cells.size,
        cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), dp, op))
    return out


def residual(x, q, dv, dt, scheme=VANLEER, nsub=1, return_status=False):
    """Residual upwind step with the interface velocity dv (Eq. 6)."""
    lib = _load()
    x, xp = _f64(x)
    q, qp = _f64(q)
    dv, dvp = _f64(dv)
    out, op = _f64(np.empty(q.size))
    st = lib.oracle_residual(q.size, xp, qp, dvp, float(dt), int(scheme), int(nsub), op)
    _check(st, allow_cfl=True)
    return (out, st) if return_status else out


def step(x, q, s, order=2, limiter=True, dv=None, dt=0.0, scheme=VANLEER, nsub=1,
         return_status=False):
    """One RAM step: shift by s, then the residual step (Eqs. 5-6)."""
    lib = _load()
    x, xp = _f64(x)
    q, qp = _f64(q)
    if dv is None:
        dvp = None
    else:
        dv, dvp = _f64(dv)
    out, op = _f64(np.empty(q.size))
    st = lib.oracle_step(q.size, xp, qp, int(order), int(bool(limiter)), float(s), dvp,
                         float(dt), int(scheme), int(nsub), op)
    _check(st, allow_cfl=True)
    return (out, st) if return_status else out


def shift_adjoint(x, g_out, s, order=2):
    """Transpose of the limiter-off shift."""
    lib = _load()
    x, xp = _f64(x)
    g, gp = _f64(g_out)
    out, op = _f64(np.empty(g.size))
    _check(lib.oracle_shift_adjoint(g.size, xp, int(order), float(s), gp, op))
    return out


def residual_adjoint_donor(x, q_in, dv, dt, g_out, nsub=1):
    """Transpose of the donor residual step; returns (g_in, g_dv)."""
    lib = _load()
    x, xp = _f64(x)
    q, qp = _f64(q_in)
    dv, dvp = _f64(dv)
    g, gp = _f64(g_out)
    gi, gip = _f64(np.empty(q.size))
    gdv, gdvp = _f64(np.zeros(q.size))
    _check(lib.oracle_residual_adjoint_donor(q.size, xp, qp, dvp, float(dt), int(nsub),
                                             gp, gip, gdvp))
    return gi, gdv


def step_adjoint(x, q_in, g_out, s, order=2, dv=None, dt=0.0, nsub=1):
    """Transpose of one linear step (limiter-off shift, donor residual).
    Returns (g_in, g_dv); g_dv is None when dv is None."""
    lib = _load()
    x, xp = _f64(x)
    q, qp = _f64(q_in)
    g, gp = _f64(g_out)
    gi, gip = _f64(np.empty(q.size))
    if dv is None:
        dvp = None
        gdv, gdvp = None, None
    else:
        dv, dvp = _f64(dv)
        gdv, gdvp = _f64(np.zeros(q.size))
    _check(lib.oracle_step_adjoint(q.size, xp, qp, int(order), float(s), dvp, float(dt),
                                   int(nsub), gp, gip, gdvp))
    return gi, gdv


def shift_from_velocity(v0, dt):
    return _load().oracle_shift_from_velocity(float(v0), float(dt))


def phase_update(phase, v0, dt, L):
    return _load().oracle_phase_update(float(phase), float(v0), float(dt), float(L))


def step_rows(row_offset, nodes, shared_mesh, order, limiter, shift_per_row, q_in,
              dv=None, dt=0.0, scheme=VANLEER, nsub=None):
    """Batched oracle step over packed rows (OpenMP over rows when available)."""
    lib = _load()
    ro = np.ascontiguousarray(row_offset, dtype=np.int64)
    n_rows = ro.size - 1
    nodes, np_ = _f64(nodes)
    order = np.ascontiguousarray(np.broadcast_to(order, (n_rows,)), dtype=np.int8)
    sh, shp = _f64(shift_per_row)
    q, qp = _f64(q_in)
    out, op = _f64(np.empty(q.size))
    if dv is None:
        dvp = None
    else:
        dv, dvp = _f64(dv)
    if nsub is None:
        nsp = None
    else:
        nsub = np.ascontiguousarray(nsub, dtype=np.int32)
        nsp = nsub.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    st = lib.oracle_step_rows(
        n_rows, ro.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), np_,
        int(bool(shared_mesh)), order.ctypes.data_as(ctypes.POINTER(ctypes.c_byte)),
        int(bool(limiter)), shp, dvp, float(dt), int(scheme), nsp, qp, op)
    _check(st, allow_cfl=True)
    return out


def a4_average(q):
    """Fourth-order cell averages from point values (Sec. 3.1), periodic."""
    lib = _load()
    q, qp = _f64(q)
    out, op = _f64(np.empty(q.size))
    _check(lib.oracle_a4_average(q.size, qp, op))
    return out


def a4_point(avg):
    """Point values whose fourth-order cell averages are `avg` (periodic solve)."""
    lib = _load()
    a, ap = _f64(avg)
    out, op = _f64(np.empty(a.size))
    _check(lib.oracle_a4_point(a.size, ap, op))
    return out


def step_a4(x, q, s, limiter=True, dv=None, dt=0.0, scheme=VANLEER, nsub=1,
            return_status=False):
    """One RAM step with the A4 correction: PPM remap of the corrected averages,
    point values recovered, then the residual step."""
    lib = _load()
    x, xp = _f64(x)
    q, qp = _f64(q)
    if dv is None:
        dvp = None
    else:
        dv, dvp = _f64(dv)
    out, op = _f64(np.empty(q.size))
    st = lib.oracle_step_a4(q.size, xp, qp, int(bool(limiter)), float(s), dvp, float(dt),
                            int(scheme), int(nsub), op)
    _check(st, allow_cfl=True)
    return (out, st) if return_status else out


def radial_upwind(rf, q, vr, dt, scheme=VANLEER, return_status=False):
    """Radial sweep of a polar disk (cylindrical geometry, closed ends): q and vr are
    (rings, phi cells) and (rings + 1, phi cells) arrays, rf the ring face radii."""
    lib = _load()
    rf, rfp = _f64(rf)
    q = np.ascontiguousarray(q, dtype=np.float64)
    nr, nphi = q.shape
    assert rf.size == nr + 1
    vr = np.ascontiguousarray(vr, dtype=np.float64)
    assert vr.shape == (nr + 1, nphi)
    out = np.empty_like(q)
    d = ctypes.POINTER(ctypes.c_double)
    st = lib.oracle_radial_upwind(nr, nphi, rfp, q.ctypes.data_as(d), vr.ctypes.data_as(d),
                                  float(dt), int(scheme), out.ctypes.data_as(d))
    _check(st, allow_cfl=True)
    return (out, st) if return_status else out


def shear_dt(omega, dphi_min, beta):
    """The shear limit of the split step: beta dphi_min / max |omega_{j+1} - omega_j|."""
    lib = _load()
    om, omp = _f64(omega)
    return lib.oracle_shear_dt(om.size, omp, float(dphi_min), float(beta))


def step_2d(phi, rf, omega, q, dt, order=3, limiter=True, dvphi=None, scheme=VANLEER,
            nsub=None, vr=None):
    """One split step of a polar disk: RAM in phi on every ring, then the radial
    sweep (q: (rings, phi cells))."""
    lib = _load()
    phi, phip = _f64(phi)
    rf, rfp = _f64(rf)
    om, omp = _f64(omega)
    q = np.ascontiguousarray(q, dtype=np.float64)
    nr, nphi = q.shape
    d = ctypes.POINTER(ctypes.c_double)
    dvp = None
    if dvphi is not None:
        dvphi = np.ascontiguousarray(dvphi, dtype=np.float64)
        dvp = dvphi.ctypes.data_as(d)
    nsp = None
    if nsub is not None:
        nsub = np.ascontiguousarray(nsub, dtype=np.int32)
        nsp = nsub.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    vr = np.zeros((nr + 1, nphi)) if vr is None else np.ascontiguousarray(vr, dtype=np.float64)
    out = np.empty_like(q)
    st = lib.oracle_step_2d(nr, nphi, phip, rfp, omp, q.ctypes.data_as(d), int(order),
                            int(bool(limiter)), dvp, int(scheme), nsp, vr.ctypes.data_as(d),
                            float(dt), out.ctypes.data_as(d))
    _check(st, allow_cfl=True)
    return out


def shift_jvp(x, q0, v, s, order=3, limiter=True):
    """The shift's derivative at q0 along v (the limiters' branches as q0 decides)."""
    lib = _load()
    x, xp = _f64(x)
    q0, qp = _f64(q0)
    v, vp = _f64(v)
    out, op = _f64(np.empty(q0.size))
    _check(lib.oracle_shift_jvp(q0.size, xp, qp, int(order), int(bool(limiter)), float(s), vp, op))
    return out


def shift_vjp(x, q0, g, s, order=3, limiter=True):
    """The transpose of shift_jvp applied to g (small rows: one tangent per cell)."""
    lib = _load()
    x, xp = _f64(x)
    q0, qp = _f64(q0)
    g, gp = _f64(g)
    out, op = _f64(np.empty(q0.size))
    _check(lib.oracle_shift_vjp(q0.size, xp, qp, int(order), int(bool(limiter)), float(s), gp, op))
    return out


def step_adjoint_limited(x, q_in, g_out, s, order=3, limiter=True, dv=None, dt=0.0, nsub=1):
    """Transpose of the step linearised at q_in (PLM / PPM shift, donor residual);
    returns (g_in, g_dv)."""
    lib = _load()
    x, xp = _f64(x)
    q, qp = _f64(q_in)
    g, gp = _f64(g_out)
    gi, gip = _f64(np.empty(q.size))
    if dv is None:
        dvp = None
        gdv, gdvp = None, None
    else:
        dv, dvp = _f64(dv)
        gdv, gdvp = _f64(np.zeros(q.size))
    _check(lib.oracle_step_adjoint_limited(q.size, xp, qp, int(order), int(bool(limiter)),
                                           float(s), dvp, float(dt), int(nsub), gp, gip, gdvp))
    return gi, gdv


def num_threads():
    return _load().oracle_num_threads()


def mass(x, q):
    """Total mass sum_i Q_i dx_i (Eq. 10), summed with math.fsum."""
    import math
    x = np.asarray(x, dtype=np.float64)
    return math.fsum((np.asarray(q, dtype=np.float64) * np.diff(x)).tolist())


__all__ = ["shift", "reconstruct", "cell_cumulative", "residual", "step",
           "shift_adjoint", "residual_adjoint_donor", "step_adjoint",
           "shift_from_velocity", "phase_update", "step_rows", "num_threads", "mass",
           "a4_average", "a4_point", "step_a4", "radial_upwind", "shear_dt", "step_2d",
           "shift_jvp", "shift_vjp", "step_adjoint_limited",
           "DONOR", "VANLEER", "OracleError"]
