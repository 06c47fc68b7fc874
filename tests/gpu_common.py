"""Helpers shared by the GPU parity tests: run the oracle row by row on the same
inputs and compare per row in relative L1 (sum |a-b| dx / sum |b| dx)."""
import numpy as np

import oracle

TOL = {"float64": 1e-12, "float32": 1e-5}


def rel_l1_rows(w, got, ref):
    """Max over rows of the relative L1 error, weighted by the cell widths."""
    worst = 0.0
    for r in range(w.n_rows):
        sl = w.row_slice(r)
        dx = np.diff(w.row_nodes(r))
        num = float(np.sum(np.abs(got[sl] - ref[sl]) * dx))
        den = float(np.sum(np.abs(ref[sl]) * dx))
        worst = max(worst, num / den if den > 0 else num)
    return worst


def oracle_shifts(w, mode="step", shift=None):
    if mode == "shift":
        return np.asarray(shift, dtype=np.float64)
    return np.array([oracle.shift_from_velocity(v, w.dt) for v in w.v0])


def oracle_step(w, q, shifts, dv=None, nsub=None, rows=None, limiter=None, scheme=None,
                dt=None):
    """Oracle step of every row (or of `rows`), inputs in FP64."""
    q = np.asarray(q, dtype=np.float64)
    out = np.zeros_like(q)
    lim = w.limiter if limiter is None else limiter
    sch = w.scheme if scheme is None else scheme
    dt = w.dt if dt is None else dt
    rows = range(w.n_rows) if rows is None else rows
    for r in rows:
        sl = w.row_slice(r)
        x = w.row_nodes(r)
        d = None if dv is None else np.asarray(dv, dtype=np.float64)[sl]
        ns = 1 if nsub is None else int(nsub[r])
        out[sl] = oracle.step(x, q[sl], float(shifts[r]), int(w.order[r]), lim, d, dt,
                              sch, ns)
    return out
