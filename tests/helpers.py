"""Shared test helpers: build matching oracle parameters for a workload and
run both sides on the same seeded inputs."""
import numpy as np

from oracle import oracle as O
from paper_2110_12448_gb300 import synth


def oracle_params(w, scheme=None, bc=None, step=0, **over):
    """Oracle parameters of workload w (walls, frozen temperature) for a call
    that starts at time step `step` of the simulation."""
    if bc is None:
        bc = O.BC_PERIODIC_X if getattr(w, "bc_x", 0) else O.BC_MIRROR
    d = dict(dim=w.dim, nx=w.nx, ny=w.ny, nz=w.nz, scheme=synth.SCHEMES[scheme or w.scheme],
             bc=bc, h=w.h, dt=w.dt, k=w.k, eps4=w.eps4, lam=w.lam, D=w.D,
             thermal=getattr(w, "thermal", 0), Vp=getattr(w, "Vp", 0.0), lT=getattr(w, "lT", 1.0),
             yT=getattr(w, "yT", 0.0), t0=step * w.dt)
    d.update(over)
    return O.params(**d)


def small_workload(dim, nx, ny, nz=1, scheme=None, **phys):
    if dim == 2:
        w = synth.free_dendrite_2d(nx, ny=ny, scheme=scheme or "SBAR21", **phys)
    else:
        w = synth.free_dendrite_3d(nx, scheme=scheme or "SBAR120", **phys)
        w.ny, w.nz = ny, nz
    return w


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))))
