"""ctypes front end of the FP64 CPU oracle (``pf_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark call this module; the product library never does.  It shares
no code with the CUDA path.  ``build()`` compiles the C file with gcc into
``oracle/_build/liboracle.so``; every call below marshals numpy arrays and
forwards to the C function of the same name.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

S10, S21, SBAR21, S100, SBAR120 = 0, 1, 2, 3, 4
T1, T0 = 0, 1
BC_MIRROR, BC_PERIODIC, BC_PERIODIC_X = 0, 1, 2

OPS = {
    "lap_10": 0, "lap_01": 1, "lap_21": 2, "grad2_10": 3, "grad2_01": 4, "grad2_21": 5,
    "div_10": 6, "div_01": 7, "div_21": 8, "div_std2": 9, "at_std2": 10, "at_21": 11,
    "lap_100": 20, "lap_010": 21, "lap_001": 22, "lap_120": 23,
    "grad2_100": 24, "grad2_010": 25, "grad2_001": 26, "grad2_120": 27,
    "div_100": 28, "div_010": 29, "div_001": 30, "div_120": 31, "div_std3": 32, "at_std3": 33,
    "aniso_n": 40,
}


class Params(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("scheme", C.c_int), ("bc", C.c_int),
                ("h", C.c_double), ("dt", C.c_double), ("k", C.c_double), ("eps4", C.c_double),
                ("lam", C.c_double), ("D", C.c_double),
                ("thermal", C.c_int), ("time_level", C.c_int),
                ("Vp", C.c_double), ("lT", C.c_double), ("yT", C.c_double), ("t0", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP rows).
    The ORACLE_LIB environment variable names a prebuilt library to use
    instead (the mutation tests point it at deliberately broken builds)."""
    if os.environ.get("ORACLE_LIB"):
        return os.environ["ORACLE_LIB"]
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.or_step.argtypes = [C.POINTER(Params), C.c_int, dp, C.POINTER(C.c_int16), dp, dp, C.c_long, dp]
            L.or_apply.argtypes = [C.POINTER(Params), C.c_int, dp, dp, dp, dp]
            L.or_init_seeds.argtypes = [C.POINTER(Params), C.c_double, C.c_int, dp, C.POINTER(C.c_int16),
                                        dp, dp, C.POINTER(C.c_int16)]
            L.or_observe.argtypes = [C.POINTER(Params), C.c_int, dp, dp, C.POINTER(C.c_int16), dp, dp, C.c_int, dp]
            L.or_aniso.argtypes = [C.c_int, dp, C.c_double, dp, C.c_double, C.c_double, dp]
            L.or_aniso.restype = C.c_double
            L.or_appb_grad.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, dp]
            L.or_dt_max.argtypes = [C.POINTER(Params)]
            L.or_dt_max.restype = C.c_double
            L.or_set_at21_floor.argtypes = [C.c_int]
            L.or_set_at21_floor.restype = C.c_int
            L.or_tip_radius.argtypes = [C.POINTER(Params), dp, dp, dp, dp]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i16(a):
    return a.ctypes.data_as(C.POINTER(C.c_int16))


def params(dim=2, nx=16, ny=16, nz=1, scheme=SBAR21, bc=BC_MIRROR, h=0.8, dt=0.02, k=0.15, eps4=0.02,
           lam=10.0, D=None, thermal=0, Vp=0.0, lT=1.0, yT=0.0, t0=0.0, time_level=0) -> Params:
    """Oracle parameters; thermal=1 selects the frozen temperature along +y
    (zeta = (y - yT - Vp t) / lT, t = t0 + step * dt); time_level=1 selects
    T0 (pure forward Euler of Eq. PF_b) instead of T1."""
    if D is None:
        D = 0.6267 * lam
    return Params(dim, nx, ny, nz if dim == 3 else 1, scheme, bc, h, dt, k, eps4, lam, D, int(thermal),
                  int(time_level), Vp, lT, yT, t0)


def _shape(p: Params):
    return (p.nz, p.ny, p.nx) if p.dim == 3 else (p.ny, p.nx)


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == shape, (a.shape, shape)
    return a


def step(p: Params, rot, grain, psi, U, nsteps=1, want_rate=False):
    """Advance copies of psi, U by nsteps steps; returns (psi, U[, dpsi/dt of the last step])."""
    shape = _shape(p)
    psi = _f64(psi, shape).copy()
    U = _f64(U, shape).copy()
    grain = np.ascontiguousarray(grain, dtype=np.int16).reshape(shape)
    rot = np.ascontiguousarray(rot, dtype=np.float64).reshape(-1, 9)
    rate = np.zeros(shape) if want_rate else None
    rc = lib().or_step(C.byref(p), rot.shape[0], _dp(rot), _i16(grain), _dp(psi), _dp(U), int(nsteps),
                       _dp(rate) if want_rate else None)
    if rc != 0:
        raise ValueError(f"or_step failed: {rc}")
    return (psi, U, rate) if want_rate else (psi, U)


# Three-shell 3D combinations T_{s1,s2,s3} (Eq. tau_3D): the weights (s1, s2, s3)
# of the <100>, <110> and <111> base discretizations, normalised by their sum.
# Sec. 6.1 names these as the isotropic solutions of Eqs. Constrain_Lap1/2 (L),
# Constrain_Div1/2 (D~) and the App. A constraints (G); "m1" spells the weight -1
# of T_{0,4,-1}.  The paper runs no simulation with a <111> shell (Sec. 6.2.1,
# pinning), so these serve the symbol pins only.
COMBOS3 = {"120": (1, 2, 0), "201": (2, 0, 1), "04m1": (0, 4, -1), "441": (4, 4, 1), "561": (5, 6, 1),
           "762": (7, 6, 2)}
_SHELLS3 = ("100", "010", "001")


def apply_combo(p: Params, fam: str, weights, a, b=None):
    """T_{s1,s2,s3} of Eq. tau_3D for fam in {"lap", "div", "grad2"}: the
    weighted mean of the three 3D base operators (each from the C oracle)."""
    if fam not in ("lap", "div", "grad2") or len(weights) != 3 or sum(weights) == 0:
        raise ValueError(f"bad combination {fam} {weights}")
    tot = float(sum(weights))
    out = np.zeros(_shape(p))
    for w, sh in zip(weights, _SHELLS3):
        if w != 0:
            out += (w / tot) * apply(p, f"{fam}_{sh}", a, b)
    return out


def apply(p: Params, op: str, a, b=None, rot=None):
    """Evaluate one operator at every cell (boundary rule of p).  Besides the C
    oracle's operators, op may name a three-shell combination "<fam>_c<key>"
    with key in COMBOS3 (e.g. "lap_c441")."""
    fam, _, key = op.partition("_c")
    if key in COMBOS3 and op not in OPS:
        return apply_combo(p, fam, COMBOS3[key], a, b)
    shape = _shape(p)
    a = _f64(a, shape)
    b = _f64(b, shape) if b is not None else None
    r = np.ascontiguousarray(rot if rot is not None else np.eye(3), dtype=np.float64).reshape(9)
    out = np.zeros(shape)
    rc = lib().or_apply(C.byref(p), OPS[op], _dp(a), _dp(b) if b is not None else None, _dp(r), _dp(out))
    if rc != 0:
        raise ValueError(f"or_apply failed: {rc}")
    return out


def init_seeds(p: Params, U0, seeds, seed_grain):
    """Initial psi, U, grain from seeds = array (n, 4) of (x, y, z, r)."""
    shape = _shape(p)
    seeds = np.ascontiguousarray(seeds, dtype=np.float64).reshape(-1, 4)
    sg = np.ascontiguousarray(seed_grain, dtype=np.int16).reshape(-1)
    psi = np.zeros(shape)
    U = np.zeros(shape)
    g = np.zeros(shape, np.int16)
    rc = lib().or_init_seeds(C.byref(p), float(U0), seeds.shape[0], _dp(seeds), _i16(sg), _dp(psi), _dp(U), _i16(g))
    if rc != 0:
        raise ValueError(f"or_init_seeds failed: {rc}")
    return psi, U, g


OBS_KEYS = ("tip_x", "tip_y", "tip_z", "score", "solute", "solid_fraction", "nonfinite", "found", "tip_index",
            "angle_xy_deg", "angle_out_deg")


def observe(p: Params, rot, centres, grain, psi, U, g=-1):
    shape = _shape(p)
    rot = np.ascontiguousarray(rot, dtype=np.float64).reshape(-1, 9)
    centres = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
    grain = np.ascontiguousarray(grain, dtype=np.int16).reshape(shape)
    out = np.zeros(11)
    rc = lib().or_observe(C.byref(p), rot.shape[0], _dp(rot), _dp(centres), _i16(grain), _dp(_f64(psi, shape)),
                          _dp(_f64(U, shape)), int(g), _dp(out))
    if rc != 0:
        raise ValueError(f"or_observe failed: {rc}")
    return dict(zip(OBS_KEYS, out.tolist()))


def aniso(dim, rot, eps4, g, h=1.0, guard2=1e-20):
    """Returns (a_s, J - g) for one lab-frame gradient g."""
    r = np.ascontiguousarray(rot, dtype=np.float64).reshape(9)
    gv = np.zeros(3)
    gv[: len(g)] = g
    out = np.zeros(3)
    a = lib().or_aniso(int(dim), _dp(r), float(eps4), _dp(gv), float(h), float(guard2), _dp(out))
    return a, out


def appb_grad(field, i, j, kind, h=1.0):
    """App. B derivative pair at (i+1/2, j) [kind 0], (i, j+1/2) [kind 1] or (i+1/2, j+1/2) [kind 2]."""
    f = np.ascontiguousarray(field, dtype=np.float64)
    ny, nx = f.shape
    out = np.zeros(2)
    rc = lib().or_appb_grad(_dp(f), nx, ny, int(i), int(j), int(kind), float(h), _dp(out))
    if rc != 0:
        raise ValueError("or_appb_grad failed")
    return out


def dt_max(p: Params) -> float:
    return float(lib().or_dt_max(C.byref(p)))


def set_at21_floor(on: bool) -> bool:
    """Turn the magnitude floor of A_{2,1} (reading R-A21G) on or off; returns
    the previous setting.  Off reproduces App. B's form without the floor, for
    tests that show why the floor is there."""
    return bool(lib().or_set_at21_floor(1 if on else 0))


def tip_radius(p: Params, psi, tip, axis):
    """Tip radius by the parabola fit of the psi = 0 contour (reading R-RHO):
    returns dict(rho, rho_x, rho_z, n_x, n_z); rho_z is NaN in 2D."""
    shape = _shape(p)
    t = np.zeros(3)
    t[: len(tip)] = tip
    a = np.zeros(3)
    a[: len(axis)] = axis
    out = np.zeros(5)
    rc = lib().or_tip_radius(C.byref(p), _dp(_f64(psi, shape)), _dp(t), _dp(a), _dp(out))
    if rc != 0:
        raise ValueError("or_tip_radius failed")
    return dict(rho=out[0], rho_x=out[1], rho_z=out[2], n_x=int(out[3]), n_z=int(out[4]))
