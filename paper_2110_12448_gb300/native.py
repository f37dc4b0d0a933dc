"""ctypes binding of ``libpf.so`` (the C-ABI declared in ``include/pf.h``).

Argument marshalling only: every step of the path runs in the library's
CUDA kernels.  PyTorch supplies the device buffers (``torch.empty`` of
``pf_required_bytes``) and the stream.  There is no CPU fallback: if the
library is missing, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

SCHEMES = {"S10": 0, "S21": 1, "SBAR21": 2, "S100": 3, "SBAR120": 4}
PRECISIONS = {"f32": 0, "f64": 1, "f32c": 2}  # f32c: FP32 arithmetic on a compensated (hi + lo) state
PF_OK, PF_ERR_INVALID, PF_ERR_BUDGET, PF_ERR_CUDA, PF_ERR_NONFINITE, PF_ERR_TIMEOUT, PF_ERR_STATE = 0, -1, -2, -3, -4, -5, -6


class PfError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {code} ({status_string(code)})"
        if code == PF_ERR_CUDA:
            msg += f" [{lib().pf_last_cuda_error().decode()}]"
        super().__init__(msg)


class Params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("h", C.c_double), ("dt", C.c_double), ("k", C.c_double), ("eps4", C.c_double),
                ("lam", C.c_double), ("D", C.c_double), ("U0", C.c_double),
                ("scheme", C.c_int32), ("precision", C.c_int32), ("max_grains", C.c_int32),
                ("max_seeds", C.c_int32), ("bc_x", C.c_int32), ("thermal", C.c_int32),
                ("Vp", C.c_double), ("lT", C.c_double), ("yT", C.c_double),
                ("time_level", C.c_int32), ("kernels", C.c_int32)]


PF_BC_MIRROR, PF_BC_PERIODIC = 0, 1
PF_ISOTHERMAL, PF_FROZEN_GRADIENT = 0, 1
PF_T1, PF_T0 = 0, 1
PF_FUSED, PF_TWO_KERNELS = 0, 1


class Seed(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("z", C.c_double), ("r", C.c_double),
                ("grain", C.c_int32), ("reserved", C.c_int32)]


class Obs(C.Structure):
    _fields_ = [("step", C.c_int64), ("t", C.c_double), ("tip", C.c_double * 3), ("v_tip", C.c_double),
                ("angle_xy_deg", C.c_double), ("angle_out_deg", C.c_double), ("solute", C.c_double),
                ("solid_fraction", C.c_double), ("tip_score", C.c_double), ("tip_index", C.c_int64),
                ("found", C.c_int32), ("nonfinite", C.c_int32)]


class Tip(C.Structure):
    _fields_ = [("rho", C.c_double), ("rho_x", C.c_double), ("rho_z", C.c_double), ("sigma_star", C.c_double),
                ("d0_star", C.c_double), ("axis", C.c_double * 3), ("n_x", C.c_int32), ("n_z", C.c_int32)]


def lib_path() -> str:
    """Path of libpf.so; the PF_LIBRARY environment variable overrides it."""
    return os.environ.get("PF_LIBRARY", _build.LIB)


def lib():
    """Load libpf.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("PF_LIBRARY") or _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libpf.so missing at {path}: the CUDA library is required (no CPU fallback)")
            L = C.CDLL(path)
            vp, i64 = C.c_void_p, C.c_int64
            P = C.POINTER
            sig = {
                "pf_required_bytes": (C.c_size_t, [P(Params)]),
                "pf_create": (C.c_int, [P(Params), vp, C.c_size_t, vp, P(vp)]),
                "pf_set_grains": (C.c_int, [vp, C.c_int, P(C.c_double), P(C.c_double)]),
                "pf_init_seeds": (C.c_int, [vp, C.c_int, P(Seed)]),
                "pf_set_grain_index": (C.c_int, [vp, P(C.c_int16)]),
                "pf_get_grain_index": (C.c_int, [vp, P(C.c_int16)]),
                "pf_step": (C.c_int, [vp, i64]),
                "pf_observe": (C.c_int, [vp, C.c_int, P(Obs)]),
                "pf_tip_radius": (C.c_int, [vp, C.c_int, P(C.c_double), C.c_double, P(Tip)]),
                "pf_get_fields": (C.c_int, [vp, vp, vp]),
                "pf_set_fields": (C.c_int, [vp, vp, vp]),
                "pf_get_fields_async": (C.c_int, [vp, vp, vp]),
                "pf_set_fields_async": (C.c_int, [vp, vp, vp]),
                "pf_synchronize": (C.c_int, [vp]),
                "pf_get_step": (C.c_int, [vp, P(i64)]),
                "pf_set_step": (C.c_int, [vp, i64]),
                "pf_shift_frame": (C.c_int, [vp, C.c_int]),
                "pf_device_fields": (C.c_int, [vp, P(vp), P(vp), P(vp)]),
                "pf_set_tile": (C.c_int, [vp, C.c_int, C.c_int, C.c_int]),
                "pf_get_tile": (C.c_int, [vp, P(C.c_int), P(C.c_int), P(C.c_int)]),
                "pf_resident_units": (C.c_int, [vp]),
                "pf_debug_bounds": (C.c_int, [P(C.c_uint64), P(C.c_int)]),
                "pf_debug_inject_launch_failure": (C.c_int, [C.c_longlong]),
                "pf_destroy": (C.c_int, [vp]),
                "pf_status_string": (C.c_char_p, [C.c_int]),
                "pf_last_cuda_error": (C.c_char_p, []),
                "pf_group_required_bytes": (C.c_size_t, [C.c_int, C.c_int]),
                "pf_group_work_items": (C.c_int, [vp]),
                "pf_group_create": (C.c_int, [C.c_int, C.c_int, vp, C.c_size_t, vp, P(vp)]),
                "pf_group_add": (C.c_int, [vp, vp]),
                "pf_group_remove": (C.c_int, [vp, vp]),
                "pf_group_step": (C.c_int, [vp, i64, C.c_int]),
                "pf_group_size": (C.c_int, [vp]),
                "pf_group_observe": (C.c_int, [vp, C.c_int, vp]),
                "pf_group_destroy": (C.c_int, [vp]),
                "pf_group_set_depth": (C.c_int, [vp, C.c_int, C.c_int]),
                "pf_group_get_depth": (C.c_int, [vp, P(C.c_int), P(C.c_int), P(C.c_int)]),
                "pf_wavefront_order": (C.c_int, [C.c_int, P(C.c_int), P(C.c_int), C.c_int]),
                "pf_observe_fields_noalloc": (C.c_int, [P(Params), vp, vp, vp, P(C.c_double), P(C.c_double), C.c_int,
                                                        vp, P(Obs)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def debug_bounds():
    """(failures, first source line) of a bounds-checked build; None in a
    build without the checks."""
    n, line = C.c_uint64(), C.c_int()
    rc = lib().pf_debug_bounds(C.byref(n), C.byref(line))
    if rc == PF_ERR_STATE:
        return None
    _check(rc, "pf_debug_bounds")
    return n.value, line.value


def inject_launch_failure(after_steps: int):
    """Arm (>= 0) or disarm (< 0) the host-side injected launch failure."""
    _check(lib().pf_debug_inject_launch_failure(int(after_steps)), "pf_debug_inject_launch_failure")


def status_string(code: int) -> str:
    return lib().pf_status_string(int(code)).decode()


def _check(rc: int, what: str):
    if rc != PF_OK:
        raise PfError(rc, what)


def make_params(dim, nx, ny, nz=1, h=0.8, dt=0.02, k=0.15, eps4=0.02, lam=10.0, D=None, U0=-0.55,
                scheme="SBAR21", precision="f32", max_grains=1, max_seeds=0, bc_x=PF_BC_MIRROR,
                thermal=PF_ISOTHERMAL, Vp=0.0, lT=1.0, yT=0.0, time_level=PF_T1, kernels=PF_FUSED) -> Params:
    if D is None:
        D = 0.6267 * lam
    return Params(int(dim), int(nx), int(ny), int(nz if dim == 3 else 1), float(h), float(dt), float(k), float(eps4),
                  float(lam), float(D), float(U0), SCHEMES[scheme] if isinstance(scheme, str) else int(scheme),
                  PRECISIONS[precision] if isinstance(precision, str) else int(precision), int(max_grains),
                  int(max_seeds), int(bc_x), int(thermal), float(Vp), float(lT), float(yT), int(time_level),
                  int(kernels))


def required_bytes(p: Params) -> int:
    return int(lib().pf_required_bytes(C.byref(p)))


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return int(getattr(stream, "cuda_stream", stream) or 0)


class Sim:
    """One simulation on caller-owned (torch) device memory."""

    def __init__(self, p: Params, stream=None, device="cuda"):
        import torch
        self.p = p
        self.np_dtype = np.float32 if p.precision == 0 else np.float64  # f32c: the host sees FP64 fields
        n = required_bytes(p)
        if n == 0:
            raise PfError(PF_ERR_INVALID, "pf_required_bytes")
        self.nbytes = n
        self.mem = torch.empty(n, dtype=torch.uint8, device=device)
        self.stream = stream
        self._st = _stream_handle(stream)
        h = C.c_void_p()
        _check(lib().pf_create(C.byref(p), C.c_void_p(self.mem.data_ptr()), n, C.c_void_p(self._st), C.byref(h)),
               "pf_create")
        self.h = h
        self.shape = (p.nz, p.ny, p.nx) if p.dim == 3 else (p.ny, p.nx)

    @classmethod
    def from_workload(cls, w, precision="f32", scheme=None, stream=None, init=True):
        p = make_params(w.dim, w.nx, w.ny, w.nz, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, scheme or w.scheme,
                        precision, max_grains=max(1, w.n_grains), max_seeds=max(1, len(w.seeds)),
                        bc_x=getattr(w, "bc_x", 0), thermal=getattr(w, "thermal", 0), Vp=getattr(w, "Vp", 0.0),
                        lT=getattr(w, "lT", 1.0), yT=getattr(w, "yT", 0.0), time_level=getattr(w, "time_level", 0),
                        kernels=getattr(w, "kernels", 0))
        s = cls(p, stream=stream)
        s.set_grains(w.rots, w.centres)
        if init:
            s.init_seeds(w.seeds, w.seed_grain)
            if getattr(w, "psi_init", None) is not None:
                s.set_fields(w.psi_init, w.U_init)
        return s

    # -- configuration -------------------------------------------------
    def set_grains(self, rots, centres=None):
        r = np.ascontiguousarray(rots, dtype=np.float64).reshape(-1, 9)
        c = None if centres is None else np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
        _check(lib().pf_set_grains(self.h, r.shape[0], r.ctypes.data_as(C.POINTER(C.c_double)),
                                   None if c is None else c.ctypes.data_as(C.POINTER(C.c_double))), "pf_set_grains")

    def init_seeds(self, seeds, seed_grain):
        s = np.asarray(seeds, dtype=np.float64).reshape(-1, 4)
        g = np.asarray(seed_grain).reshape(-1)
        arr = (Seed * len(s))()
        for i in range(len(s)):
            arr[i] = Seed(s[i, 0], s[i, 1], s[i, 2], s[i, 3], int(g[i]), 0)
        _check(lib().pf_init_seeds(self.h, len(s), arr), "pf_init_seeds")

    def set_grain_index(self, g):
        g = np.ascontiguousarray(g, dtype=np.int16).reshape(self.shape)
        _check(lib().pf_set_grain_index(self.h, g.ctypes.data_as(C.POINTER(C.c_int16))), "pf_set_grain_index")

    def get_grain_index(self):
        g = np.zeros(self.shape, np.int16)
        _check(lib().pf_get_grain_index(self.h, g.ctypes.data_as(C.POINTER(C.c_int16))), "pf_get_grain_index")
        return g

    def set_tile(self, bx=0, by=0, sweep=0):
        _check(lib().pf_set_tile(self.h, int(bx), int(by), int(sweep)), "pf_set_tile")

    def resident_units(self) -> int:
        """Warps (2D) or blocks (3D) of the current tile resident at once."""
        n = lib().pf_resident_units(self.h)
        _check(min(n, 0), "pf_resident_units")
        return n

    def get_tile(self):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        _check(lib().pf_get_tile(self.h, C.byref(a), C.byref(b), C.byref(c)), "pf_get_tile")
        return a.value, b.value, c.value

    # -- stepping and observation --------------------------------------
    def step(self, n: int = 1):
        _check(lib().pf_step(self.h, int(n)), "pf_step")

    def observe(self, grain: int = -1, allow_nonfinite=False) -> dict:
        o = Obs()
        rc = lib().pf_observe(self.h, int(grain), C.byref(o))
        if rc != PF_OK and not (allow_nonfinite and rc == PF_ERR_NONFINITE):
            raise PfError(rc, "pf_observe")
        d = {f: getattr(o, f) for f, _ in Obs._fields_}
        d["tip"] = tuple(o.tip)
        d["status"] = rc
        return d

    def tip_radius(self, obs: dict, grain: int = -1) -> dict:
        """pf_tip_radius at the tip of an observe() result of the same grain:
        tip radius, its fits, sigma* (with the observed tip velocity)."""
        t = (C.c_double * 3)(*obs["tip"])
        o = Tip()
        _check(lib().pf_tip_radius(self.h, int(grain), t, float(obs.get("v_tip", 0.0)), C.byref(o)), "pf_tip_radius")
        d = {f: getattr(o, f) for f, _ in Tip._fields_}
        d["axis"] = tuple(o.axis)
        return d

    def get_fields(self, out=None):
        """Copy of the current psi, U.  `out` = (psi, U) writes into caller
        arrays instead (C-contiguous, the handle's shape and dtype), e.g. views
        of pinned host tensors, which the copy reaches at full link speed."""
        if out is None:
            psi = np.zeros(self.shape, self.np_dtype)
            U = np.zeros(self.shape, self.np_dtype)
        else:
            psi, U = out
            for a in (psi, U):
                if a.shape != tuple(self.shape) or a.dtype != self.np_dtype or not a.flags.c_contiguous:
                    raise ValueError("get_fields(out=...): arrays must be C-contiguous with the handle's shape and dtype")
        _check(lib().pf_get_fields(self.h, C.c_void_p(psi.ctypes.data), C.c_void_p(U.ctypes.data)), "pf_get_fields")
        return psi, U

    def set_fields(self, psi, U):
        psi = np.ascontiguousarray(psi, dtype=self.np_dtype).reshape(self.shape)
        U = np.ascontiguousarray(U, dtype=self.np_dtype).reshape(self.shape)
        _check(lib().pf_set_fields(self.h, C.c_void_p(psi.ctypes.data), C.c_void_p(U.ctypes.data)), "pf_set_fields")

    def set_fields_async(self, psi, U):
        """Queue the upload of psi, U (C-contiguous arrays of the handle's shape
        and dtype, ideally views of pinned host tensors) on the handle's stream
        without waiting; the arrays must stay alive until synchronize()."""
        for a in (psi, U):
            if a.shape != tuple(self.shape) or a.dtype != self.np_dtype or not a.flags.c_contiguous:
                raise ValueError("set_fields_async: arrays must be C-contiguous with the handle's shape and dtype")
        _check(lib().pf_set_fields_async(self.h, C.c_void_p(psi.ctypes.data), C.c_void_p(U.ctypes.data)),
               "pf_set_fields_async")

    def get_fields_async(self, psi, U):
        """Queue the download of the current psi, U into caller arrays without
        waiting; read them only after synchronize()."""
        for a in (psi, U):
            if a.shape != tuple(self.shape) or a.dtype != self.np_dtype or not a.flags.c_contiguous:
                raise ValueError("get_fields_async: arrays must be C-contiguous with the handle's shape and dtype")
        _check(lib().pf_get_fields_async(self.h, C.c_void_p(psi.ctypes.data), C.c_void_p(U.ctypes.data)),
               "pf_get_fields_async")

    def synchronize(self):
        _check(lib().pf_synchronize(self.h), "pf_synchronize")

    @property
    def steps_done(self) -> int:
        v = C.c_int64()
        _check(lib().pf_get_step(self.h, C.byref(v)), "pf_get_step")
        return v.value

    def set_step(self, n: int):
        _check(lib().pf_set_step(self.h, int(n)), "pf_set_step")

    def shift_frame(self, rows: int):
        """Move the state `rows` cells toward -y (a box that follows the tip
        upward); the frozen temperature stays put (pf_shift_frame)."""
        _check(lib().pf_shift_frame(self.h, int(rows)), "pf_shift_frame")

    def device_fields(self):
        a, b, c = C.c_void_p(), C.c_void_p(), C.c_void_p()
        _check(lib().pf_device_fields(self.h, C.byref(a), C.byref(b), C.byref(c)), "pf_device_fields")
        return a.value, b.value, c.value

    @property
    def n_cells(self) -> int:
        return int(np.prod(self.shape))

    def close(self):
        if getattr(self, "h", None):
            _check(lib().pf_destroy(self.h), "pf_destroy")
            self.h = None
            self.mem = None

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().pf_destroy(self.h)
        except Exception:
            pass


def observe_fields_noalloc(p: Params, psi_dev: int, U_dev: int, grain_dev: Optional[int], rot9, centre3,
                           grain: int = -1, stream=None, allow_nonfinite=False) -> dict:
    """pf_observe_fields_noalloc: the observe reductions on caller-held device
    fields, using the library's fixed device scratch instead of caller memory."""
    r = np.ascontiguousarray(rot9, dtype=np.float64).reshape(9)
    c = np.ascontiguousarray(centre3, dtype=np.float64).reshape(3)
    o = Obs()
    rc = lib().pf_observe_fields_noalloc(C.byref(p), C.c_void_p(psi_dev), C.c_void_p(U_dev),
                                         C.c_void_p(grain_dev) if grain_dev else None,
                                         r.ctypes.data_as(C.POINTER(C.c_double)),
                                         c.ctypes.data_as(C.POINTER(C.c_double)), int(grain),
                                         C.c_void_p(_stream_handle(stream)), C.byref(o))
    if rc != PF_OK and not (allow_nonfinite and rc == PF_ERR_NONFINITE):
        raise PfError(rc, "pf_observe_fields_noalloc")
    d = {f: getattr(o, f) for f, _ in Obs._fields_}
    d["tip"] = tuple(o.tip)
    d["status"] = rc
    return d


def wavefront_order(n_bands: int) -> list:
    """pf_wavefront_order: the (level, band) launches of one depth-2
    wavefront, level 0 = step n+1, level 1 = step n+2."""
    m = 2 * int(n_bands)
    lv, bd = (C.c_int * max(1, m))(), (C.c_int * max(1, m))()
    n = lib().pf_wavefront_order(int(n_bands), lv, bd, m)
    if n < 0:
        raise PfError(n, "pf_wavefront_order")
    return [(lv[i], bd[i]) for i in range(n)]


class Group:
    """Instances stepped together by one persistent launch per class."""

    def __init__(self, max_instances: int, max_work: int, stream=None, device="cuda"):
        import torch
        n = int(lib().pf_group_required_bytes(int(max_instances), int(max_work)))
        if n == 0:
            raise PfError(PF_ERR_INVALID, "pf_group_required_bytes")
        self.mem = torch.empty(n, dtype=torch.uint8, device=device)
        self.stream = stream
        h = C.c_void_p()
        _check(lib().pf_group_create(int(max_instances), int(max_work), C.c_void_p(self.mem.data_ptr()), n,
                                     C.c_void_p(_stream_handle(stream)), C.byref(h)), "pf_group_create")
        self.h = h
        self.members = []

    @staticmethod
    def work_items(sim: Sim) -> int:
        n = lib().pf_group_work_items(sim.h)
        if n < 0:
            raise PfError(n, "pf_group_work_items")
        return n

    def add(self, sim: Sim):
        _check(lib().pf_group_add(self.h, sim.h), "pf_group_add")
        self.members.append(sim)

    def remove(self, sim: Sim):
        _check(lib().pf_group_remove(self.h, sim.h), "pf_group_remove")
        self.members.remove(sim)

    def step(self, n: int = 1, use_graph: bool = True):
        _check(lib().pf_group_step(self.h, int(n), 1 if use_graph else 0), "pf_group_step")

    def set_depth(self, depth: int, band_sweeps: int = 1):
        """pf_group_set_depth: temporal-blocking depth 1 or 2 (two steps per
        wavefront over bands of band_sweeps sweeps)."""
        _check(lib().pf_group_set_depth(self.h, int(depth), int(band_sweeps)), "pf_group_set_depth")

    def depth(self) -> tuple:
        """(depth, band_sweeps, depth in effect for the current members)"""
        d, b, e = C.c_int(), C.c_int(), C.c_int()
        _check(lib().pf_group_get_depth(self.h, C.byref(d), C.byref(b), C.byref(e)), "pf_group_get_depth")
        return d.value, b.value, e.value

    def observe(self, grain: int = -1, allow_nonfinite=False) -> list:
        """pf_group_observe: observe() of every member, one synchronisation;
        dicts in the order the members were added."""
        n = len(self.members)
        arr = (Obs * max(1, n))()
        rc = lib().pf_group_observe(self.h, int(grain), arr)
        if rc != PF_OK and not (allow_nonfinite and rc == PF_ERR_NONFINITE):
            raise PfError(rc, "pf_group_observe")
        out = []
        for i in range(n):
            d = {f: getattr(arr[i], f) for f, _ in Obs._fields_}
            d["tip"] = tuple(arr[i].tip)
            d["status"] = PF_ERR_NONFINITE if arr[i].nonfinite else PF_OK
            out.append(d)
        return out

    def __len__(self):
        return int(lib().pf_group_size(self.h))

    def close(self):
        if getattr(self, "h", None):
            _check(lib().pf_group_destroy(self.h), "pf_group_destroy")
            self.h = None
            self.members = []

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().pf_group_destroy(self.h)
        except Exception:
            pass
