"""Host-side checks of the C-ABI library that need no GPU: the library builds
and loads, exports every function include/pf.h declares, and validates the
problem statement (sizes, scheme vs dimension, explicit-Euler bound on dt)
in pf_required_bytes, which touches no device."""
import ctypes as C
import os
import re

import pytest

from paper_2110_12448_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(pf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = C.CDLL(native.lib_path() if os.path.exists(native.lib_path()) else native.lib()._name)
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings():
    assert native.status_string(0) == "ok"
    assert "buffer" in native.status_string(native.PF_ERR_BUDGET)
    assert native.status_string(12345) == "unknown status"


def _p(**kw):
    d = dict(dim=2, nx=64, ny=48, nz=1, scheme="SBAR21", precision="f32")
    d.update(kw)
    return native.make_params(**d)


def test_required_bytes_layout():
    b32 = native.required_bytes(_p())
    b64 = native.required_bytes(_p(precision="f64"))
    n = 64 * 48
    assert b32 >= 4 * n * 4 + n * 2 and b64 >= 4 * n * 8 + n * 2
    assert b64 > b32
    assert native.required_bytes(_p(dim=3, nx=16, ny=16, nz=16, scheme="SBAR120", dt=0.015)) > 4 * 4 * 16 ** 3


@pytest.mark.parametrize("bad", [
    dict(nx=3), dict(ny=0), dict(dim=4), dict(scheme="SBAR120"), dict(dim=3, nz=8, scheme="SBAR21"),
    dict(precision=7), dict(h=0.0), dict(dt=-1.0), dict(k=1.0), dict(k=0.0), dict(eps4=-0.1), dict(max_grains=0),
    dict(D=-1.0), dict(U0=float("nan")),
    # explicit Euler bound: 2 h^2 / (16/3 D) for the isotropic Laplacian
    dict(dt=2 * 0.64 / (16 / 3 * 6.267) * 1.01),
    dict(scheme="S10", dt=2 * 0.64 / (8 * 6.267) * 1.01),
])
def test_invalid_parameters_rejected(bad):
    assert native.required_bytes(_p(**bad)) == 0


def test_stability_bound_boundary():
    ok = 2 * 0.64 / (16 / 3 * 6.267) * 0.99
    assert native.required_bytes(_p(dt=ok)) > 0
    # S10 has the larger Laplacian symbol (8) and so the tighter bound
    assert native.required_bytes(_p(scheme="S10", dt=ok)) == 0


DS = dict(thermal=1, bc_x=1, Vp=0.1, lT=100.0, yT=5.0)  # frozen gradient, periodic x


@pytest.mark.parametrize("bad", [
    dict(bc_x=2), dict(thermal=2),
    dict(DS, lT=0.0), dict(DS, lT=float("inf")), dict(DS, Vp=-0.1), dict(DS, yT=float("nan")),
    # F1 = 1 - (1-k) ((ny-1) h - yT) / lT at the top row: 1 - 0.85 * (47 * 0.8 - 5) / 30 < 0.05
    dict(DS, lT=30.0),
])
def test_invalid_directional_parameters_rejected(bad):
    assert native.required_bytes(_p(**bad)) == 0


def test_directional_parameters_accepted_and_bound():
    assert native.required_bytes(_p(**DS)) > 0
    assert native.required_bytes(_p(dim=3, nz=8, scheme="SBAR120", dt=0.01, **DS)) > 0
    # with F1min = 1 - 0.85 * (47 * 0.8 - 5) / 36 = 0.230 the psi mobility 1/F1min = 4.35 < D,
    # so the D bound still applies; with a small D the 1/F1min term takes over
    F1min = 1 - 0.85 * (47 * 0.8 - 5) / 36.0
    d_small = dict(DS, lT=36.0, D=1.0, lam=10.0)
    bound = 2 * 0.64 / (16 / 3 * (1 / F1min))
    assert native.required_bytes(_p(**dict(d_small, dt=bound * 0.99))) > 0
    assert native.required_bytes(_p(**dict(d_small, dt=bound * 1.01))) == 0


def test_unchecked_build_reports_no_bounds_record():
    # the default library compiles the index checks away
    assert native.debug_bounds() is None


@pytest.mark.parametrize("kw", [dict(dim=3, nz=16, scheme="SBAR120", dt=0.015),
                                dict(thermal=native.PF_FROZEN_GRADIENT, lT=100.0),
                                dict(bc_x=native.PF_BC_PERIODIC), dict(time_level=native.PF_T0)])
def test_compensated_precision_scope(kw):
    """PF_F32C (compensated FP32 state) is 2D, isothermal, mirror walls, T1 only;
    its fields take 8 bytes per cell and level (hi and lo halves)."""
    assert native.required_bytes(_p(**dict(kw, precision="f32c"))) == 0
    n = 64 * 48
    assert native.required_bytes(_p(precision="f32c")) >= 4 * n * 8 + n * 2


def test_two_kernel_form_scope():
    """PF_TWO_KERNELS is the 2D T0 form with FP32 or FP64 fields; it adds one
    field-sized buffer for d psi/dt."""
    t0 = dict(time_level=native.PF_T0, kernels=native.PF_TWO_KERNELS)
    n = 64 * 48
    assert native.required_bytes(_p(**t0)) >= native.required_bytes(_p(time_level=native.PF_T0)) + 4 * n
    assert native.required_bytes(_p(precision="f64", **t0)) > 0
    for bad in (dict(time_level=native.PF_T1, kernels=native.PF_TWO_KERNELS), dict(t0, precision="f32c"),
                dict(t0, dim=3, nz=16, scheme="SBAR120", dt=0.015), dict(kernels=2)):
        assert native.required_bytes(_p(**bad)) == 0, bad
