"""GPU parity of the tip-radius measurement (Sec. 3.3.2, Sec. 6.2.2) through the
C-ABI against the FP64 oracle: planted parabolas are recovered exactly, and on
grown dendrites (2D and 3D, FP32 and FP64 fields) the device's contour
crossings and fits equal the oracle's on the same fields and tip (both use
the same explicitly rounded FP64 steps; tolerance 1e-12 relative)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    return N


def oracle_tip(w, psi, tip, centre):
    p = oracle_params(w)
    axis = np.asarray(tip[:w.dim], dtype=np.float64) - np.asarray(centre[:w.dim], dtype=np.float64)
    return O.tip_radius(p, psi.astype(np.float64), tip[:w.dim], axis)


def close(a, b, tol=1e-12):
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    return abs(a - b) <= tol * abs(b)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_planted_parabola_recovered(native, prec):
    n = 97  # centre ((n-1)/2 h, (n-1)/2 h) sits on a cell centre
    w = synth.free_dendrite_2d(n)
    s = native.Sim.from_workload(w, prec)
    h = w.h
    c = w.centres[0]
    tip = (c[0], c[1] + 20 * h, 0.0)
    rho = 9.0
    y, x = np.meshgrid(np.arange(n) * h, np.arange(n) * h, indexing="ij")
    psi = (tip[1] - (x - tip[0]) ** 2 / (2 * rho)) - y
    s.set_fields(psi, np.zeros_like(psi))
    psi_dev, _ = s.get_fields()
    r = s.tip_radius({"tip": tip, "v_tip": 0.0})
    o = oracle_tip(w, psi_dev, tip, c)
    assert close(r["rho"], o["rho"]) and r["n_x"] == o["n_x"]
    assert abs(r["rho"] - rho) <= (1e-10 if prec == "f64" else 1e-4) * rho
    assert math.isnan(r["sigma_star"])  # no velocity given
    assert r["axis"][0] == 0.0 and r["axis"][1] == 1.0


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("theta", [0.0, 25.0])
def test_grown_dendrite_2d_matches_oracle(native, prec, theta):
    w = synth.free_dendrite_2d(160, theta)
    s = native.Sim.from_workload(w, prec)
    s.step(300)
    s.observe()
    s.step(100)
    ob = s.observe()
    assert ob["found"] == 1
    r = s.tip_radius(ob)
    psi, _ = s.get_fields()
    o = oracle_tip(w, psi, ob["tip"], w.centres[0])
    assert close(r["rho"], o["rho"]) and r["n_x"] == o["n_x"]
    assert r["rho"] > 0 and r["n_x"] >= 4
    # sigma* = 2 D d0* / (rho^2 V), d0* = (1 - (1-k) Omega) / k * a1 / lambda, Omega = -U0
    d0s = (1 - (1 - w.k) * (-w.U0)) / w.k * (5 * math.sqrt(2) / 8) / w.lam
    assert close(r["d0_star"], d0s, 1e-14)
    assert ob["v_tip"] > 0 and close(r["sigma_star"], 2 * w.D * d0s / (r["rho"] ** 2 * ob["v_tip"]), 1e-12)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_grown_dendrite_3d_matches_oracle(native, prec):
    w = synth.free_dendrite_3d(56)
    s = native.Sim.from_workload(w, prec)
    s.step(120)
    ob = s.observe()
    assert ob["found"] == 1
    r = s.tip_radius(ob)
    psi, _ = s.get_fields()
    o = oracle_tip(w, psi, ob["tip"], w.centres[0])
    for key in ("rho", "rho_x", "rho_z"):
        assert close(r[key], o[key]), (key, r[key], o[key])
    assert (r["n_x"], r["n_z"]) == (o["n_x"], o["n_z"])


def test_invalid_tip_rejected(native):
    w = synth.free_dendrite_2d(64)
    s = native.Sim.from_workload(w, "f32")
    with pytest.raises(native.PfError):
        s.tip_radius({"tip": (float("nan"), 1.0, 0.0)})
    with pytest.raises(native.PfError):
        s.tip_radius({"tip": tuple(w.centres[0])})  # zero growth axis
