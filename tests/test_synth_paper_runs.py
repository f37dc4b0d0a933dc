"""The workloads of the paper's own isothermal runs carry the numbers the
paper states for them (Sec. 4.3.2 in 2D, Sec. 6.2.2 in 3D): W/d0* = 16,
h/W = 1.2, eps4 = 0.014, Omega = 0.43 (2D) / 0.25 (3D), k = 0.1, a seed of
radius 50 d0*, dt = 0.8 h^2 / (4 D) (2D) / 0.8 h^2 / (6 D) (3D), a box of
side 1.5e4 d0* (2D) and a run to t = 1.5e6 d0*^2 / D.  d0* follows the
definition d0* = d0 (1 - (1-k) Omega) / k with d0 = a1 W / lambda (Sec. 2.1)
and D = a2 lambda (thin-interface relation of the quantitative model)."""
import math

from paper_2110_12448_gb300 import synth

A1 = 5 * math.sqrt(2) / 8


def d0_star(w):
    omega = -w.U0
    return (1 - (1 - w.k) * omega) / w.k * A1 / w.lam


def test_paper_isothermal_2d_parameters():
    w = synth.paper_isothermal_2d(30.0, "S21")
    d0s = d0_star(w)
    assert abs(1 / d0s - 16.0) < 1e-12                       # W/d0* = 16
    assert (w.h, w.eps4, w.k, w.U0) == (1.2, 0.014, 0.1, -0.43)
    assert abs(w.dt - 0.8 * w.h ** 2 / (4 * w.D)) < 1e-15
    assert abs(w.D / w.lam - synth.A2) < 1e-15
    assert w.nx == w.ny == round(1.5e4 * d0s / w.h) == 781     # side 1.5e4 d0*
    assert abs(w.steps * w.dt - 1.5e6 * d0s ** 2 / w.D) < w.dt  # t = 1.5e6 d0*^2 / D
    assert abs(w.seeds[0, 3] - 50 * d0s) < 1e-12
    assert abs(w.seeds[0, 0] - (w.nx - 1) / 2 * w.h) < 1e-12    # at the centre
    R = w.rots[0].reshape(3, 3)
    assert abs(math.degrees(math.atan2(R[1, 0], R[0, 0])) - 30.0) < 1e-12


def test_paper_isothermal_3d_parameters():
    w = synth.paper_isothermal_3d(15.0, "SBAR120", n=64)
    d0s = d0_star(w)
    assert abs(1 / d0s - 16.0) < 1e-12
    assert (w.h, w.eps4, w.k, w.U0, w.dim) == (1.2, 0.014, 0.1, -0.25, 3)
    assert abs(w.dt - 0.8 * w.h ** 2 / (6 * w.D)) < 1e-15
    assert abs(w.steps * w.dt - 1.5e6 * d0s ** 2 / w.D) < w.dt
    assert abs(w.seeds[0, 3] - 50 * d0s) < 1e-12
    assert synth.paper_isothermal_3d(0.0, steps=100).steps == 100


def test_paper_directional_2d_units_and_seed():
    """Sec. 4.3.3 in model units: with the isothermal runs' Delta t rule the
    stated dt = 1e-5 s gives W = 0.210 um and d0 = 1.90 nm; the 3D runs'
    numbers (W/d0 = 194.2, h/W = 1, dt = 1.46e-5 s, the 3D rule 0.8 h^2/(6 D))
    give the same d0 within 1.5%.  The seed is periodic in x and a distance
    field (|grad psi| = 1 up to the finite differences)."""
    import numpy as np
    w = synth.paper_directional_2d(30.0)
    tau0 = 1e-5 / w.dt
    W = math.sqrt(1270.0 * tau0 / w.D)
    assert abs(W - 0.210) < 1e-3 and abs(W / 110.4 * 1e3 - 1.902) < 2e-3
    lam3 = A1 * 194.2
    dt3 = 0.8 * 1.0 / (6 * synth.A2 * lam3)
    W3 = math.sqrt(1270.0 * (1.46e-5 / dt3) / (synth.A2 * lam3))
    assert abs(W3 / 194.2 / (W / 110.4) - 1) < 0.015
    assert (w.nx, w.ny) == (758, 1948)
    assert abs(w.Vp - 86.0 * tau0 / W) < 1e-12
    assert abs(w.lT - 3.02 * 1.3 * 0.9 / 0.1 / 19e-4 / W) < 1e-6
    assert w.bc_x == 1 and w.thermal == 1 and w.U0 == -1.0
    p = w.psi_init
    assert np.abs(p[:, 0] - p[:, -1]).max() <= 1.01 * w.h  # continuous across the periodic wall
    gy, gx = np.gradient(p, w.h)
    assert np.hypot(gx, gy).max() < 1.1
    # the front starts delta0 = 0.03 below the liquidus (zeta = 1 at U = -1)
    y0 = w.ny * w.h / 8
    assert abs((y0 - w.yT) / w.lT - 0.97) < 1e-12
