"""Pins of the oracle's directional-solidification terms (frozen temperature,
Eqs. Thermal_F1 and Thermal_F2 in Eq. PF_a; Sec. 2.1, Sec. 4.2) and of the
periodic-x boundary, against what the model fixes:
- an infinite thermal length reduces the step to the isothermal one exactly;
- for a field psi linear in y (and eps4 = 0) the Laplacian and the anisotropy
  fluxes vanish and the gradient square is exact, so Eq. PF_a reduces to the
  closed form  F1 dpsi/dt = sqrt2 phi (1 - |grad psi|^2) - sqrt2 lambda
  (1 - phi^2) (U + zeta);
- periodic x commutes with periodic shifts of the grid, bit for bit;
- the sharp-interface steady state of a pulled planar front: the interface
  sits on the isotherm zeta = 0 (U = 0 at the interface, no curvature, no
  kinetics) and moves at Vp; ahead of it U = -1 + exp(-Vp eta / D)."""
import math

import numpy as np
import pytest

from oracle import oracle as O

SQ2 = math.sqrt(2.0)


def rand_state(rng, nx, ny):
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    psi = 3.0 * np.sin(2 * np.pi * x / nx) + 0.4 * (ny / 2 - y) + rng.normal(0, 0.3, (ny, nx))
    U = -0.5 + 0.2 * rng.random((ny, nx))
    return psi, U


def test_infinite_thermal_length_is_isothermal():
    rng = np.random.default_rng(1)
    psi, U = rand_state(rng, 24, 20)
    g = np.zeros((20, 24), np.int16)
    rot = np.eye(3).reshape(1, 9)
    base = dict(nx=24, ny=20, eps4=0.03)
    a = O.step(O.params(**base), rot, g, psi, U, 3)
    b = O.step(O.params(thermal=1, Vp=0.0, lT=1e30, yT=5.0, **base), rot, g, psi, U, 3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("gy", [-1.0, 0.7])
@pytest.mark.parametrize("bc", [O.BC_MIRROR, O.BC_PERIODIC_X])
def test_linear_psi_closed_form_rate(gy, bc):
    nx, ny, h = 12, 40, 0.8
    rng = np.random.default_rng(2)
    y = (np.arange(ny) * h)[:, None] * np.ones((1, nx))
    psi = 1.5 + gy * (y - 16.0)
    U = -0.6 + 0.3 * rng.random((ny, nx))
    k, lam, Vp, lT, yT, t0 = 0.15, 10.0, 0.4, 37.0, 9.0, 3.1
    p = O.params(nx=nx, ny=ny, h=h, eps4=0.0, k=k, lam=lam, thermal=1, Vp=Vp, lT=lT, yT=yT, t0=t0, bc=bc)
    _, _, rate = O.step(p, np.eye(3).reshape(1, 9), np.zeros((ny, nx), np.int16), psi, U, 1, want_rate=True)
    phi = np.tanh(psi / SQ2)
    zeta = (y - yT - Vp * t0) / lT
    F1 = 1.0 - (1.0 - k) * zeta
    expect = (SQ2 * phi * (1.0 - gy * gy) - SQ2 * lam * (1.0 - phi ** 2) * (U + zeta)) / F1
    inner = slice(2, ny - 2)  # the linear profile is exact away from the mirror walls in y
    assert np.max(np.abs(rate[inner] - expect[inner])) <= 1e-12 * np.max(np.abs(expect[inner])) + 1e-13


@pytest.mark.parametrize("scheme", [O.SBAR21, O.S21, O.S10])
def test_periodic_x_commutes_with_shifts(scheme):
    rng = np.random.default_rng(3)
    nx, ny = 20, 16
    psi, U = rand_state(rng, nx, ny)
    g = (rng.random((ny, nx)) < 0.3).astype(np.int16)
    rot = np.stack([np.eye(3).ravel(),
                    np.array([[0.8, -0.6, 0], [0.6, 0.8, 0], [0, 0, 1]]).ravel()])
    p = O.params(nx=nx, ny=ny, scheme=scheme, bc=O.BC_PERIODIC_X, eps4=0.04, thermal=1, Vp=0.3, lT=50.0, yT=4.0)
    a = O.step(p, rot, g, psi, U, 2)
    for m in (1, 7):
        b = O.step(p, rot, np.roll(g, m, 1), np.roll(psi, m, 1), np.roll(U, m, 1), 2)
        assert np.array_equal(np.roll(a[0], m, 1), b[0]) and np.array_equal(np.roll(a[1], m, 1), b[1])


def test_pulled_planar_front_tracks_the_isotherm():
    # Thin-interface regime (V W / D = 0.016, diffusion length D / V = 63 W);
    # the thermal length keeps F1 = 1 - (1-k) zeta >= 0.3 over the liquid.
    # Start from the steady state and check that it is kept for 10^4 steps:
    # speed Vp (mass balance), new solid at U = 0 (c_s = c_inf), the front on
    # zeta = 0, and the diffusion profile ahead.  (At V W / D of order 0.1 the
    # model traps solute and the front runs away from the isotherm.)
    nx, ny, h, dt = 4, 220, 0.8, 0.02
    k, lam = 0.15, 10.0
    D = 0.6267 * lam
    Vp, lT, yT = 0.1, 150.0, 30.0
    y = (np.arange(ny) * h)[:, None] * np.ones((1, nx))
    eta = y - yT
    psi = -eta
    U = np.where(eta < 0, 0.0, -1.0 + np.exp(-Vp * np.maximum(eta, 0) / D))
    g = np.zeros((ny, nx), np.int16)
    rot = np.eye(3).reshape(1, 9)

    def front(ps):
        col = ps[:, 0]
        j = int(np.nonzero((col[:-1] >= 0) & (col[1:] < 0))[0][0])
        return (j + col[j] / (col[j] - col[j + 1])) * h, j

    t = 0.0
    fronts = []
    for _ in range(2):
        p = O.params(nx=nx, ny=ny, h=h, dt=dt, k=k, lam=lam, D=D, eps4=0.0, bc=O.BC_PERIODIC_X, thermal=1,
                     Vp=Vp, lT=lT, yT=yT, t0=t)
        psi, U = O.step(p, rot, g, psi, U, 5000)
        t += 5000 * dt
        fronts.append(front(psi))
    (y1, _), (y2, j2) = fronts
    assert abs((y2 - y1) / (5000 * dt) - Vp) <= 0.01 * Vp
    assert abs(y2 - (yT + Vp * t)) < 0.25
    assert abs(U[j2 - 12, 0]) < 0.01  # solidified during the run
    for d in (5.0, 20.0, 50.0):
        jj = int(round((y2 + d) / h))
        assert abs(U[jj, 0] - (-1.0 + math.exp(-Vp * (jj * h - y2) / D))) < 0.01


# ---- 3D: the same terms in Eq. PF_a (pulling along +y), periodic x, mirror y and z ----

def rand_state3(rng, nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    psi = 2.0 * np.sin(2 * np.pi * x / nx) + np.cos(2 * np.pi * z / nz) + 0.4 * (ny / 2 - y) + \
        rng.normal(0, 0.3, (nz, ny, nx))
    U = -0.5 + 0.2 * rng.random((nz, ny, nx))
    return psi, U


def test_infinite_thermal_length_is_isothermal_3d():
    rng = np.random.default_rng(11)
    psi, U = rand_state3(rng, 10, 9, 8)
    g = np.zeros((8, 9, 10), np.int16)
    rot = np.eye(3).reshape(1, 9)
    base = dict(dim=3, nx=10, ny=9, nz=8, scheme=O.SBAR120, dt=0.01, eps4=0.03)
    a = O.step(O.params(**base), rot, g, psi, U, 2)
    b = O.step(O.params(thermal=1, Vp=0.0, lT=1e30, yT=3.0, **base), rot, g, psi, U, 2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("scheme", [O.SBAR120, O.S100])
def test_linear_psi_closed_form_rate_3d(scheme):
    nx, ny, nz, h = 6, 24, 5, 0.8
    rng = np.random.default_rng(12)
    y = (np.arange(ny) * h)[None, :, None] * np.ones((nz, 1, nx))
    gy = 0.8
    psi = 1.0 + gy * (y - 9.0)
    U = -0.6 + 0.3 * rng.random((nz, ny, nx))
    k, lam, Vp, lT, yT, t0 = 0.15, 10.0, 0.3, 41.0, 7.0, 2.3
    p = O.params(dim=3, nx=nx, ny=ny, nz=nz, h=h, dt=0.01, scheme=scheme, eps4=0.0, k=k, lam=lam, thermal=1,
                 Vp=Vp, lT=lT, yT=yT, t0=t0, bc=O.BC_PERIODIC_X)
    _, _, rate = O.step(p, np.eye(3).reshape(1, 9), np.zeros((nz, ny, nx), np.int16), psi, U, 1, want_rate=True)
    phi = np.tanh(psi / SQ2)
    zeta = (y - yT - Vp * t0) / lT
    expect = (SQ2 * phi * (1.0 - gy * gy) - SQ2 * lam * (1.0 - phi ** 2) * (U + zeta)) / (1.0 - (1.0 - k) * zeta)
    inner = (slice(None), slice(2, ny - 2), slice(None))
    assert np.max(np.abs(rate[inner] - expect[inner])) <= 1e-12 * np.max(np.abs(expect[inner])) + 1e-13


@pytest.mark.parametrize("scheme", [O.SBAR120, O.S100])
def test_periodic_x_commutes_with_shifts_3d(scheme):
    rng = np.random.default_rng(13)
    nx, ny, nz = 11, 9, 8
    psi, U = rand_state3(rng, nx, ny, nz)
    g = (rng.random((nz, ny, nx)) < 0.3).astype(np.int16)
    c, s_ = math.cos(0.4), math.sin(0.4)
    rot = np.stack([np.eye(3).ravel(), np.array([[c, -s_, 0], [s_, c, 0], [0, 0, 1]]).ravel()])
    p = O.params(dim=3, nx=nx, ny=ny, nz=nz, scheme=scheme, dt=0.01, bc=O.BC_PERIODIC_X, eps4=0.04, thermal=1,
                 Vp=0.3, lT=50.0, yT=2.0)
    a = O.step(p, rot, g, psi, U, 2)
    for m in (1, 6):
        b = O.step(p, rot, np.roll(g, m, 2), np.roll(psi, m, 2), np.roll(U, m, 2), 2)
        assert np.array_equal(np.roll(a[0], m, 2), b[0]) and np.array_equal(np.roll(a[1], m, 2), b[1])


def test_observe_pulling_axis_tip_on_a_tilted_front(oracle):
    """Observation g = -2 takes the pulling axis +y as the growth axis (the most
    advanced interface along y, tracked in Sec. 4.3.3 and 6.2.3); g = -1 the
    crystal axis.  On the planar front psi = Y0 + s (x - x0) - y (linear, so
    the interpolated crossing is exact: y = Y0 + s (x - x0)) rising to the
    right, with the crystal turned 30 deg counter-clockwise (axis
    (-1/2, sqrt3/2)), the +y tip is the last column and the crystal-axis tip
    the first, whose projection falls as -1/2 + s sqrt3/2 < 0 per unit x."""
    nx, ny, h, Y0, x0, slope = 24, 20, 0.8, 7.3, 4.0, 0.2
    p = oracle.params(dim=2, nx=nx, ny=ny, h=h)
    y, x = np.mgrid[0:ny, 0:nx] * h
    psi = (Y0 + slope * (x - x0)) - y
    U = np.zeros_like(psi)
    t = np.radians(30.0)
    rot = np.array([[np.cos(t), -np.sin(t), 0.0], [np.sin(t), np.cos(t), 0.0], [0.0, 0.0, 1.0]]).reshape(1, 9)
    centres = np.array([[nx * h / 2, ny * h / 2, 0.0]])
    g = np.zeros((ny, nx), np.int16)
    o2 = oracle.observe(p, rot, centres, g, psi, U, g=-2)
    o1 = oracle.observe(p, rot, centres, g, psi, U, g=-1)
    xe = (nx - 1) * h
    assert abs(o2["tip_x"] - xe) < 1e-12 and abs(o2["tip_y"] - (Y0 + slope * (xe - x0))) < 1e-12
    assert abs(o2["score"] - (o2["tip_y"] - centres[0, 1])) < 1e-12
    assert abs(o1["tip_x"] - 0.0) < 1e-12 and abs(o1["tip_y"] - (Y0 + slope * (0.0 - x0))) < 1e-12
