"""Pins of the oracle's tip-radius fit (Sec. 3.3.2, Sec. 6.2.2; reading R-RHO)
against shapes whose radius is known in closed form: grid-aligned parabolas
and paraboloids are recovered to round-off (the contour lines then run along
grid columns, where multilinear interpolation of a field linear along the line
is exact), the one-radius window ignores a tail that leaves the parabola, and
rotated shapes are recovered to the interpolation error."""
import math

import numpy as np
import pytest

from oracle import oracle as O

H = 0.5


def grid2(nx, ny):
    y, x = np.meshgrid(np.arange(ny) * H, np.arange(nx) * H, indexing="ij")
    return x, y


def test_aligned_parabola_recovered_exactly():
    nx, ny = 96, 128
    x, y = grid2(nx, ny)
    xt, yt, rho = 40 * H, 100 * H, 8.0
    psi = (yt - (x - xt) ** 2 / (2 * rho)) - y
    p = O.params(dim=2, nx=nx, ny=ny, h=H)
    r = O.tip_radius(p, psi, (xt, yt), (0.0, 1.0))
    assert abs(r["rho"] - rho) <= 1e-10 * rho
    assert math.isnan(r["rho_z"])
    # window t <= rho keeps |s| <= sqrt(2) rho = 11.3 (22 lines of spacing h = 0.5) on each side
    assert r["n_x"] == 44


def test_window_ignores_tail_beyond_one_radius():
    nx, ny = 96, 160
    x, y = grid2(nx, ny)
    xt, yt, rho = 48 * H, 140 * H, 6.0
    t = (x - xt) ** 2 / (2 * rho)
    # beyond 1.5 rho behind the tip the contour bends away (three times steeper)
    t = np.where(t <= 1.5 * rho, t, 1.5 * rho + 3.0 * (t - 1.5 * rho))
    psi = (yt - t) - y
    p = O.params(dim=2, nx=nx, ny=ny, h=H)
    r = O.tip_radius(p, psi, (xt, yt), (0.0, 1.0))
    assert abs(r["rho"] - rho) <= 1e-10 * rho


def test_growth_axis_direction_matters():
    # a tip growing toward -y: the lines must march toward +y into the solid
    nx, ny = 96, 128
    x, y = grid2(nx, ny)
    xt, yt, rho = 40 * H, 20 * H, 7.0
    psi = y - (yt + (x - xt) ** 2 / (2 * rho))
    p = O.params(dim=2, nx=nx, ny=ny, h=H)
    assert abs(O.tip_radius(p, psi, (xt, yt), (0.0, -1.0))["rho"] - rho) <= 1e-10 * rho
    # with the axis reversed the lines start inside the solid: no samples
    assert math.isnan(O.tip_radius(p, psi, (xt, yt), (0.0, 1.0))["rho"])


@pytest.mark.parametrize("alpha_deg", [15.0, 30.0, 45.0])
def test_rotated_parabola_within_interpolation_error(alpha_deg):
    nx = ny = 160
    x, y = grid2(nx, ny)
    a = math.radians(alpha_deg)
    epar = np.array([-math.sin(a), math.cos(a)])
    eperp = np.array([math.cos(a), math.sin(a)])
    tip = np.array([70.3 * H, 110.7 * H])
    rho = 12.0
    dx, dy = x - tip[0], y - tip[1]
    xp = dx * eperp[0] + dy * eperp[1]
    yp = dx * epar[0] + dy * epar[1]
    psi = -(xp ** 2) / (2 * rho) - yp
    p = O.params(dim=2, nx=nx, ny=ny, h=H)
    r = O.tip_radius(p, psi, tip, epar)
    assert abs(r["rho"] - rho) <= 0.03 * rho


def test_aligned_elliptic_paraboloid_3d():
    n = 64
    z, y, x = np.meshgrid(np.arange(n) * H, np.arange(n) * H, np.arange(n) * H, indexing="ij")
    xt, yt, zt = 30 * H, 50 * H, 28 * H
    rx, rz = 5.0, 9.0
    psi = (yt - (x - xt) ** 2 / (2 * rx) - (z - zt) ** 2 / (2 * rz)) - y
    p = O.params(dim=3, nx=n, ny=n, nz=n, h=H, scheme=O.SBAR120, dt=0.01)
    r = O.tip_radius(p, psi, (xt, yt, zt), (0.0, 1.0, 0.0))
    assert abs(r["rho_x"] - rx) <= 1e-10 * rx and abs(r["rho_z"] - rz) <= 1e-10 * rz
    assert abs(r["rho"] - 2.0 / (1.0 / rx + 1.0 / rz)) <= 1e-10 * r["rho"]


def test_axis_along_z_uses_x_as_reference():
    n = 64
    z, y, x = np.meshgrid(np.arange(n) * H, np.arange(n) * H, np.arange(n) * H, indexing="ij")
    xt, yt, zt = 32 * H, 30 * H, 50 * H
    ra, rb = 6.0, 4.0  # curvature radii along x and along y
    psi = (zt - (x - xt) ** 2 / (2 * ra) - (y - yt) ** 2 / (2 * rb)) - z
    p = O.params(dim=3, nx=n, ny=n, nz=n, h=H, scheme=O.SBAR120, dt=0.01)
    r = O.tip_radius(p, psi, (xt, yt, zt), (0.0, 0.0, 1.0))
    # reference axis x: rho_z is the x-curvature, rho_x the y-curvature
    assert abs(r["rho_z"] - ra) <= 1e-10 * ra and abs(r["rho_x"] - rb) <= 1e-10 * rb


def test_circle_fit_matches_analytic_crossings():
    # A circle is not a parabola one radius behind its apex, so the fit lands
    # below R.  The expected value applies the fit's window rounds to the exact
    # crossings t(s) = R - sqrt(R^2 - s^2); the oracle's crossings come from
    # interpolating the grid samples of the distance field, within ~h^2 / R.
    nx = ny = 128
    x, y = grid2(nx, ny)
    R = 14.0
    c = np.array([64 * H, 40 * H])
    psi = R - np.hypot(x - c[0], y - c[1])
    p = O.params(dim=2, nx=nx, ny=ny, h=H)
    r = O.tip_radius(p, psi, (c[0], c[1] + R), (0.0, 1.0))
    s = np.array([j * H for j in range(-32, 33) if j != 0])
    t = np.where(np.abs(s) < R, R - np.sqrt(np.maximum(R * R - s * s, 0.0)), np.nan)  # no crossing beyond R
    w = 160 * H / 4
    for _ in range(4):
        m = t <= w
        w = 0.5 * np.sum(s[m] ** 4) / np.sum(t[m] * s[m] ** 2)
    assert 0.7 * R < w < R
    assert abs(r["rho"] - w) <= 0.02 * w


@pytest.mark.parametrize("alpha_deg", [20.0, 35.0])
def test_oblique_axis_3d_within_interpolation_error(alpha_deg):
    # growth axis in the x-y plane at alpha from +y (the paper's 3D rotations):
    # rho_x belongs to the in-plane transverse axis, rho_z to z
    n = 72
    z, y, x = np.meshgrid(np.arange(n) * H, np.arange(n) * H, np.arange(n) * H, indexing="ij")
    a = math.radians(alpha_deg)
    epar = np.array([-math.sin(a), math.cos(a), 0.0])
    eperp = np.array([math.cos(a), math.sin(a), 0.0])
    tip = np.array([37.3 * H, 52.6 * H, 35.2 * H])
    rx, rz = 7.0, 11.0
    dx, dy, dz = x - tip[0], y - tip[1], z - tip[2]
    xp = dx * eperp[0] + dy * eperp[1]
    yp = dx * epar[0] + dy * epar[1]
    psi = -(xp ** 2) / (2 * rx) - dz ** 2 / (2 * rz) - yp
    p = O.params(dim=3, nx=n, ny=n, nz=n, h=H, scheme=O.SBAR120, dt=0.01)
    r = O.tip_radius(p, psi, tip, epar)
    assert abs(r["rho_x"] - rx) <= 0.03 * rx and abs(r["rho_z"] - rz) <= 0.03 * rz
