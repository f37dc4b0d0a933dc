"""Pins of the oracle's explicit-Euler bound or_dt_max (the bound the
library's pf_create enforces).

The bound is dt <= 2 h^2 / (Lambda max(D, 1)) with Lambda the largest
|symbol| h^2 of the scheme's Laplacian: 16/3 for L_{2,1} and L_{1,2,0}, 8 for
L_{1,0}, 12 for L_{1,0,0}.  Two checks that do not reuse those constants:
  * Lambda found by brute force: the oracle's own Laplacian applied to every
    Fourier mode of a small periodic grid, largest |L(k)| h^2 over the modes;
  * the step itself: in an all-liquid periodic box the most unstable mode of
    U (D > 1) or of psi (D < 1) shrinks per step just below the bound and
    grows just above it (the growth factor passes -1 there).
"""
import math

import numpy as np
import pytest

from paper_2110_12448_gb300 import synth

LAP = {"SBAR21": "lap_21", "S21": "lap_21", "S10": "lap_10", "SBAR120": "lap_120", "S100": "lap_100"}
LAMBDA = {"SBAR21": 16 / 3, "S21": 16 / 3, "S10": 8.0, "SBAR120": 16 / 3, "S100": 12.0}


def modes(dim, n, h):
    ax = np.arange(n) * h
    if dim == 2:
        X, Y = np.meshgrid(ax, ax, indexing="xy")
        coords = (X, Y)
    else:
        Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
        coords = (X, Y, Z)
    for m in np.ndindex(*(n,) * dim):
        k = [2 * math.pi * mq / (n * h) for mq in m]
        yield k, np.cos(sum(kq * c for kq, c in zip(k, coords)))


def brute_lambda(O, scheme, n):
    dim = 3 if scheme in ("SBAR120", "S100") else 2
    h = 1.0
    p = O.params(dim=dim, nx=n, ny=n, nz=n, scheme=synth.SCHEMES[scheme], h=h, bc=O.BC_PERIODIC)
    best, kbest = 0.0, None
    for k, f in modes(dim, n, h):
        if not np.any(f):
            continue
        Lf = O.apply(p, LAP[scheme], f)
        lam = -float(np.sum(Lf * f) / np.sum(f * f)) * h * h
        if lam > best:
            best, kbest = lam, k
    return best, kbest


@pytest.mark.parametrize("scheme", ["SBAR21", "S10", "SBAR120", "S100"])
def test_lambda_by_brute_force(oracle, scheme):
    n = 8 if scheme in ("SBAR21", "S10") else 4
    lam, _ = brute_lambda(oracle, scheme, n)
    assert abs(lam - LAMBDA[scheme]) < 1e-12, (scheme, lam)
    dim = 3 if scheme in ("SBAR120", "S100") else 2
    for D, h in ((6.267, 0.8), (0.5, 1.2)):
        p = oracle.params(dim=dim, nx=8, ny=8, nz=8, scheme=synth.SCHEMES[scheme], h=h, D=D)
        assert abs(oracle.dt_max(p) - 2 * h * h / (lam * max(D, 1.0))) <= 1e-15 * oracle.dt_max(p)


@pytest.mark.parametrize("D", [6.267, 0.5])
@pytest.mark.parametrize("scheme", ["SBAR21", "S21", "S10", "SBAR120", "S100"])
def test_step_is_stable_just_below_the_bound(oracle, scheme, D):
    dim = 3 if scheme in ("SBAR120", "S100") else 2
    n = 8 if dim == 2 else 4
    h = 0.8
    lam, k = brute_lambda(oracle, scheme, n)
    f = next(f for kk, f in modes(dim, n, h) if np.allclose(kk, [kq / h for kq in k]))
    g = np.zeros(f.shape, np.int16)
    growth = {}
    for frac in (0.999, 1.001):
        p = oracle.params(dim=dim, nx=n, ny=n, nz=n, scheme=synth.SCHEMES[scheme], h=h, D=D, eps4=0.0,
                          bc=oracle.BC_PERIODIC)
        p.dt = frac * oracle.dt_max(p)
        if D > 1:  # U carries the fastest mode: phi = -1 everywhere
            psi, U = np.full(f.shape, -60.0), -0.5 + 1e-3 * f
            _, U1 = oracle.step(p, np.eye(3), g, psi, U, 1)
            a = float(np.sum((U1 - U1.mean()) * f) / np.sum(f * f)) / 1e-3
        else:  # psi's mobility 1 exceeds D
            psi, U = -60.0 + 1e-6 * f, np.full(f.shape, -0.5)
            psi1, _ = oracle.step(p, np.eye(3), g, psi, U, 1)
            a = float(np.sum((psi1 - psi1.mean()) * f) / np.sum(f * f)) / 1e-6
        growth[frac] = a
    assert -1.0 < growth[0.999] < -0.99, growth
    assert growth[1.001] < -1.0, growth
