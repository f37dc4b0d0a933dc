"""Pins of the S_{2,1} standard anti-trapping term A_{2,1} (App. B) with the
magnitude floor of reading R-A21G.

App. B divides each of the eight D~_{2,1} fluxes of alpha grad(psi) by
|grad psi| from the 21-point derivatives at the flux point, so every flux
carries the quotient (psi_e - psi_0) / (|e| |grad psi|), the unit normal's
component along the flux direction e.  The oracle floors the magnitude at half
of the two-point slope, which bounds every quotient by 2:

* with alpha = 1 the term is then bounded on any field by
  (2/3)(1/h) 4 * 2 + (1/3)(1/(sqrt2 h)) 4 * 2 = (16/3 + 8/(3 sqrt2)) / h,
  the value with every quotient at +-2 (checked on rough random fields, where
  the 21-point and two-point gradients disagree often);
* on a linear field the 21-point derivatives are exact, every quotient is the
  normal component e.n (|.| <= 1), the floor never acts and the divergence of
  the constant unit-normal flux is zero.
"""
import math

import numpy as np
import pytest

BOUND = 16 / 3 + 8 / (3 * math.sqrt(2))


@pytest.mark.parametrize("scale", [0.05, 1.0, 20.0])
def test_at21_bounded_on_rough_fields(oracle, scale):
    rng = np.random.default_rng(int(scale * 100) + 7)
    n, h = 24, 0.9
    p = oracle.params(dim=2, nx=n, ny=n, h=h, bc=oracle.BC_PERIODIC)
    one = np.ones((n, n))
    worst = 0.0
    for _ in range(4):
        b = scale * rng.normal(size=(n, n))
        A = oracle.apply(p, "at_21", one, b)
        worst = max(worst, float(np.abs(A).max()) * h)
    assert worst <= BOUND * (1 + 1e-12), worst
    # rough fields come close to the bound: the floor is what holds them
    assert worst > 0.5 * BOUND, worst


@pytest.mark.parametrize("angle", [0.0, 0.3, math.pi / 4, 1.1, 2.0])
def test_at21_zero_on_linear_fields(oracle, angle):
    n, h = 17, 0.8
    p = oracle.params(dim=2, nx=n, ny=n, h=h, bc=oracle.BC_MIRROR)
    y, x = np.mgrid[0:n, 0:n] * h
    b = 1.7 * (math.cos(angle) * x + math.sin(angle) * y) - 3.0
    a = np.ones((n, n))
    A = oracle.apply(p, "at_21", a, b)
    inner = A[4:n - 4, 4:n - 4]  # away from the mirror walls (App. B reaches two cells)
    assert np.abs(inner).max() < 1e-12


@pytest.mark.parametrize("scale", [0.05, 1.0, 20.0])
def test_at21_corner_fluxes_bounded(oracle, scale):
    """Cells whose four face neighbours equal the cell's value have zero <10>
    fluxes; what remains are the four <11> fluxes, bounded by
    (1/3)(1/(sqrt2 h)) 4 * 2 = 8 / (3 sqrt2 h)."""
    rng = np.random.default_rng(int(scale * 100) + 11)
    n, h = 30, 0.9
    p = oracle.params(dim=2, nx=n, ny=n, h=h, bc=oracle.BC_PERIODIC)
    one = np.ones((n, n))
    cells = [(j, i) for j in range(3, n, 6) for i in range(3, n, 6)]
    worst = 0.0
    for _ in range(6):
        b = scale * rng.normal(size=(n, n))
        for j, i in cells:
            b[j, i - 1] = b[j, i + 1] = b[j - 1, i] = b[j + 1, i] = b[j, i]
        A = oracle.apply(p, "at_21", one, b)
        worst = max(worst, max(abs(A[j, i]) for j, i in cells) * h)
    corner_bound = 8 / (3 * math.sqrt(2))
    assert worst <= corner_bound * (1 + 1e-12), worst
    assert worst > 0.5 * corner_bound, worst
