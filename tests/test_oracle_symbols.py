"""Pins of the oracle's stencils against what the paper prints.

* Small-k Fourier symbols of every base and combined operator (Sec. 4.2,
  Eqs. L_k_10, L_k_01, L_k_21, D_k_10, D_k_01, D_k_21; Sec. 6.1 for the 3D
  shells; App. A for the gradient square).  The symbol of a linear stencil is
  its value on a plane wave divided by the wave; for the divergence it is
  divided by alpha*beta with alpha = beta = the wave (Eq. Fourier_divergence),
  for the gradient square by psi*psi (Eq. Fourier_Gradient).
* Uniqueness of the isotropic weights (Eqs. prove1-prove2, Constrain_Lap1/2,
  Constrain_Div1/2): solved from the oracle's own base symbols.
* Reductions: each divergence with alpha = 1 equals the Laplacian of the same
  shell (Eqs. flux_10 and 2D_L10 etc.).
"""
import itertools
import math

import numpy as np
import pytest

N2, N3 = 9, 9
KMAG = 0.02


def _wave(dim, kvec, n):
    ax = np.arange(n, dtype=np.float64)
    if dim == 2:
        X, Y = np.meshgrid(ax, ax, indexing="xy")  # [y, x]
        th = kvec[0] * X + kvec[1] * Y
    else:
        Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")  # [z, y, x]
        th = kvec[0] * X + kvec[1] * Y + kvec[2] * Z
    return th


def symbol(O, dim, op, kind, kvec):
    n = N2 if dim == 2 else N3
    p = O.params(dim=dim, nx=n, ny=n, nz=n, h=1.0, bc=O.BC_MIRROR)
    th = _wave(dim, kvec, n)
    c, s = np.cos(th), np.sin(th)
    ctr = (n // 2,) * dim
    if kind == "lin":
        v = O.apply(p, op, c) + 1j * O.apply(p, op, s)
        return v[ctr] / np.exp(1j * th[ctr])
    if kind == "bil":
        v = (O.apply(p, op, c, c) - O.apply(p, op, s, s)) + 1j * (O.apply(p, op, c, s) + O.apply(p, op, s, c))
        return v[ctr] / np.exp(2j * th[ctr])
    # quadratic form Q: Q(c + i s) = Q(c) - Q(s) + i (Q(c+s) - Q(c) - Q(s))
    qc, qs, qcs = O.apply(p, op, c), O.apply(p, op, s), O.apply(p, op, c + s)
    v = (qc - qs) + 1j * (qcs - qc - qs)
    return v[ctr] / np.exp(2j * th[ctr])


def dirs(dim, n=12):
    if dim == 2:
        return [(math.cos(t), math.sin(t)) for t in np.linspace(0.03, math.pi / 2 - 0.03, n)]
    rng = np.random.default_rng(7)
    out = [(1.0, 0.0, 0.0), (1 / math.sqrt(2), 1 / math.sqrt(2), 0.0), (1 / math.sqrt(3),) * 3]
    for _ in range(n):
        v = rng.normal(size=3)
        out.append(tuple(v / np.linalg.norm(v)))
    return out


def q2(kx, ky, cross):
    return kx ** 4 + cross * kx * kx * ky * ky + ky ** 4


def q3(k, cross):
    kx, ky, kz = k
    return kx ** 4 + ky ** 4 + kz ** 4 + cross * (kx * kx * ky * ky + kx * kx * kz * kz + ky * ky * kz * kz)


# (operator, kind, continuum coefficient c2 with S = -c2 k^2 + ..., quartic(k))
CASES_2D = [
    ("lap_10", "lin", 1.0, lambda k: q2(*k, 0.0) / 12),           # Eq. L_k_10
    ("lap_01", "lin", 1.0, lambda k: q2(*k, 6.0) / 12),           # Eq. L_k_01
    ("lap_21", "lin", 1.0, lambda k: q2(*k, 2.0) / 12),           # Eq. L_k_21
    ("div_10", "bil", 2.0, lambda k: 2 / 3 * q2(*k, 0.75)),       # Eq. D_k_10
    ("div_01", "bil", 2.0, lambda k: 2 / 3 * q2(*k, 4.5)),        # Eq. D_k_01
    ("div_21", "bil", 2.0, lambda k: 2 / 3 * q2(*k, 2.0)),        # Eq. D_k_21
    ("grad2_10", "quad", 1.0, lambda k: q2(*k, 0.0) / 3),         # App. A
    ("grad2_01", "quad", 1.0, lambda k: q2(*k, 6.0) / 3),         # App. A
    ("grad2_21", "quad", 1.0, lambda k: q2(*k, 2.0) / 3),         # App. A, G_{2,1}
]
CASES_3D = [
    ("lap_100", "lin", 1.0, lambda k: q3(k, 0.0) / 12),
    ("lap_010", "lin", 1.0, lambda k: q3(k, 3.0) / 12),
    ("lap_001", "lin", 1.0, lambda k: q3(k, 6.0) / 12),
    ("lap_120", "lin", 1.0, lambda k: q3(k, 2.0) / 12),
    ("div_100", "bil", 2.0, lambda k: 2 / 3 * q3(k, 0.75)),
    ("div_010", "bil", 2.0, lambda k: 2 / 3 * q3(k, 21 / 8)),
    ("div_001", "bil", 2.0, lambda k: 2 / 3 * q3(k, 4.5)),
    ("div_120", "bil", 2.0, lambda k: 2 / 3 * q3(k, 2.0)),
    ("grad2_100", "quad", 1.0, lambda k: q3(k, 0.0) / 3),
    ("grad2_010", "quad", 1.0, lambda k: q3(k, 3.0) / 3),
    ("grad2_001", "quad", 1.0, lambda k: q3(k, 6.0) / 3),        # with the 1/16 reading of Eq. Grad_111
    ("grad2_120", "quad", 1.0, lambda k: q3(k, 2.0) / 3),
]


@pytest.mark.parametrize("op,kind,c2,quartic", CASES_2D, ids=[c[0] for c in CASES_2D])
def test_symbol_2d(oracle, op, kind, c2, quartic):
    for d in dirs(2):
        k = (KMAG * d[0], KMAG * d[1])
        S = symbol(oracle, 2, op, kind, k)
        k2 = k[0] ** 2 + k[1] ** 2
        got = (S + c2 * k2) / k2 ** 2
        want = quartic(k) / k2 ** 2
        assert abs(got.imag) < 1e-6
        assert abs(got.real - want) < 2e-3, (op, d, got, want)


@pytest.mark.parametrize("op,kind,c2,quartic", CASES_3D, ids=[c[0] for c in CASES_3D])
def test_symbol_3d(oracle, op, kind, c2, quartic):
    for d in dirs(3, 6):
        k = tuple(KMAG * x for x in d)
        S = symbol(oracle, 3, op, kind, k)
        k2 = sum(x * x for x in k)
        got = (S + c2 * k2) / k2 ** 2
        want = quartic(k) / k2 ** 2
        assert abs(got.imag) < 1e-6
        assert abs(got.real - want) < 2e-3, (op, d, got, want)


def _aniso_part(O, dim, op, kind):
    """k^4 coefficient of the cross term (kx^2 ky^2 [+ ...]) from two directions."""
    if dim == 2:
        k_ax = (KMAG, 0.0)
        k_dg = (KMAG / math.sqrt(2), KMAG / math.sqrt(2))
    else:
        k_ax = (KMAG, 0.0, 0.0)
        k_dg = (KMAG / math.sqrt(2), KMAG / math.sqrt(2), 0.0)
    c2 = 2.0 if kind == "bil" else 1.0
    q_ax = (symbol(O, dim, op, kind, k_ax).real + c2 * KMAG ** 2) / KMAG ** 4
    q_dg = (symbol(O, dim, op, kind, k_dg).real + c2 * KMAG ** 2) / KMAG ** 4
    # along an axis: a; along the diagonal: a/2 + cross/4 (2D) -> cross coefficient relative to a
    return q_ax, q_dg


@pytest.mark.parametrize("fam", ["lap", "div", "grad2"])
def test_unique_isotropic_weights_2d(oracle, fam):
    """Eqs. prove1-prove2: c1 L10 + c2 L01 isotropic and c1 + c2 = 1 -> (2/3, 1/3);
    the same weights for the divergence (Sec. 4.2.2) and the gradient square (App. A)."""
    kind = {"lap": "lin", "div": "bil", "grad2": "quad"}[fam]
    a1, d1 = _aniso_part(oracle, 2, f"{fam}_10", kind)
    a2, d2 = _aniso_part(oracle, 2, f"{fam}_01", kind)
    # isotropic quartic c k^4: along axis c, along diagonal c as well -> (d - a) weighted sum = 0
    # c1 (d1 - a1) + c2 (d2 - a2) = 0, c1 + c2 = 1
    M = np.array([[d1 - a1, d2 - a2], [1.0, 1.0]])
    c = np.linalg.solve(M, [0.0, 1.0])
    assert np.allclose(c, [2 / 3, 1 / 3], atol=3e-3), c


@pytest.mark.parametrize("fam", ["lap", "div", "grad2"])
def test_isotropic_weights_3d(oracle, fam):
    """Eqs. Constrain_Lap1/2 and Constrain_Div1/2: with no <111> weight the unique
    isotropic combination is (1/3, 2/3); with no <110> weight (2/3, 0, 1/3), and
    with no <100> weight (0, 4/3, -1/3)."""
    kind = {"lap": "lin", "div": "bil", "grad2": "quad"}[fam]
    an = [_aniso_part(oracle, 3, f"{fam}_{s}", kind) for s in ("100", "010", "001")]
    diff = [d - a for a, d in an]

    def solve(i, j):
        M = np.array([[diff[i], diff[j]], [1.0, 1.0]])
        return np.linalg.solve(M, [0.0, 1.0])

    assert np.allclose(solve(0, 1), [1 / 3, 2 / 3], atol=3e-3)
    assert np.allclose(solve(0, 2), [2 / 3, 1 / 3], atol=3e-3)
    assert np.allclose(solve(1, 2), [4 / 3, -1 / 3], atol=3e-3)


def test_printed_constraints_solutions():
    """The printed constraint systems themselves give the named combinations
    L_{1,2,0}, L_{2,0,1}, L_{0,4,-1} (Sec. 6.1.1) and the same for D (Sec. 6.1.2)."""
    for s1, s2, s3 in [(1, 2, 0), (2, 0, 1), (0, 4, -1), (5, 6, 1), (7, 6, 2), (4, 4, 1)]:
        t = s1 + s2 + s3
        c = (s1 / t, s2 / t, s3 / t)
        assert abs(sum(c) - 1) < 1e-15
        assert abs(3 * c[1] + 6 * c[2] - 2) < 1e-14                      # Eq. Constrain_Lap2
        assert abs(0.75 * c[0] + 21 / 8 * c[1] + 4.5 * c[2] - 2) < 1e-14  # Eq. Constrain_Div2
    # 2D: 6 c2 = 2 (c1 + c2) with c1 + c2 = 1
    assert abs(6 * (1 / 3) - 2 * 1) < 1e-15


REDUCTIONS = [
    (2, "div_10", "lap_10"), (2, "div_01", "lap_01"), (2, "div_21", "lap_21"), (2, "div_std2", "lap_10"),
    (3, "div_100", "lap_100"), (3, "div_010", "lap_010"), (3, "div_001", "lap_001"), (3, "div_120", "lap_120"),
    (3, "div_std3", "lap_100"),
]


@pytest.mark.parametrize("dim,div,lap", REDUCTIONS)
def test_divergence_with_unit_alpha_is_laplacian(oracle, dim, div, lap):
    rng = np.random.default_rng(3)
    n = 7
    shape = (n,) * dim
    p = oracle.params(dim=dim, nx=n, ny=n, nz=n, h=0.7, bc=oracle.BC_PERIODIC)
    b = rng.normal(size=shape)
    one = np.ones(shape)
    assert np.allclose(oracle.apply(p, div, one, b), oracle.apply(p, lap, b), rtol=0, atol=1e-12)


# Three-shell combinations of Eq. tau_3D that Sec. 6.1 names as isotropic
# solutions (row f4: symbol tools only; no <111> scheme is simulated).
COMBO_QUARTIC = {"lap": ("lin", 1.0, lambda k: q3(k, 2.0) / 12),
                 "div": ("bil", 2.0, lambda k: 2 / 3 * q3(k, 2.0)),
                 "grad2": ("quad", 1.0, lambda k: q3(k, 2.0) / 3)}


@pytest.mark.parametrize("fam", ["lap", "div", "grad2"])
@pytest.mark.parametrize("key", ["201", "04m1", "441", "561", "762"])
def test_symbol_isotropic_combinations_3d(oracle, fam, key):
    """L, D~ and G_{2,0,1}, _{0,4,-1}, _{4,4,1}, _{5,6,1}, _{7,6,2} (Sec. 6.1.1,
    6.1.2, App. A): every such combination has the isotropic k^4 error of the
    continuum-normalised form, (k^2)^2 / 12 for L and (2/3)(k^2)^2 for D~ as
    for L_{1,2,0} and D~_{1,2,0}; G likewise with (k^2)^2 / 3."""
    kind, c2, quartic = COMBO_QUARTIC[fam]
    for d in dirs(3, 6):
        k = tuple(KMAG * x for x in d)
        S = symbol(oracle, 3, f"{fam}_c{key}", kind, k)
        k2 = sum(x * x for x in k)
        got = (S + c2 * k2) / k2 ** 2
        assert abs(got.imag) < 1e-6
        assert abs(got.real - quartic(k) / k2 ** 2) < 2e-3, (fam, key, d, got)


def _quartic_about_kz_pi(O, op, d):
    """k^4 coefficient of the Laplacian symbol about (0, 0, pi) along the
    in-plane direction d, from S(r d, pi) = S0 + a r^2 + b r^4 at two radii."""
    s0 = symbol(O, 3, op, "lin", (0.0, 0.0, math.pi)).real
    r1, r2 = 0.04, 0.08
    f1 = symbol(O, 3, op, "lin", (r1 * d[0], r1 * d[1], math.pi)).real - s0
    f2 = symbol(O, 3, op, "lin", (r2 * d[0], r2 * d[1], math.pi)).real - s0
    a, b = np.linalg.solve([[r1 ** 2, r1 ** 4], [r2 ** 2, r2 ** 4]], [f1, f2])
    return a, b


def test_cross_section_kz_pi_441_isotropic_120_not(oracle):
    """Sec. 6.1.1 (Fig. of the 3D Laplacian symbols): L_{1,2,0} is isotropic only
    in the cross section k_z = 0, L_{4,4,1} in both k_z = 0 and k_z = pi.
    About (0, 0, pi) the exact symbols are (4 cx + 4 cy + 2 cx cy - 46) / 9 for
    L_{4,4,1} and (2 cx cy - 14) / 3 for L_{1,2,0}: both fall off as -k^2/3,
    the first with the isotropic quartic (k^2)^2 / 36, the second with
    (kx^4 + ky^4 + 6 kx^2 ky^2) / 36, twice as large on the diagonal."""
    ax, dg = (1.0, 0.0), (1 / math.sqrt(2), 1 / math.sqrt(2))
    for op in ("lap_c441", "lap_c120"):
        for d in (ax, dg, (math.cos(0.4), math.sin(0.4))):
            a, _ = _quartic_about_kz_pi(oracle, op, d)
            assert abs(a + 1 / 3) < 1e-3, (op, d, a)
    b441 = [_quartic_about_kz_pi(oracle, "lap_c441", d)[1] for d in (ax, dg, (math.cos(0.4), math.sin(0.4)))]
    assert np.allclose(b441, 1 / 36, rtol=0, atol=2e-3), b441
    b_ax = _quartic_about_kz_pi(oracle, "lap_c120", ax)[1]
    b_dg = _quartic_about_kz_pi(oracle, "lap_c120", dg)[1]
    assert abs(b_ax - 1 / 36) < 2e-3 and abs(b_dg - 2 / 36) < 2e-3, (b_ax, b_dg)
    assert abs(symbol(oracle, 3, "lap_c441", "lin", (0.0, 0.0, math.pi)).real + 4.0) < 1e-12
    assert abs(symbol(oracle, 3, "lap_c120", "lin", (0.0, 0.0, math.pi)).real + 4.0) < 1e-12


@pytest.mark.parametrize("fam", ["lap", "div", "grad2"])
def test_combination_120_is_the_two_shell_scheme(oracle, fam):
    """Eq. tau_3D with (1, 2, 0) reproduces the oracle's own S-bar_{1,2,0} operators."""
    rng = np.random.default_rng(5)
    n = 7
    p = oracle.params(dim=3, nx=n, ny=n, nz=n, h=0.9, bc=oracle.BC_PERIODIC)
    a, b = rng.normal(size=(n,) * 3), rng.normal(size=(n,) * 3)
    bb = b if fam == "div" else None
    assert np.allclose(oracle.apply(p, f"{fam}_c120", a, bb), oracle.apply(p, f"{fam}_120", a, bb), rtol=0, atol=1e-12)
