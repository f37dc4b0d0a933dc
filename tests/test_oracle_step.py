"""Pins of the oracle's operators and time step against facts the paper and
the mathematics fix (none re-types the oracle's formulas):

* polynomial exactness: Laplacians on quadratics, gradient squares on
  linear fields, divergences with linear alpha and quadratic beta, and the
  App. B derivatives on every cubic;
* the real-space error of L_{2,1} is (h^2/12) bilaplacian (Sec. 4.1);
* the anisotropic flux J equals the g-gradient of a_s^2 |g|^2 / 2 with a_s
  from Eq. anis_function, and div(J - g) converges at O(h^2);
* App. B's standard anti-trapping A_{2,1} and the <10> forms converge to the
  continuum divergence at O(h^2);
* the planar interface psi = -n.r / a_s(n), U = 0 is a fixed point of the
  step (Eqs. PF_a, PF_b, any orientation);
* exact solute conservation with no-flux walls (Eq. Supersaturation, T1);
* Fourier-mode decay of U in an all-liquid box (closed form);
* lattice symmetry: transposing or mirroring the grid maps the step exactly
  when the orientation maps to -alpha0;
* the anti-trapping current of an advancing planar interface carries solute
  from the solid side into the liquid with the magnitude of Eq. Anti_convention.
"""
import math

import numpy as np
import pytest

from paper_2110_12448_gb300 import synth


def grid2(n, h):
    ax = np.arange(n) * h
    X, Y = np.meshgrid(ax, ax, indexing="xy")
    return X, Y


def grid3(n, h):
    ax = np.arange(n) * h
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    return X, Y, Z


def interior(a, r, dim):
    sl = tuple(slice(r, -r) for _ in range(dim))
    return a[sl]


@pytest.mark.parametrize("op", ["lap_10", "lap_01", "lap_21"])
def test_laplacian_exact_on_quadratics_2d(oracle, op):
    rng = np.random.default_rng(1)
    h = 0.37
    X, Y = grid2(10, h)
    c = rng.normal(size=6)
    f = c[0] + c[1] * X + c[2] * Y + c[3] * X * X + c[4] * X * Y + c[5] * Y * Y
    p = oracle.params(nx=10, ny=10, h=h)
    L = interior(oracle.apply(p, op, f), 2, 2)
    assert np.allclose(L, 2 * c[3] + 2 * c[5], rtol=0, atol=1e-10)


@pytest.mark.parametrize("op", ["lap_100", "lap_010", "lap_001", "lap_120"])
def test_laplacian_exact_on_quadratics_3d(oracle, op):
    rng = np.random.default_rng(2)
    h = 0.45
    X, Y, Z = grid3(8, h)
    c = rng.normal(size=10)
    f = (c[0] + c[1] * X + c[2] * Y + c[3] * Z + c[4] * X * X + c[5] * Y * Y + c[6] * Z * Z + c[7] * X * Y
         + c[8] * X * Z + c[9] * Y * Z)
    p = oracle.params(dim=3, nx=8, ny=8, nz=8, h=h)
    L = interior(oracle.apply(p, op, f), 2, 3)
    assert np.allclose(L, 2 * (c[4] + c[5] + c[6]), rtol=0, atol=1e-10)


@pytest.mark.parametrize("dim,op", [(2, "grad2_10"), (2, "grad2_01"), (2, "grad2_21"), (3, "grad2_100"),
                                    (3, "grad2_010"), (3, "grad2_001"), (3, "grad2_120")])
def test_gradient_square_exact_on_linear(oracle, dim, op):
    rng = np.random.default_rng(4)
    h = 0.6
    n = 8
    if dim == 2:
        X, Y = grid2(n, h)
        a = rng.normal(size=3)
        f = a[0] + a[1] * X + a[2] * Y
        want = a[1] ** 2 + a[2] ** 2
    else:
        X, Y, Z = grid3(n, h)
        a = rng.normal(size=4)
        f = a[0] + a[1] * X + a[2] * Y + a[3] * Z
        want = a[1] ** 2 + a[2] ** 2 + a[3] ** 2
    p = oracle.params(dim=dim, nx=n, ny=n, nz=n, h=h)
    G = interior(oracle.apply(p, op, f), 2, dim)
    assert np.allclose(G, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim,op", [(2, "div_10"), (2, "div_01"), (2, "div_21"), (2, "div_std2"),
                                    (3, "div_100"), (3, "div_010"), (3, "div_001"), (3, "div_120"),
                                    (3, "div_std3")])
def test_divergence_exact_linear_alpha_quadratic_beta(oracle, dim, op):
    rng = np.random.default_rng(5)
    h = 0.55
    n = 8
    if dim == 2:
        X, Y = grid2(n, h)
        a = rng.normal(size=3)
        b = rng.normal(size=6)
        al = 2.0 + a[1] * X + a[2] * Y
        be = b[0] + b[1] * X + b[2] * Y + b[3] * X * X + b[4] * X * Y + b[5] * Y * Y
        bx = b[1] + 2 * b[3] * X + b[4] * Y
        by = b[2] + b[4] * X + 2 * b[5] * Y
        want = a[1] * bx + a[2] * by + al * (2 * b[3] + 2 * b[5])
    else:
        X, Y, Z = grid3(n, h)
        a = rng.normal(size=4)
        b = rng.normal(size=7)
        al = 2.0 + a[1] * X + a[2] * Y + a[3] * Z
        be = b[0] + b[1] * X + b[2] * Y + b[3] * Z + b[4] * X * X + b[5] * Y * Y + b[6] * X * Z
        bx = b[1] + 2 * b[4] * X + b[6] * Z
        by = b[2] + 2 * b[5] * Y
        bz = b[3] + b[6] * X
        want = a[1] * bx + a[2] * by + a[3] * bz + al * (2 * b[4] + 2 * b[5])
    p = oracle.params(dim=dim, nx=n, ny=n, nz=n, h=h)
    D = oracle.apply(p, op, al, be)
    if op.startswith("div_std"):
        # the two-point face mean is exact for linear alpha as well
        pass
    assert np.allclose(interior(D, 2, dim), interior(want, 2, dim), rtol=0, atol=1e-10)


def test_appendix_b_derivatives_exact_on_cubics(oracle):
    """App. B: the face and corner derivatives have no h^2 error, hence are
    exact on every cubic polynomial."""
    rng = np.random.default_rng(6)
    h = 0.8
    n = 12
    X, Y = grid2(n, h)
    monos = [(i, j) for i in range(4) for j in range(4) if i + j <= 3]
    c = rng.normal(size=len(monos))
    f = sum(ci * X ** i * Y ** j for ci, (i, j) in zip(c, monos))

    def grad(x, y):
        gx = sum(ci * i * x ** (i - 1) * y ** j for ci, (i, j) in zip(c, monos) if i > 0)
        gy = sum(ci * j * x ** i * y ** (j - 1) for ci, (i, j) in zip(c, monos) if j > 0)
        return gx, gy

    for i, j in [(4, 4), (5, 6), (6, 5)]:
        for kind, off in [(0, (0.5, 0.0)), (1, (0.0, 0.5)), (2, (0.5, 0.5))]:
            got = oracle.appb_grad(f, i, j, kind, h)
            want = grad((i + off[0]) * h, (j + off[1]) * h)
            assert np.allclose(got, want, rtol=0, atol=1e-9), (kind, got, want)


def test_isotropic_laplacian_error_is_bilaplacian(oracle):
    """Sec. 4.1: L_{2,1} = lap + (h^2/12) lap^2 + O(h^4), and L_{1,0} has the
    anisotropic error (h^2/12)(psi_xxxx + psi_yyyy)."""
    n = 40
    for h in (0.2, 0.1):
        X, Y = grid2(n, h)
        cx = cy = (n - 1) / 2 * h
        s = 3.0 * 0.2 * 10
        r2 = ((X - cx) ** 2 + (Y - cy) ** 2) / s
        f = np.exp(-r2)
        # analytic derivatives of exp(-r^2/s)
        lap = f * (4 * r2 / s - 4 / s)
        bilap = f * (16 * r2 * r2 / s ** 2 - 64 * r2 / s ** 2 + 32 / s ** 2)
        p = oracle.params(nx=n, ny=n, h=h)
        err = interior(oracle.apply(p, "lap_21", f) - lap - h * h / 12 * bilap, 3, 2)
        assert np.max(np.abs(err)) < 40 * h ** 4 / s ** 3


def _energy_grad_2d(g, theta0, eps4, d=1e-6):
    """d/dg of a_s^2 |g|^2 / 2 with a_s = 1 + eps4 cos 4(theta - theta0) (Eq. anis_function)."""
    def e(gx, gy):
        th = math.atan2(gy, gx)
        a = 1 + eps4 * math.cos(4 * (th - theta0))
        return 0.5 * a * a * (gx * gx + gy * gy)
    gx, gy = g
    return np.array([(e(gx + d, gy) - e(gx - d, gy)) / (2 * d), (e(gx, gy + d) - e(gx, gy - d)) / (2 * d)])


def test_anisotropic_flux_is_energy_gradient_2d(oracle):
    rng = np.random.default_rng(8)
    for _ in range(40):
        th0 = rng.uniform(-math.pi, math.pi)
        eps4 = rng.uniform(0.0, 0.06)
        g = rng.normal(size=2) * rng.uniform(0.1, 3)
        R = synth.rot2d(math.degrees(th0))
        a, jmg = oracle.aniso(2, R, eps4, g)
        th = math.atan2(g[1], g[0])
        assert abs(a - (1 + eps4 * math.cos(4 * (th - th0)))) < 1e-13
        J = _energy_grad_2d(g, th0, eps4)
        assert np.allclose(jmg[:2] + g, J, rtol=1e-7, atol=1e-8)


def test_cubic_anisotropy_3d_reduces_and_is_energy_gradient(oracle):
    """The 3D cubic form restricted to a crystal {100} plane is Eq. anis_function;
    it is invariant under the cubic group; J is the g-gradient of a^2|g|^2/2."""
    rng = np.random.default_rng(9)
    for _ in range(30):
        R = synth.random_rot3(rng)
        eps4 = rng.uniform(0.0, 0.05)
        th = rng.uniform(-math.pi, math.pi)
        gc = np.array([math.cos(th), math.sin(th), 0.0]) * rng.uniform(0.2, 2)
        g = R @ gc
        a, _ = oracle.aniso(3, R, eps4, g)
        assert abs(a - (1 + eps4 * math.cos(4 * th))) < 1e-12
        # cubic symmetry: permute / flip crystal axes
        gc2 = rng.normal(size=3)
        P = np.eye(3)[rng.permutation(3)] * rng.choice([-1, 1], size=3)
        a1, _ = oracle.aniso(3, R, eps4, R @ gc2)
        a2, _ = oracle.aniso(3, R, eps4, R @ (P @ gc2))
        assert abs(a1 - a2) < 1e-13
        # energy gradient
        gv = rng.normal(size=3)
        d = 1e-6

        def e(v):
            aa, _ = oracle.aniso(3, R, eps4, v)
            return 0.5 * aa * aa * float(v @ v)
        J = np.array([(e(gv + d * np.eye(3)[q]) - e(gv - d * np.eye(3)[q])) / (2 * d) for q in range(3)])
        _, jmg = oracle.aniso(3, R, eps4, gv)
        assert np.allclose(jmg + gv, J, rtol=1e-6, atol=1e-7)


def _smooth_fields(X, Y):
    psi = 0.8 * np.sin(0.7 * X + 0.3) + 0.5 * np.cos(0.45 * Y - 0.2) + 0.6 * X - 0.3 * Y
    return psi


def _err_rate(errs):
    return math.log(errs[0] / errs[1]) / math.log(2.0)


def test_anisotropy_divergence_converges(oracle):
    """div(J - grad psi) on the <10> face shell -> continuum, at O(h^2)."""
    th0 = math.radians(23.0)
    eps4 = 0.05
    R = synth.rot2d(23.0)
    errs = []
    L = 6.0
    for n in (24, 48):
        h = L / n
        X, Y = grid2(n + 1, h)
        psi = _smooth_fields(X, Y)
        p = oracle.params(nx=n + 1, ny=n + 1, h=h, eps4=eps4, bc=oracle.BC_MIRROR)
        N = oracle.apply(p, "aniso_n", psi, rot=R)

        def gradpsi(x, y):
            return np.array([0.8 * 0.7 * math.cos(0.7 * x + 0.3) + 0.6, -0.5 * 0.45 * math.sin(0.45 * y - 0.2) - 0.3])

        def Qfield(x, y):
            g = gradpsi(x, y)
            return _energy_grad_2d(g, th0, eps4) - g
        e = 0.0
        d = 1e-4
        for (i, j) in [(n // 2, n // 2), (n // 3, 2 * n // 3), (2 * n // 3, n // 4)]:
            x, y = i * h, j * h
            div = (Qfield(x + d, y)[0] - Qfield(x - d, y)[0]) / (2 * d) + (Qfield(x, y + d)[1] - Qfield(x, y - d)[1]) / (2 * d)
            e = max(e, abs(N[j, i] - div))
        errs.append(e)
    assert _err_rate(errs) > 1.7, errs


@pytest.mark.parametrize("op", ["at_21", "at_std2"])
def test_standard_antitrapping_converges(oracle, op):
    """App. B (A_{2,1}) and the <10> form converge to div(alpha grad b / |grad b|) at O(h^2)."""
    errs = []
    L = 5.0
    for n in (20, 40):
        h = L / n
        X, Y = grid2(n + 1, h)
        al = 1.0 + 0.3 * np.sin(0.8 * X) * np.cos(0.5 * Y)
        be = _smooth_fields(X, Y)
        p = oracle.params(nx=n + 1, ny=n + 1, h=h, bc=oracle.BC_MIRROR)
        A = oracle.apply(p, op, al, be)

        def flux(x, y):
            a = 1.0 + 0.3 * math.sin(0.8 * x) * math.cos(0.5 * y)
            g = np.array([0.8 * 0.7 * math.cos(0.7 * x + 0.3) + 0.6, -0.5 * 0.45 * math.sin(0.45 * y - 0.2) - 0.3])
            return a * g / np.linalg.norm(g)
        d = 1e-4
        e = 0.0
        for (i, j) in [(n // 2, n // 2), (n // 3, 2 * n // 3), (2 * n // 3, n // 3)]:
            x, y = i * h, j * h
            div = (flux(x + d, y)[0] - flux(x - d, y)[0]) / (2 * d) + (flux(x, y + d)[1] - flux(x, y - d)[1]) / (2 * d)
            e = max(e, abs(A[j, i] - div))
        errs.append(e)
    assert _err_rate(errs) > 1.7, errs


PLANAR = [("SBAR21", 2), ("S21", 2), ("S10", 2), ("SBAR120", 3), ("S100", 3)]


@pytest.mark.parametrize("scheme,dim", PLANAR)
def test_planar_interface_is_fixed_point(oracle, scheme, dim):
    """psi = -(n.r)/a_s(n), U = 0: L = 0, G = 1/a_s^2 and every face flux is
    the same, so d psi/dt = 0 and U stays 0 at cells away from the walls."""
    rng = np.random.default_rng(11)
    n = 10
    h = 0.8
    for _ in range(3):
        if dim == 2:
            R = synth.rot2d(rng.uniform(0, 90))
            t = rng.uniform(0, 2 * math.pi)
            nv = np.array([math.cos(t), math.sin(t), 0.0])
            X, Y = grid2(n, h)
            coords = [X, Y]
        else:
            R = synth.random_rot3(rng)
            nv = rng.normal(size=3)
            nv /= np.linalg.norm(nv)
            X, Y, Z = grid3(n, h)
            coords = [X, Y, Z]
        a, _ = oracle.aniso(dim, R, 0.02, nv)
        c0 = (n - 1) / 2 * h
        psi = -sum(nv[q] * (coords[q] - c0) for q in range(dim)) / a
        U = np.zeros_like(psi)
        p = oracle.params(dim=dim, nx=n, ny=n, nz=n, scheme=synth.SCHEMES[scheme], h=h, dt=0.02)
        g = np.zeros(psi.shape, np.int16)
        psi1, U1, rate = oracle.step(p, R, g, psi, U, 1, want_rate=True)
        assert np.max(np.abs(interior(rate, 2, dim))) < 1e-12
        assert np.max(np.abs(interior(U1, 3, dim))) < 1e-13


@pytest.mark.parametrize("scheme,dim", PLANAR)
def test_solute_conserved_with_noflux_walls(oracle, scheme, dim):
    """sum (1+k-(1-k)phi)(1+(1-k)U)/2 is constant to round-off (reading T1)."""
    rng = np.random.default_rng(12)
    n = 20 if dim == 2 else 10
    w = synth.free_dendrite_2d(n) if dim == 2 else synth.free_dendrite_3d(n)
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, 3)
    p = oracle.params(dim=dim, nx=n, ny=n, nz=n, scheme=synth.SCHEMES[scheme], h=w.h, dt=w.dt, k=w.k,
                      eps4=w.eps4, lam=w.lam, D=w.D)
    cen = np.zeros((3, 3))
    c0 = oracle.observe(p, rots, cen, g, psi, U)["solute"]
    psi1, U1 = oracle.step(p, rots, g, psi, U, 60)
    c1 = oracle.observe(p, rots, cen, g, psi1, U1)["solute"]
    assert abs(c1 - c0) / abs(c0) < 1e-13
    assert np.max(np.abs(psi1 - psi)) > 1e-3  # the state did evolve


@pytest.mark.parametrize("scheme,dim", [("SBAR21", 2), ("S10", 2), ("S21", 2), ("SBAR120", 3), ("S100", 3)])
def test_fourier_mode_decay_all_liquid(oracle, scheme, dim):
    """phi = -1 everywhere: U = cos(k.r) decays per step by 1 + dt D L(k) with
    L(k) the closed-form symbol of the scheme's Laplacian on a periodic grid."""
    n = 16
    h = 0.8
    dt = 0.02
    D = 6.267
    m = (1, 2, 1)
    kv = [2 * math.pi * m[q] / (n * h) for q in range(dim)]
    if dim == 2:
        X, Y = grid2(n, h)
        th = kv[0] * X + kv[1] * Y
    else:
        X, Y, Z = grid3(n, h)
        th = kv[0] * X + kv[1] * Y + kv[2] * Z
    c = [math.cos(kq * h) for kq in kv]
    if dim == 2:
        L10 = (2 * c[0] + 2 * c[1] - 4) / h ** 2
        L01 = (2 * math.cos((kv[0] + kv[1]) * h) + 2 * math.cos((kv[0] - kv[1]) * h) - 4) / (2 * h ** 2)
        sym = L10 if scheme == "S10" else 2 / 3 * L10 + 1 / 3 * L01
    else:
        L100 = (2 * sum(c) - 6) / h ** 2
        s = 0.0
        for a in range(3):
            for b in range(a + 1, 3):
                s += 2 * math.cos((kv[a] + kv[b]) * h) + 2 * math.cos((kv[a] - kv[b]) * h)
        L010 = (s - 12) / (4 * h ** 2)
        sym = L100 if scheme == "S100" else 1 / 3 * L100 + 2 / 3 * L010
    U = 0.05 * np.cos(th)
    psi = np.full(U.shape, -60.0)
    p = oracle.params(dim=dim, nx=n, ny=n, nz=n, scheme=synth.SCHEMES[scheme], h=h, dt=dt, D=D,
                      bc=oracle.BC_PERIODIC)
    g = np.zeros(U.shape, np.int16)
    _, U1 = oracle.step(p, np.eye(3), g, psi, U, 1)
    assert np.allclose(U1, (1 + dt * D * sym) * U, rtol=0, atol=1e-15)


@pytest.mark.parametrize("scheme", ["SBAR21", "S21", "S10"])
def test_lattice_symmetry_2d(oracle, scheme):
    """Transposing the grid or mirroring x maps the step exactly when alpha0 -> -alpha0."""
    rng = np.random.default_rng(13)
    n = 18
    w = synth.free_dendrite_2d(n)
    psi, U = synth.random_state(rng, w)
    th = 17.0
    p = oracle.params(nx=n, ny=n, scheme=synth.SCHEMES[scheme], h=w.h, dt=w.dt, k=w.k, eps4=0.05, lam=w.lam, D=w.D)
    g = np.zeros(psi.shape, np.int16)
    a1, b1 = oracle.step(p, synth.rot2d(th), g, psi, U, 4)
    a2, b2 = oracle.step(p, synth.rot2d(-th), g, psi.T.copy(), U.T.copy(), 4)
    assert np.allclose(a2.T, a1, rtol=0, atol=1e-11) and np.allclose(b2.T, b1, rtol=0, atol=1e-11)
    a3, b3 = oracle.step(p, synth.rot2d(-th), g, psi[:, ::-1].copy(), U[:, ::-1].copy(), 4)
    assert np.allclose(a3[:, ::-1], a1, rtol=0, atol=1e-11) and np.allclose(b3[:, ::-1], b1, rtol=0, atol=1e-11)
    # and a genuinely different orientation does not map
    a4, _ = oracle.step(p, synth.rot2d(th), g, psi.T.copy(), U.T.copy(), 4)
    assert np.max(np.abs(a4.T - a1)) > 1e-6


@pytest.mark.parametrize("scheme", ["SBAR120", "S100"])
def test_lattice_symmetry_3d(oracle, scheme):
    """Permuting lab axes by P maps the step exactly when R -> P R."""
    rng = np.random.default_rng(14)
    n = 9
    w = synth.free_dendrite_3d(n)
    psi, U = synth.random_state(rng, w)
    R = synth.random_rot3(rng)
    p = oracle.params(dim=3, nx=n, ny=n, nz=n, scheme=synth.SCHEMES[scheme], h=w.h, dt=w.dt, k=w.k, eps4=0.05,
                      lam=w.lam, D=w.D)
    g = np.zeros(psi.shape, np.int16)
    a1, b1 = oracle.step(p, R, g, psi, U, 3)
    # arrays are [z, y, x]; swap lab x <-> z: array transpose (2, 1, 0)
    P = np.array([[0, 0, 1], [0, 1, 0], [1, 0, 0]], float)
    a2, b2 = oracle.step(p, P @ R, g, psi.transpose(2, 1, 0).copy(), U.transpose(2, 1, 0).copy(), 3)
    assert np.allclose(a2.transpose(2, 1, 0), a1, rtol=0, atol=1e-11)
    assert np.allclose(b2.transpose(2, 1, 0), b1, rtol=0, atol=1e-11)


def test_one_dimensional_profile_relaxes_to_tanh(oracle):
    """Sec. 2.3: the stationary 1D profile is phi = -tanh(x / sqrt 2), i.e.
    psi = -x; a perturbed psi relaxes back towards it (U = 0, eps4 = 0)."""
    n = 64
    h = 0.5
    x = (np.arange(n) - (n - 1) / 2) * h
    X = np.tile(x, (6, 1))
    psi0 = -X
    pert = 0.3 * np.exp(-X ** 2 / 4)
    p = oracle.params(nx=n, ny=6, h=h, dt=0.02, eps4=0.0, bc=oracle.BC_MIRROR)
    g = np.zeros(X.shape, np.int16)
    U = np.zeros(X.shape)
    psi1, _ = oracle.step(p, np.eye(3), g, psi0 + pert, U, 2000)
    mid = slice(8, n - 8)
    # profile recovers shape phi = -tanh((x - x0)/sqrt2) up to a shift x0
    phi = np.tanh(psi1[3, mid] / math.sqrt(2))
    x0 = np.interp(0.0, -psi1[3, mid], x[mid])
    want = -np.tanh((x[mid] - x0) / math.sqrt(2))
    assert np.max(np.abs(phi - want)) < 2e-3
    assert np.max(np.abs((psi0 + pert)[3, mid] / math.sqrt(2) - 0)) > 0  # sanity


def test_init_seeds_signed_distance_and_voronoi(oracle):
    n = 30
    h = 0.5
    p = oracle.params(nx=n, ny=n, h=h)
    seeds = np.array([[4.0, 4.0, 0, 2.0], [10.0, 9.0, 0, 3.0]])
    psi, U, g = oracle.init_seeds(p, -0.4, seeds, np.array([3, 1], np.int16))
    X, Y = grid2(n, h)
    d0 = 2.0 - np.hypot(X - 4, Y - 4)
    d1 = 3.0 - np.hypot(X - 10, Y - 9)
    assert np.allclose(psi, np.maximum(d0, d1), atol=1e-14)
    assert np.all(g == np.where(d1 > d0, 1, 3))
    assert np.all(U == -0.4)


def test_observe_closed_forms(oracle):
    n = 41
    h = 0.8
    p = oracle.params(nx=n, ny=n, h=h, k=0.15)
    c = (20 * h, 20 * h)
    X, Y = grid2(n, h)
    r = 7.3
    psi = r - np.hypot(X - c[0], Y - c[1])
    U = np.full(psi.shape, -0.3)
    g = np.zeros(psi.shape, np.int16)
    o = oracle.observe(p, synth.rot2d(0.0), np.array([[c[0], c[1], 0]]), g, psi, U, 0)
    assert o["found"] == 1
    assert abs(o["tip_x"] - c[0]) < 1e-12 and abs(o["tip_y"] - (c[1] + r)) < 1e-12
    assert abs(o["angle_xy_deg"]) < 1e-9
    phi = np.tanh(psi / math.sqrt(2))
    sol = np.sum((1 + 0.15 - 0.85 * phi) * (1 + 0.85 * U) / 2) * h * h
    assert abs(o["solute"] - sol) < 1e-12 * abs(sol)
    # uniform liquid: closed form (1 + (1-k)) ... with phi = -1 exactly
    liq = oracle.observe(p, synth.rot2d(0.0), np.array([[c[0], c[1], 0]]), g, np.full(psi.shape, -80.0), U, 0)
    assert abs(liq["solute"] - n * n * h * h * (1 + 0.85 * -0.3)) < 1e-9
    assert liq["found"] == 0
    # rotated growth axis: tip angle follows alpha0 to within the lattice resolution
    for th in (10.0, 30.0, -20.0):
        o = oracle.observe(p, synth.rot2d(th), np.array([[c[0], c[1], 0]]), g, psi, U, 0)
        assert abs(o["angle_xy_deg"] - th) < math.degrees(h / r)


@pytest.mark.parametrize("scheme,dim", PLANAR)
def test_antitrapping_moves_solute_from_solid_to_liquid(oracle, scheme, dim):
    """Sec. 2.3: the anti-trapping current (1+(1-k)U) d phi/dt n / sqrt2 with
    n = grad psi / |grad psi| (Eq. Anti_convention; Anti_approx for the barred
    schemes) carries solute out of an advancing solid into the liquid: for a
    planar interface psi = -(x - x0) advancing into a uniformly supersaturated
    liquid, its divergence A is negative on the solid side, positive on the
    liquid side, sums to zero, and equals (1+(1-k)U) / sqrt2 * (-d/dx dphi/dt)
    (unit |grad psi|).  With U uniform the diffusion term vanishes, so one step
    of the U equation isolates A:  A dt = (U' - U)(1+k-(1-k)phi') - (1+(1-k)U) dphi."""
    n, h, dt, k, U0 = 96, 0.25, 0.002, 0.15, -0.5
    x = np.arange(n) * h
    x0 = (n - 1) / 2 * h + 0.13
    shape = (6, n) if dim == 2 else (4, 4, n)
    psi = np.broadcast_to(-(x - x0), shape).copy()
    U = np.full(shape, U0)
    p = oracle.params(dim=dim, nx=n, ny=shape[-2], nz=shape[0] if dim == 3 else 1, scheme=synth.SCHEMES[scheme],
                      h=h, dt=dt, k=k, eps4=0.0, lam=10.0, D=6.267)
    g = np.zeros(shape, np.int16)
    psi1, U1 = oracle.step(p, np.eye(3), g, psi, U, 1)
    line = (3,) if dim == 2 else (2, 2)
    phi0 = np.tanh(psi[line] / math.sqrt(2))
    phi1 = np.tanh(psi1[line] / math.sqrt(2))
    dphi = phi1 - phi0
    A = ((U1[line] - U0) * (1 + k - (1 - k) * phi1) - (1 + (1 - k) * U0) * dphi) / dt
    inner = slice(10, n - 10)
    assert np.all(dphi[inner] >= 0) and dphi.max() > 1e-5  # the interface advances
    solid, liquid = x[inner] < x0, x[inner] > x0
    assert abs(A[inner].sum()) < 1e-9 * np.abs(A[inner]).sum()
    assert A[inner][solid].sum() < -0.4 * np.abs(A[inner]).sum()
    assert A[inner][liquid].sum() > 0.4 * np.abs(A[inner]).sum()
    want = (1 + (1 - k) * U0) / math.sqrt(2) * -np.gradient(dphi / dt, h)
    assert np.max(np.abs(A[inner] - want[inner])) < 0.03 * np.max(np.abs(want[inner]))
