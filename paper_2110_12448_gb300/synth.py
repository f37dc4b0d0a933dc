"""Seeded synthetic inputs shaped like the paper's solidification runs.

This module holds no phase-field arithmetic: it only draws the problem
definitions (grid sizes, physical constants, seed positions and radii, grain
orientations as rotation matrices) that both the CUDA path and the CPU
oracle consume.  All randomness is ``numpy.random.default_rng(seed)``.

Orientation convention: a grain's rotation matrix maps crystal coordinates
to lab coordinates (row-major 3x3).  In 2D the crystal is turned by alpha0
counter-clockwise, so the crystal axis that starts on +y points at alpha0
from the y axis (the misorientation of Sec. 3.3.2).  In 3D the matrix is
Rz(phi1) Rx(Phi) Rz(phi2) (ZXZ Euler angles).

Workloads (sizes and physics of the isothermal free-dendrite runs):
  * ``free_dendrite_2d``   200 x 200, h = 0.8, dt = 0.02, k = 0.15,
    eps4 = 0.02, lambda = 10, D = 0.6267 lambda, U0 = -0.55, one seed of
    radius 10 h at the centre, one grain at theta = 0.
  * ``orientation_sweep_2d``  1024 x 1024, same physics, one run per
    theta in 0, 5, ..., 45 degrees.
  * ``free_dendrite_3d``   256^3, h = 0.8, dt = 0.9 h^2 / (6 D), sphere of
    radius 8 h at the centre, ZXZ Euler angles drawn from the seed.
  * ``polycrystal_batch_2d``  64 instances, sides uniform in 256..1536,
    3-12 seeds each of radius 8 h with orientations uniform in [0, 90).
  * ``request_stream``      Poisson arrivals of 2D (128..2048) and 3D
    (64..192) runs with 1-16 seeds, U0 in [-0.7, -0.4], 1000-20000 steps.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 2110_12448

# scheme names shared by the C-ABI enum and the oracle (same numbering)
SCHEMES = {"S10": 0, "S21": 1, "SBAR21": 2, "S100": 3, "SBAR120": 4}
A2 = 0.6267  # a2 of D = a1 a2 W / d0 in the workloads' rounding


def rot2d(theta_deg: float) -> np.ndarray:
    t = math.radians(theta_deg)
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_zxz(phi1: float, Phi: float, phi2: float) -> np.ndarray:
    def rz(a):
        c, s = math.cos(a), math.sin(a)
        return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])

    def rx(a):
        c, s = math.cos(a), math.sin(a)
        return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])

    return rz(phi1) @ rx(Phi) @ rz(phi2)


def random_rot3(rng: np.random.Generator) -> np.ndarray:
    """Uniformly distributed rotation: phi1, phi2 ~ U[0, 2 pi), cos(Phi) ~ U[-1, 1]."""
    phi1 = rng.uniform(0.0, 2.0 * math.pi)
    phi2 = rng.uniform(0.0, 2.0 * math.pi)
    Phi = math.acos(rng.uniform(-1.0, 1.0))
    return rot_zxz(phi1, Phi, phi2)


@dataclasses.dataclass
class Workload:
    """One simulation: grid, physics, seeds and grains."""
    dim: int
    nx: int
    ny: int
    nz: int
    h: float
    dt: float
    k: float
    eps4: float
    lam: float
    D: float
    U0: float
    scheme: str
    seeds: np.ndarray        # (n, 4): x, y, z, r in units of W
    seed_grain: np.ndarray   # (n,) int16
    rots: np.ndarray         # (n_grains, 9) crystal -> lab, row-major
    centres: np.ndarray      # (n_grains, 3) reference point of each grain
    steps: int = 1
    name: str = ""
    # directional solidification (frozen temperature along +y) and x walls
    bc_x: int = 0            # 0 mirror, 1 periodic
    thermal: int = 0         # 0 isothermal, 1 frozen gradient
    Vp: float = 0.0          # pulling speed (W / tau0)
    lT: float = 1.0          # thermal length (W)
    yT: float = 0.0          # isotherm T0 at t = 0 (W)
    psi_init: Optional[np.ndarray] = None  # explicit initial fields (else from the seeds)
    U_init: Optional[np.ndarray] = None

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)

    @property
    def n_grains(self) -> int:
        return int(self.rots.shape[0])

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.dim == 3 else (self.ny, self.nx)


def _physics_2d(**kw):
    lam = kw.get("lam", 10.0)
    d = dict(h=0.8, dt=0.02, k=0.15, eps4=0.02, lam=lam, D=A2 * lam, U0=-0.55)
    d.update(kw)
    return d


def free_dendrite_2d(n: int = 200, theta_deg: float = 0.0, scheme: str = "SBAR21", steps: int = 2000,
                     ny: Optional[int] = None, **phys) -> Workload:
    ny = n if ny is None else ny
    p = _physics_2d(**phys)
    c = ((n - 1) / 2 * p["h"], (ny - 1) / 2 * p["h"], 0.0)
    seeds = np.array([[c[0], c[1], 0.0, 10 * p["h"]]])
    return Workload(2, n, ny, 1, p["h"], p["dt"], p["k"], p["eps4"], p["lam"], p["D"], p["U0"], scheme,
                    seeds, np.zeros(1, np.int16), rot2d(theta_deg).reshape(1, 9), np.array([c]), steps,
                    f"free_dendrite_2d_{n}x{ny}_theta{theta_deg:g}_{scheme}")


def orientation_sweep_2d(n: int = 1024, scheme: str = "SBAR21", steps: int = 20000,
                         thetas=tuple(range(0, 50, 5))) -> List[Workload]:
    return [free_dendrite_2d(n, float(t), scheme, steps) for t in thetas]


A1 = 5.0 * math.sqrt(2.0) / 8.0  # a1 of d0 = a1 W / lambda (Sec. 2.1)


def paper_isothermal_2d(theta_deg: float = 0.0, scheme: str = "SBAR21", W_d0: float = 16.0, h: float = 1.2,
                        eps4: float = 0.014, k: float = 0.1, Omega: float = 0.43, side_d0: float = 1.5e4,
                        seed_d0: float = 50.0, t_d0: float = 1.5e6) -> Workload:
    """The isothermal runs behind Sec. 4.3.2 (Figs. of alpha/alpha0 and sigma*
    vs alpha0, and the scheme timings of Table 1): a circular seed of radius
    50 d0* at the centre of a square box of side 1.5e4 d0* with no-flux
    walls, melt at scaled supersaturation Omega = 0.43, W/d0* = 16, h/W = 1.2,
    eps4 = 0.014, k = 0.1 (the paper's k throughout), dt = 0.8 h^2 / (4 D),
    run to t = 1.5e6 d0*^2 / D.  d0* = d0 (1 - (1-k) Omega) / k with
    d0 = a1 W / lambda fixes lambda; D = a2 lambda; U0 = -Omega.
    Defaults: a 781^2 grid and 20 345 steps."""
    lam = W_d0 * A1 * (1.0 - (1.0 - k) * Omega) / k
    D = A2 * lam
    dt = 0.8 * h * h / (4.0 * D)
    d0s = 1.0 / W_d0  # d0* in units of W
    n = int(round(side_d0 * d0s / h))
    steps = int(round(t_d0 * d0s * d0s / D / dt))
    c = ((n - 1) / 2 * h, (n - 1) / 2 * h, 0.0)
    seeds = np.array([[c[0], c[1], 0.0, seed_d0 * d0s]])
    return Workload(2, n, n, 1, h, dt, k, eps4, lam, D, -Omega, scheme, seeds, np.zeros(1, np.int16),
                    rot2d(theta_deg).reshape(1, 9), np.array([c]), steps,
                    f"paper_isothermal_2d_{n}^2_theta{theta_deg:g}_{scheme}")


def paper_isothermal_3d(theta_deg: float = 0.0, scheme: str = "SBAR120", n: int = 192, W_d0: float = 16.0,
                        h: float = 1.2, eps4: float = 0.014, k: float = 0.1, Omega: float = 0.25,
                        seed_d0: float = 50.0, t_d0: float = 1.5e6, steps: Optional[int] = None) -> Workload:
    """The isothermal 3D runs behind Sec. 6.2.2 (alpha/alpha0 and sigma* vs
    alpha0, Table 2): a spherical seed of radius 50 d0* at the centre of a cube
    with no-flux walls, Omega = 0.25, W/d0* = 16, h/W = 1.2, eps4 = 0.014,
    k = 0.1, dt = 0.8 h^2 / (6 D), the crystal turned by theta about z, run to
    t = 1.5e6 d0*^2 / D (about 30 500 steps).  The paper's cube of side
    9.6e4 d0* (5000^3 cells) does not fit one GPU; the side here is n cells
    (default 192 = 230 W = 3690 d0*), and `steps` can shorten the run."""
    lam = W_d0 * A1 * (1.0 - (1.0 - k) * Omega) / k
    D = A2 * lam
    dt = 0.8 * h * h / (6.0 * D)
    d0s = 1.0 / W_d0
    if steps is None:
        steps = int(round(t_d0 * d0s * d0s / D / dt))
    c = ((n - 1) / 2 * h,) * 3
    seeds = np.array([[c[0], c[1], c[2], seed_d0 * d0s]])
    return Workload(3, n, n, n, h, dt, k, eps4, lam, D, -Omega, scheme, seeds, np.zeros(1, np.int16),
                    rot2d(theta_deg).reshape(1, 9), np.array([c]), steps,
                    f"paper_isothermal_3d_{n}^3_theta{theta_deg:g}_{scheme}")


def free_dendrite_3d(n: int = 256, scheme: str = "SBAR120", steps: int = 10000, seed: int = SEED_BASE + 2,
                     **phys) -> Workload:
    p = _physics_2d(**phys)
    p["dt"] = phys.get("dt", 0.9 * p["h"] ** 2 / (6 * p["D"]))
    rng = np.random.default_rng(seed)
    R = random_rot3(rng)
    c = ((n - 1) / 2 * p["h"],) * 3
    seeds = np.array([[c[0], c[1], c[2], 8 * p["h"]]])
    return Workload(3, n, n, n, p["h"], p["dt"], p["k"], p["eps4"], p["lam"], p["D"], p["U0"], scheme, seeds,
                    np.zeros(1, np.int16), R.reshape(1, 9), np.array([c]), steps, f"free_dendrite_3d_{n}^3_{scheme}")


def directional_2d(nx: int = 256, ny: int = 512, theta_deg: float = 0.0, scheme: str = "SBAR21",
                   Vp: float = 0.1, lT: float = 500.0, steps: int = 5000, seed: int = SEED_BASE + 5,
                   modes: int = 6, amp: float = 0.5, **phys) -> Workload:
    """Directional solidification of one grain (crystal turned by theta from the
    pulling axis +y) in a frozen temperature field, periodic in x (Sec. 4.2):
    a planar front on the isotherm T0 at y = yT = ny h / 8, perturbed by a few
    seeded sine modes of amplitude `amp` (W); U = 0 in the solid and the steady
    diffusion profile -1 + exp(-Vp (y - y_front) / D) ahead of it (U = -1 far
    away: c_l0 = c_inf / k at T0)."""
    p = _physics_2d(U0=-1.0, **phys)
    rng = np.random.default_rng(seed)
    h = p["h"]
    yT = ny * h / 8.0
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    front = np.full(nx, yT)
    Lx = nx * h
    for m in range(1, modes + 1):
        front += amp / math.sqrt(modes) * np.sin(2 * math.pi * m * x / Lx + rng.uniform(0, 2 * math.pi))
    eta = y[:, None] - front[None, :]
    psi = -eta
    U = np.where(eta < 0, 0.0, -1.0 + np.exp(-Vp * np.maximum(eta, 0.0) / p["D"]))
    c = (Lx / 2, 0.0, 0.0)
    return Workload(2, nx, ny, 1, h, p["dt"], p["k"], p["eps4"], p["lam"], p["D"], p["U0"], scheme,
                    np.array([[c[0], -100.0 * h, 0.0, h]]), np.zeros(1, np.int16), rot2d(theta_deg).reshape(1, 9),
                    np.array([c]), steps, f"directional_2d_{nx}x{ny}_{theta_deg:g}deg_{scheme}",
                    bc_x=1, thermal=1, Vp=Vp, lT=lT, yT=yT, psi_init=psi, U_init=U)


def paper_directional_2d(theta_deg: float = 0.0, scheme: str = "SBAR21", W_d0: float = 110.4, h: float = 1.2,
                         eps4: float = 0.014, k: float = 0.1, dt_s: float = 1e-5, D_um2_s: float = 1270.0,
                         Vp_um_s: float = 86.0, G_K_cm: float = 19.0, m_K_wt: float = -3.02, c_inf_wt: float = 1.3,
                         Lx_um: float = 191.0, Ly_um: float = 491.0, finger_W: float = 150.0, finger_R: float = 5.0,
                         delta0: float = 0.03, steps: int = 400000) -> Workload:
    """The 2D directional-solidification runs of Sec. 4.3.3 (SCN-1.3 wt%
    acetone, Vp = 86 um/s, G = 19 K/cm, W/d0 = 110.4, h/W = 1.2, dt = 1e-5 s,
    eps4 = 0.014, k = 0.1, m = -3.02 K/wt%, D = 1270 um^2/s, a 191 x 491 um^2
    box periodic in x) in the model's units.  The paper does not give W (nor
    Gamma); the Delta t rule of its isothermal runs, dt = 0.8 h^2 / (4 D), with
    the stated dt fixes it: W = 0.210 um, d0 = 1.90 nm (its 3D runs give the
    same d0 by the 3D rule).  Then lambda = a1 W/d0, D~ = a2 lambda,
    tau0 = dt / dt~, Vp~ = Vp tau0 / W and lT~ = (|m| c_inf (1-k)/k) / (G W).

    Dendrite tips grow just below the liquidus of c_inf (zeta = 1, where
    U = -1 is in equilibrium), lT~ = 88 600 W above the solidus isotherm T0
    (zeta = 0), so the box is placed there: a planar front at y0 = Ly/8,
    `delta0` below the liquidus (zeta = 1 - delta0, yT = y0 - lT~ (1 - delta0)),
    with a finger of length `finger_W` and radius
    `finger_R` (W; psi = the signed distance to a capsule) along the crystal
    axis, turned by theta from the pulling axis, in a melt at c_inf (U = -1
    everywhere).  The finger
    grows into the dendrite whose tip the runs follow (pf_shift_frame keeps it
    inside the box)."""
    lam = A1 * W_d0
    D = A2 * lam
    dt = 0.8 * h * h / (4.0 * D)
    tau0 = dt_s / dt
    W_um = math.sqrt(D_um2_s * tau0 / D)
    Vp = Vp_um_s * tau0 / W_um
    lT = abs(m_K_wt) * c_inf_wt * (1.0 - k) / k / (G_K_cm * 1e-4) / W_um  # Delta T0 / G in units of W
    nx = int(round(Lx_um / (h * W_um)))
    ny = int(round(Ly_um / (h * W_um)))
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    X, Y = np.meshgrid(x, y, indexing="xy")
    y0 = ny * h / 8.0
    xc = nx * h / 2.0
    t = math.radians(theta_deg)
    ax, ay = -math.sin(t), math.cos(t)  # crystal axis (+y turned counter-clockwise by theta)
    Lx = nx * h
    dist = np.full(X.shape, np.inf)
    for img in (-Lx, 0.0, Lx):  # the capsule and its periodic images: psi stays periodic in x
        s_ = np.clip((X - xc - img) * ax + (Y - y0) * ay, 0.0, finger_W)  # nearest point of the finger's axis
        dist = np.minimum(dist, np.hypot(X - (xc + img + s_ * ax), Y - (y0 + s_ * ay)))
    psi = np.maximum(-(Y - y0), finger_R - dist)  # signed distance to front + capsule
    U = np.full((ny, nx), -1.0)
    c = (xc, y0, 0.0)
    return Workload(2, nx, ny, 1, h, dt, k, eps4, lam, D, -1.0, scheme,
                    np.array([[xc, -100.0 * h, 0.0, h]]), np.zeros(1, np.int16), rot2d(theta_deg).reshape(1, 9),
                    np.array([c]), steps, f"paper_directional_2d_{nx}x{ny}_theta{theta_deg:g}_{scheme}",
                    bc_x=1, thermal=1, Vp=Vp, lT=lT, yT=y0 - lT * (1.0 - delta0), psi_init=psi, U_init=U)


def place_seeds(rng: np.random.Generator, dim: int, extent, n_seeds: int, r: float, tries: int = 1000):
    """Rejection sampling: centres >= 2r from the walls and >= 4r apart;
    after `tries` failures the radius shrinks by 0.8 and placement restarts."""
    while True:
        while any(e < 4 * r for e in extent[:dim]):
            r *= 0.8  # the box cannot hold a centre 2r from both walls
        out = []
        fails = 0
        while len(out) < n_seeds and fails < tries:
            c = [rng.uniform(2 * r, e - 2 * r) for e in extent[:dim]]
            if all(math.dist(c, o[:dim]) >= 4 * r for o in out):
                out.append(c + [0.0] * (3 - dim))
            else:
                fails += 1
        if len(out) == n_seeds:
            return np.array(out), r
        r *= 0.8


def polycrystal_2d(rng: np.random.Generator, n: int, n_seeds: int, scheme="SBAR21", steps=5000, U0=-0.55,
                   name="") -> Workload:
    p = _physics_2d(U0=U0)
    ext = ((n - 1) * p["h"], (n - 1) * p["h"])
    centres, r = place_seeds(rng, 2, ext, n_seeds, 8 * p["h"])
    seeds = np.concatenate([centres, np.full((n_seeds, 1), r)], axis=1)
    rots = np.stack([rot2d(rng.uniform(0.0, 90.0)).reshape(9) for _ in range(n_seeds)])
    return Workload(2, n, n, 1, p["h"], p["dt"], p["k"], p["eps4"], p["lam"], p["D"], p["U0"], scheme, seeds,
                    np.arange(n_seeds, dtype=np.int16), rots, centres, steps, name or f"poly2d_{n}")


def polycrystal_3d(rng: np.random.Generator, n: int, n_seeds: int, scheme="SBAR120", steps=1000, U0=-0.55,
                   name="") -> Workload:
    p = _physics_2d(U0=U0)
    p["dt"] = 0.9 * p["h"] ** 2 / (6 * p["D"])
    ext = ((n - 1) * p["h"],) * 3
    centres, r = place_seeds(rng, 3, ext, n_seeds, 8 * p["h"])
    seeds = np.concatenate([centres, np.full((n_seeds, 1), r)], axis=1)
    rots = np.stack([random_rot3(rng).reshape(9) for _ in range(n_seeds)])
    return Workload(3, n, n, n, p["h"], p["dt"], p["k"], p["eps4"], p["lam"], p["D"], p["U0"], scheme, seeds,
                    np.arange(n_seeds, dtype=np.int16), rots, centres, steps, name or f"poly3d_{n}")


def polycrystal_batch_2d(n_instances: int = 64, lo: int = 256, hi: int = 1536, steps: int = 5000,
                         seed: int = SEED_BASE + 3) -> List[Workload]:
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_instances):
        n = int(rng.integers(lo, hi + 1))
        ns = int(rng.integers(3, 13))
        out.append(polycrystal_2d(rng, n, ns, steps=steps, name=f"poly2d_{b}_{n}"))
    return out


@dataclasses.dataclass
class Request:
    arrival_s: float
    workload: Workload


def request_stream(rate_per_s: float = 20.0, window_s: float = 60.0, seed: int = SEED_BASE + 4,
                   size_scale: float = 1.0, steps_scale: float = 1.0) -> List[Request]:
    """Poisson arrivals; half 2D (side 128..2048), half 3D (side 64..192).
    size_scale / steps_scale shrink sides and step counts for short runs."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t > window_s:
            return out
        ns = int(rng.integers(1, 17))
        U0 = float(rng.uniform(-0.7, -0.4))
        steps = max(1, int(int(rng.integers(1000, 20001)) * steps_scale))
        if rng.uniform() < 0.5:
            n = max(32, int(int(rng.integers(128, 2049)) * size_scale))
            w = polycrystal_2d(rng, n, ns, steps=steps, U0=U0, name=f"req{len(out)}_2d_{n}")
        else:
            n = max(16, int(int(rng.integers(64, 193)) * size_scale))
            w = polycrystal_3d(rng, n, ns, steps=steps, U0=U0, name=f"req{len(out)}_3d_{n}")
        out.append(Request(t, w))


def random_state(rng: np.random.Generator, w: Workload, n_bumps: int = 6):
    """A smooth random (psi, U) pair with interfaces, for parity tests that
    start away from the seed state: psi = max of random discs plus a smooth
    perturbation, U = U0 plus a smooth perturbation in [-0.2, 0.2]."""
    shape = w.shape
    axes = [np.arange(s) * w.h for s in shape[::-1]]
    grids = np.meshgrid(*axes, indexing="xy") if w.dim == 2 else np.meshgrid(*axes, indexing="ij")
    if w.dim == 3:
        X, Y, Z = np.meshgrid(*axes, indexing="ij")
        X, Y, Z = X.transpose(2, 1, 0), Y.transpose(2, 1, 0), Z.transpose(2, 1, 0)
        coords = [X, Y, Z]
    else:
        X, Y = grids
        coords = [X, Y]
    ext = [s * w.h for s in shape[::-1]]
    psi = np.full(shape, -1e9)
    for _ in range(n_bumps):
        c = [rng.uniform(0.2 * e, 0.8 * e) for e in ext]
        r = rng.uniform(0.1, 0.3) * min(ext)
        d = np.sqrt(sum((coords[a] - c[a]) ** 2 for a in range(w.dim)))
        psi = np.maximum(psi, r - d)
    pert = np.zeros(shape)
    U = np.full(shape, w.U0)
    for _ in range(3):
        kv = [rng.uniform(-1, 1) * 2 * math.pi / e * 2 for e in ext]
        ph = rng.uniform(0, 2 * math.pi)
        arg = sum(kv[a] * coords[a] for a in range(w.dim)) + ph
        pert += rng.uniform(0.2, 0.6) * np.sin(arg)
        U += rng.uniform(0.02, 0.07) * np.cos(arg * 0.7 + 1.0)
    return psi + pert, U


def random_grains(rng: np.random.Generator, w: Workload, n_grains: int):
    """Voronoi-free random blocky grain map and random rotations (for tests
    of the per-cell grain lookup)."""
    shape = w.shape
    g = np.zeros(shape, np.int16)
    blk = 5
    idx = rng.integers(0, n_grains, size=tuple((s + blk - 1) // blk for s in shape)).astype(np.int16)
    sl = np.kron(idx, np.ones((blk,) * len(shape), np.int16))
    g[...] = sl[tuple(slice(0, s) for s in shape)]
    if w.dim == 2:
        rots = np.stack([rot2d(rng.uniform(0, 90)).reshape(9) for _ in range(n_grains)])
    else:
        rots = np.stack([random_rot3(rng).reshape(9) for _ in range(n_grains)])
    return g, rots
