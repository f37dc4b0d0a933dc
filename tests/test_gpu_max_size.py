"""Oracle parity at the largest grids, on sampled windows.

2D: 65536 x 32768 FP32 cells (2^31, beyond 32-bit cell indices; 38.7 GB of
state), S-bar_{2,1} with a crystal turned by 20 deg.  3D: 1024^3 FP32 cells
(1.07e9, 19 GB), S-bar_{1,2,0} with a random orientation.  The grid is liquid
(psi = -1e3, U = U0 as pf_create leaves it) except for seeded discs / spheres
written into windows at the four (eight) corners, where the mirror walls sit
at the largest indices, and at the centre.  After one step each window is
compared with the oracle's step on the window's initial state.  One step moves
information at most three cells (psi' on a one-cell ring, the anti-trapping
term of psi' a ring further), so cells at least three cells inside the
window's interior edges are exact; on the grid's own walls the oracle's mirror
is the grid's.  Tolerance: the one-step FP32 bounds (phi 2e-6, U 5e-6)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import max_abs

pytestmark = pytest.mark.gpu

HALO = 3


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    return N


def _view(N, sim, which):
    """torch view (on the device) of the current psi or U of a handle."""
    import torch
    psi_p, u_p, _ = sim.device_fields()
    off = (psi_p if which == "psi" else u_p) - sim.mem.data_ptr()
    n = int(np.prod(sim.shape))
    return sim.mem[off:off + 4 * n].view(torch.float32).view(*sim.shape)


def _phi(p):
    return np.tanh(np.asarray(p, np.float64) / math.sqrt(2.0))


def _windows(shape, w):
    """window origins: every corner and the centre"""
    dims = len(shape)
    out = []
    for corner in np.ndindex(*(2,) * dims):
        out.append(tuple(0 if c == 0 else shape[a] - w for a, c in enumerate(corner)))
    out.append(tuple(s // 2 - w // 2 for s in shape))
    return out


def _seed_window(shape_w, h, rng, dim):
    """signed distance to a few discs/spheres inside a window (psi), U0 +- 0.05"""
    axes = np.meshgrid(*[np.arange(n) * h for n in shape_w], indexing="ij")
    psi = np.full(shape_w, -1e3)
    for _ in range(3):
        c = [rng.uniform(0.25, 0.75) * n * h for n in shape_w]
        r = rng.uniform(0.08, 0.2) * min(shape_w) * h
        d = np.sqrt(sum((axes[a] - c[a]) ** 2 for a in range(dim)))
        psi = np.maximum(psi, r - d)
    return psi


def _check(N, sim, w, p_oracle_kw, rots, dim, win, seed):
    import torch
    rng = np.random.default_rng(seed)
    shape = sim.shape
    origins = _windows(shape, win)
    psi_v, u_v = _view(N, sim, "psi"), _view(N, sim, "U")
    inits = []
    for k, o in enumerate(origins):
        sl = tuple(slice(o[a], o[a] + win) for a in range(dim))
        p0 = _seed_window((win,) * dim, w.h, rng, dim).astype(np.float32)
        u0 = (w.U0 + 0.05 * rng.uniform(-1, 1, size=(win,) * dim)).astype(np.float32)
        psi_v[sl] = torch.from_numpy(p0).cuda()
        u_v[sl] = torch.from_numpy(u0).cuda()
        inits.append((sl, p0, u0))
    torch.cuda.synchronize()
    sim.step(1)
    psi_v, u_v = _view(N, sim, "psi"), _view(N, sim, "U")
    for (sl, p0, u0), o in zip(inits, origins):
        gp = psi_v[sl].cpu().numpy()
        gu = u_v[sl].cpu().numpy()
        po = O.params(**dict(p_oracle_kw, nx=win, ny=win, nz=win if dim == 3 else 1))
        op, ou = O.step(po, rots, np.zeros(p0.shape, np.int16), p0.astype(np.float64), u0.astype(np.float64), 1)
        # exact cells: HALO away from every window edge that is not a wall of the grid
        inner = []
        for a in range(dim):
            lo = 0 if o[a] == 0 else HALO
            hi = win if o[a] + win == shape[a] else win - HALO
            inner.append(slice(lo, hi))
        inner = tuple(inner)
        assert max_abs(_phi(gp[inner]), _phi(op[inner])) < 2e-6, o
        assert max_abs(gu[inner], ou[inner]) < 5e-6, o


def test_2d_two_to_the_31_cells(native):
    import torch
    w = synth.free_dendrite_2d(64, theta_deg=20.0)
    nx, ny = 65536, 32768
    p = native.make_params(2, nx, ny, 1, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, "SBAR21", "f32")
    sim = native.Sim(p)
    sim.set_grains(w.rots)
    assert sim.n_cells == 2 ** 31
    kw = dict(dim=2, scheme=O.SBAR21, h=w.h, dt=w.dt, k=w.k, eps4=w.eps4, lam=w.lam, D=w.D)
    _check(native, sim, w, kw, w.rots, 2, 96, 11)
    o = sim.observe(-1)  # the FP64 reductions over 2^31 cells
    assert o["nonfinite"] == 0 and o["found"] == 1 and 0.0 < o["solid_fraction"] < 1e-4
    sim.close()
    torch.cuda.empty_cache()


def test_3d_1024_cube(native):
    import torch
    w = synth.free_dendrite_3d(64)
    n = 1024
    p = native.make_params(3, n, n, n, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, "SBAR120", "f32")
    sim = native.Sim(p)
    sim.set_grains(w.rots)
    sim.set_tile(34, 18, 32)
    kw = dict(dim=3, scheme=O.SBAR120, h=w.h, dt=w.dt, k=w.k, eps4=w.eps4, lam=w.lam, D=w.D)
    _check(native, sim, w, kw, w.rots, 3, 40, 12)
    o = sim.observe(-1)
    assert o["nonfinite"] == 0 and o["found"] == 1 and 0.0 < o["solid_fraction"] < 1e-3
    sim.close()
    torch.cuda.empty_cache()
