"""GPU parity of the fused 3D step (S-bar_{1,2,0}, S_{1,0,0}) through the C-ABI
against the FP64 oracle.  Same tolerances as the 2D tests: FP64 1e-12 relative
per step; FP32 one step from an FP32-representable state 2e-6 on phi, 5e-6 on U.
Grids span several tiles in x and y (ragged last tiles) and several sweeps in z.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import max_abs, oracle_params, rel_err

pytestmark = pytest.mark.gpu

SCHEMES_3D = ["SBAR120", "S100"]


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    return N


def make_state(seed, nx, ny, nz, n_grains=3, eps4=0.05):
    rng = np.random.default_rng(seed)
    w = synth.free_dendrite_3d(nx, eps4=eps4)
    w.ny, w.nz = ny, nz
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, n_grains)
    return w, psi, U, g, rots


def gpu_sim(N, w, scheme, prec, g, rots, psi, U, tile=None):
    p = N.make_params(3, w.nx, w.ny, w.nz, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, scheme, prec,
                      max_grains=rots.shape[0])
    s = N.Sim(p)
    if tile:
        s.set_tile(*tile)
    s.set_grains(rots)
    s.set_grain_index(g)
    s.set_fields(psi, U)
    return s


@pytest.mark.parametrize("prec,tile", [("f64", None), ("f64", (34, 10, 8))])
@pytest.mark.parametrize("scheme", SCHEMES_3D)
def test_fp64_one_step_matches_oracle(native, scheme, prec, tile):
    w, psi, U, g, rots = make_state(1, 70, 33, 40)
    s = gpu_sim(native, w, scheme, prec, g, rots, psi, U, tile)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, scheme), rots, g, psi, U, 1)
    assert rel_err(gp, op) < 1e-12
    assert rel_err(gu, ou) < 1e-12


@pytest.mark.parametrize("scheme", SCHEMES_3D)
def test_fp64_many_steps(native, scheme):
    w, psi, U, g, rots = make_state(2, 37, 21, 19)
    s = gpu_sim(native, w, scheme, "f64", g, rots, psi, U)
    s.step(12)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, scheme), rots, g, psi, U, 12)
    assert rel_err(gp, op) < 12e-12
    assert rel_err(gu, ou) < 12e-12


@pytest.mark.parametrize("tile", [None, (34, 10, 8)])
@pytest.mark.parametrize("scheme", SCHEMES_3D)
def test_fp32_one_step_matches_oracle(native, scheme, tile):
    w, psi, U, g, rots = make_state(3, 64, 40, 35)
    psi32, U32 = psi.astype(np.float32), U.astype(np.float32)
    s = gpu_sim(native, w, scheme, "f32", g, rots, psi32, U32, tile)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, scheme), rots, g, psi32.astype(np.float64), U32.astype(np.float64), 1)
    assert max_abs(np.tanh(gp.astype(np.float64) / math.sqrt(2)), np.tanh(op / math.sqrt(2))) < 2e-6
    assert max_abs(gu, ou) < 5e-6


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 9, 4), (31, 15, 7), (61, 29, 33)])
def test_small_and_ragged_grids_3d(native, shape):
    w, psi, U, g, rots = make_state(5, *shape, n_grains=2)
    s = gpu_sim(native, w, "SBAR120", "f64", g, rots, psi, U)
    s.step(2)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, "SBAR120"), rots, g, psi, U, 2)
    assert rel_err(gp, op) < 1e-11 and rel_err(gu, ou) < 1e-11


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_init_and_observe_3d(native, prec):
    rng = np.random.default_rng(9)
    w = synth.polycrystal_3d(rng, 48, 3)
    s = native.Sim.from_workload(w, prec)
    gp, gu = s.get_fields()
    gg = s.get_grain_index()
    op, ou, og = O.init_seeds(oracle_params(w), w.U0, w.seeds, w.seed_grain)
    assert np.array_equal(gg, og)
    assert np.array_equal(gp, op.astype(gp.dtype))
    s.step(20)
    psi, U = s.get_fields()
    po = oracle_params(w)
    for g in range(-2, w.n_grains):  # -2: the pulling axis +y
        a = s.observe(g)
        b = O.observe(po, w.rots, w.centres, gg, psi.astype(np.float64), U.astype(np.float64), g)
        assert a["found"] == int(b["found"]) and a["tip_index"] == int(b["tip_index"])
        assert a["tip"] == (b["tip_x"], b["tip_y"], b["tip_z"])
        assert abs(a["solute"] - b["solute"]) <= 1e-12 * abs(b["solute"])
        assert abs(a["angle_out_deg"] - b["angle_out_deg"]) <= 1e-9


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("scheme", SCHEMES_3D)
def test_solute_conserved_3d(native, prec, scheme):
    w = synth.free_dendrite_3d(40, scheme=scheme)
    s = native.Sim.from_workload(w, prec)
    c0 = s.observe()["solute"]
    s.step(100)
    c1 = s.observe()["solute"]
    assert abs(c1 - c0) / abs(c0) < (1e-12 if prec == "f64" else 2e-6)
