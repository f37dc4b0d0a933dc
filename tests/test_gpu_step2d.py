"""GPU parity of the fused 2D step (through the C-ABI) against the FP64 oracle.

Tolerances:
  * FP64 build: 1e-12 relative per step (max over cells of |d| / max(1, |x|)),
    the figure the design targets for an FP64 GPU build.
  * FP32 build, one step from an FP32-representable state: FP32 rounding of
    psi (|psi| up to ~1e2 in the bulk, ulp 8e-6) and of the rates; compared on
    phi = tanh(psi/sqrt2): 2e-6 absolute.  U: the hardware exp2/reciprocal
    form of tanh errs by <= 2.5e-7 per evaluation, delta phi by <= 5e-7, and U'
    divides it by 1+k-(1-k)phi' >= 2k = 0.3: 5e-6 absolute.
  * Integer decisions (grain map, tip cell) are bit-exact.
Grids span several tiles in x (ragged last strip) and several sweeps in y.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import max_abs, oracle_params, rel_err

pytestmark = pytest.mark.gpu

SCHEMES_2D = ["SBAR21", "S21", "S10"]


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    return N


def make_state(seed, nx, ny, n_grains=3, eps4=0.05):
    rng = np.random.default_rng(seed)
    w = synth.free_dendrite_2d(nx, ny=ny, eps4=eps4)
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, n_grains)
    return w, psi, U, g, rots


def gpu_sim(N, w, scheme, prec, g, rots, psi, U, tile=None):
    p = N.make_params(2, w.nx, w.ny, 1, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, scheme, prec,
                      max_grains=rots.shape[0])
    s = N.Sim(p)
    if tile:
        s.set_tile(*tile)
    s.set_grains(rots)
    s.set_grain_index(g)
    s.set_fields(psi, U)
    return s


@pytest.mark.parametrize("scheme", SCHEMES_2D)
def test_fp64_one_step_matches_oracle(native, scheme):
    w, psi, U, g, rots = make_state(1, 261, 150)
    s = gpu_sim(native, w, scheme, "f64", g, rots, psi, U)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, scheme, eps4=w.eps4), rots, g, psi, U, 1)
    assert rel_err(gp, op) < 1e-12
    assert rel_err(gu, ou) < 1e-12


@pytest.mark.parametrize("scheme", SCHEMES_2D)
def test_fp64_many_steps_stay_within_roundoff(native, scheme):
    w, psi, U, g, rots = make_state(2, 133, 77)
    s = gpu_sim(native, w, scheme, "f64", g, rots, psi, U)
    s.step(40)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, scheme), rots, g, psi, U, 40)
    assert rel_err(gp, op) < 40e-12
    assert rel_err(gu, ou) < 40e-12


@pytest.mark.parametrize("scheme", SCHEMES_2D)
def test_fp32_one_step_matches_oracle(native, scheme):
    w, psi, U, g, rots = make_state(3, 200, 131)
    psi32, U32 = psi.astype(np.float32), U.astype(np.float32)
    s = gpu_sim(native, w, scheme, "f32", g, rots, psi32, U32)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, scheme), rots, g, psi32.astype(np.float64), U32.astype(np.float64), 1)
    phi_g = np.tanh(gp.astype(np.float64) / math.sqrt(2))
    phi_o = np.tanh(op / math.sqrt(2))
    assert max_abs(phi_g, phi_o) < 2e-6
    assert max_abs(gu, ou) < 5e-6


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("scheme", SCHEMES_2D)
def test_tile_shape_does_not_change_results(native, scheme, prec):
    """Cutting the grid into work items of different sweep lengths changes
    only the rounding: the first row of a sweep recomputes the fluxes that
    later rows receive from their neighbours, at a different call site whose
    FMA contraction may differ."""
    w, psi, U, g, rots = make_state(4, 300, 90)
    if prec == "f32":
        psi, U = psi.astype(np.float32), U.astype(np.float32)
    outs = []
    for sweep in (8, 17, 64, 1000):
        s = gpu_sim(native, w, scheme, prec, g, rots, psi, U, (64, 1, sweep))
        s.step(5)
        outs.append(s.get_fields())
        s.close()
    tol = 2e-6 if prec == "f32" else 1e-13
    for o in outs[1:]:
        assert rel_err(o[0], outs[0][0]) < tol and rel_err(o[1], outs[0][1]) < tol


@pytest.mark.parametrize("nx,ny", [(4, 4), (4, 37), (41, 4), (5, 6), (125, 9), (124, 65), (129, 129)])
def test_small_and_ragged_grids(native, nx, ny):
    w, psi, U, g, rots = make_state(5, nx, ny, n_grains=2)
    s = gpu_sim(native, w, "SBAR21", "f64", g, rots, psi, U)
    s.step(3)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, "SBAR21"), rots, g, psi, U, 3)
    assert rel_err(gp, op) < 1e-11 and rel_err(gu, ou) < 1e-11


def test_zero_steps_and_invalid_calls(native):
    w, psi, U, g, rots = make_state(6, 32, 32)
    s = gpu_sim(native, w, "SBAR21", "f64", g, rots, psi, U)
    s.step(0)
    a, b = s.get_fields()
    assert np.array_equal(a, psi) and np.array_equal(b, U)
    with pytest.raises(native.PfError):
        s.step(-1)
    bad = g.copy()
    bad[0, 0] = 99
    with pytest.raises(native.PfError):
        s.set_grain_index(bad)
    with pytest.raises(native.PfError):
        s.set_grains(np.zeros((0, 9)))
    with pytest.raises(native.PfError):
        s.set_tile(100, 1, 64)  # no kernel compiled for that width
    p = native.make_params(2, 32, 32, scheme="SBAR21")
    import torch
    mem = torch.empty(16, dtype=torch.uint8, device="cuda")
    import ctypes as C
    h = C.c_void_p()
    rc = native.lib().pf_create(C.byref(p), C.c_void_p(mem.data_ptr()), 16, None, C.byref(h))
    assert rc == native.PF_ERR_BUDGET


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_init_seeds_matches_oracle_bitwise(native, prec):
    rng = np.random.default_rng(7)
    w = synth.polycrystal_2d(rng, 300, 7)
    s = native.Sim.from_workload(w, prec)
    gp, gu = s.get_fields()
    gg = s.get_grain_index()
    op, ou, og = O.init_seeds(oracle_params(w), w.U0, w.seeds, w.seed_grain)
    assert np.array_equal(gg, og)
    assert np.array_equal(gp, op.astype(gp.dtype))
    assert np.all(gu == np.asarray(w.U0, gu.dtype))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_observe_matches_oracle(native, prec):
    rng = np.random.default_rng(8)
    w = synth.polycrystal_2d(rng, 257, 5)
    s = native.Sim.from_workload(w, prec)
    s.step(30)
    psi, U = s.get_fields()
    gmap = s.get_grain_index()
    po = oracle_params(w)
    for g in range(-2, w.n_grains):  # -2: the pulling axis +y
        a = s.observe(g)
        b = O.observe(po, w.rots, w.centres, gmap, psi.astype(np.float64), U.astype(np.float64), g)
        assert a["found"] == int(b["found"])
        assert a["tip_index"] == int(b["tip_index"])
        for q, key in enumerate(["tip_x", "tip_y"]):
            assert a["tip"][q] == b[key]
        assert a["tip_score"] == b["score"]
        assert abs(a["solute"] - b["solute"]) <= 1e-12 * abs(b["solute"])
        assert abs(a["solid_fraction"] - b["solid_fraction"]) <= 1e-12
        assert abs(a["angle_xy_deg"] - b["angle_xy_deg"]) <= 1e-9


def test_observe_reports_nonfinite(native):
    w, psi, U, g, rots = make_state(9, 40, 40)
    psi[3, 5] = np.nan
    U[7, 7] = np.inf
    s = gpu_sim(native, w, "SBAR21", "f64", g, rots, psi, U)
    o = s.observe(-1, allow_nonfinite=True)
    assert o["status"] == native.PF_ERR_NONFINITE and o["nonfinite"] == 2


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_solute_conserved_on_gpu(native, prec):
    w = synth.free_dendrite_2d(128)
    s = native.Sim.from_workload(w, prec)
    c0 = s.observe()["solute"]
    s.step(500)
    c1 = s.observe()["solute"]
    tol = 1e-12 if prec == "f64" else 2e-6
    assert abs(c1 - c0) / abs(c0) < tol


def test_checkpoint_resume_bitwise(native):
    w = synth.free_dendrite_2d(150, theta_deg=20.0)
    a = native.Sim.from_workload(w, "f32")
    a.step(60)
    ref = a.get_fields()
    b = native.Sim.from_workload(w, "f32")
    b.step(31)
    psi, U = b.get_fields()
    c = native.Sim.from_workload(w, "f32", init=False)
    c.set_fields(psi, U)
    c.set_step(31)
    c.step(29)
    out = c.get_fields()
    assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
    assert c.steps_done == 60


def test_get_fields_into_pinned_buffers(native):
    # reading straight into caller (pinned) arrays gives the same fields as a fresh copy
    import torch
    w = synth.free_dendrite_2d(70, ny=33)
    s = native.Sim.from_workload(w, "f32")
    s.step(5)
    a, b = s.get_fields()
    hp = torch.empty(s.shape, dtype=torch.float32).pin_memory()
    hu = torch.empty(s.shape, dtype=torch.float32).pin_memory()
    s.get_fields(out=(hp.numpy(), hu.numpy()))
    assert np.array_equal(hp.numpy(), a) and np.array_equal(hu.numpy(), b)
    with pytest.raises(ValueError):
        s.get_fields(out=(np.zeros(s.shape, np.float64), np.zeros(s.shape, np.float64)))
