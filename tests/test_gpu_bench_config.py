"""Oracle parity in the launch configurations the benchmark and the autotuner
actually use.

2D: the orientation-sweep batch (ten 1024 x 1024 S-bar_{2,1} FP32 instances
at alpha0 = 0..45 deg, one persistent launch per step, replayed from CUDA
graphs) with the autotuned tile (64, 1, 38), after 200 steps from the seeds:
16 graph-replayed steps of every instance against 16 oracle steps from the same
FP32 state.  Tolerance: 16 times the one-step FP32 bounds of the other 2D
tests (phi 2e-6, U 5e-6 per step; no amplification over 16 steps).  And the
same tile in a ten-instance FP64 group on smaller random states and grains,
20 graph-replayed steps, 1e-12 relative per step.

3D: every tile the autotuner can pick ((34, 18) and (34, 10) blocks, i.e.
30 x 14 and 30 x 6 output columns, with 16-, 32- and 64-plane sweeps and a
wave-aligned odd sweep) one step against the oracle in FP64 (1e-12) and FP32
(the one-step bounds 2e-6 on phi, 5e-6 on U) on a grid spanning several
tiles with ragged edges; and the 256^3 free dendrite at its full size with
the autotuner's two tied tiles (34, 18, 32) and (34, 10, 52), one FP32 step from
its state after 40 steps.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import max_abs, oracle_params, rel_err

pytestmark = pytest.mark.gpu

S2 = math.sqrt(2.0)


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    return N


def _phi(p):
    return np.tanh(np.asarray(p, np.float64) / S2)


def test_sweep_batch_bench_tile_fp32(native):
    import torch
    st = torch.cuda.Stream()
    ws = [synth.free_dendrite_2d(1024, float(t), "SBAR21", steps=20000) for t in range(0, 50, 5)]
    sims = [native.Sim.from_workload(w, "f32", stream=st) for w in ws]
    for s in sims:
        s.set_tile(64, 1, 38)
    grp = native.Group(len(sims), sum(native.Group.work_items(s) for s in sims), stream=st)
    for s in sims:
        grp.add(s)
    grp.step(200, use_graph=True)
    st.synchronize()
    start = [s.get_fields() for s in sims]
    grp.step(16, use_graph=True)
    st.synchronize()
    for w, s, (p0, u0) in zip(ws, sims, start):
        gp, gu = s.get_fields()
        op, ou = O.step(oracle_params(w), w.rots, np.zeros(p0.shape, np.int16), p0.astype(np.float64),
                        u0.astype(np.float64), 16)
        assert max_abs(_phi(gp), _phi(op)) < 16 * 2e-6, w.name
        assert max_abs(gu, ou) < 16 * 5e-6, w.name
    grp.close()


def test_ten_instance_group_bench_tile_fp64(native):
    import torch
    st = torch.cuda.Stream()
    cases = []
    for i in range(10):
        rng = np.random.default_rng(100 + i)
        w = synth.free_dendrite_2d(140 + 13 * i, ny=90 + 7 * i, eps4=0.05)
        psi, U = synth.random_state(rng, w)
        g, rots = synth.random_grains(rng, w, 3)
        p = native.make_params(2, w.nx, w.ny, 1, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, "SBAR21", "f64",
                               max_grains=3)
        s = native.Sim(p, stream=st)
        s.set_tile(64, 1, 38)
        s.set_grains(rots)
        s.set_grain_index(g)
        s.set_fields(psi, U)
        cases.append((w, s, psi, U, g, rots))
    grp = native.Group(10, sum(native.Group.work_items(c[1]) for c in cases), stream=st)
    for c in cases:
        grp.add(c[1])
    grp.step(20, use_graph=True)
    st.synchronize()
    for w, s, psi, U, g, rots in cases:
        gp, gu = s.get_fields()
        op, ou = O.step(oracle_params(w, "SBAR21"), rots, g, psi, U, 20)
        assert rel_err(gp, op) < 20e-12 and rel_err(gu, ou) < 20e-12
    grp.close()


def _state3(seed, nx, ny, nz, n_grains=3):
    rng = np.random.default_rng(seed)
    w = synth.free_dendrite_3d(nx, eps4=0.05)
    w.ny, w.nz = ny, nz
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, n_grains)
    return w, psi, U, g, rots


def _sim3(N, w, scheme, prec, g, rots, psi, U, tile):
    p = N.make_params(3, w.nx, w.ny, w.nz, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, scheme, prec,
                      max_grains=rots.shape[0])
    s = N.Sim(p)
    s.set_tile(*tile)
    s.set_grains(rots)
    s.set_grain_index(g)
    s.set_fields(psi, U)
    return s


TILES_3D = [(34, 18, 16), (34, 18, 32), (34, 18, 64), (34, 18, 13), (34, 10, 16), (34, 10, 32), (34, 10, 64)]
# FP64 S-bar_{1,2,0} with the 30 x 14 tile needs 246 KB of shared memory, above
# the 227 KB per block: the library refuses that tile (the autotuner skips it)
TILES_3D_F64 = {"SBAR120": [t for t in TILES_3D if t[1] == 10], "S100": TILES_3D}


def test_fp64_wide_tile_refused_cleanly(native):
    w, psi, U, g, rots = _state3(40, 40, 20, 12)
    s = _sim3(native, w, "SBAR120", "f64", g, rots, psi, U, (34, 10, 16))
    with pytest.raises(native.PfError):
        s.set_tile(34, 18, 32)
    assert s.get_tile() == (34, 10, 16)
    s2 = _sim3(native, w, "SBAR120", "f64", g, rots, psi, U, (34, 10, 16))  # later calls are unaffected
    s2.step(1)
    op, ou = O.step(oracle_params(w, "SBAR120"), rots, g, psi, U, 1)
    gp, gu = s2.get_fields()
    assert rel_err(gp, op) < 1e-12 and rel_err(gu, ou) < 1e-12


@pytest.mark.parametrize("tile", TILES_3D)
@pytest.mark.parametrize("scheme", ["SBAR120", "S100"])
def test_autotuner_tiles_3d_fp64(native, scheme, tile):
    if tile not in TILES_3D_F64[scheme]:
        pytest.skip("tile needs more shared memory than a block may have in FP64")
    w, psi, U, g, rots = _state3(41, 67, 33, 70)
    s = _sim3(native, w, scheme, "f64", g, rots, psi, U, tile)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, scheme), rots, g, psi, U, 1)
    assert rel_err(gp, op) < 1e-12 and rel_err(gu, ou) < 1e-12


@pytest.mark.parametrize("tile", TILES_3D)
@pytest.mark.parametrize("scheme", ["SBAR120", "S100"])
def test_autotuner_tiles_3d_fp32(native, scheme, tile):
    w, psi, U, g, rots = _state3(42, 64, 37, 66)
    psi32, U32 = psi.astype(np.float32), U.astype(np.float32)
    s = _sim3(native, w, scheme, "f32", g, rots, psi32, U32, tile)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, scheme), rots, g, psi32.astype(np.float64), U32.astype(np.float64), 1)
    assert max_abs(_phi(gp), _phi(op)) < 2e-6
    assert max_abs(gu, ou) < 5e-6


@pytest.mark.parametrize("tile", [(34, 18, 32), (34, 10, 52)])
def test_dendrite_256_cube_bench_tile_fp32(native, tile):
    w = synth.free_dendrite_3d(256, scheme="SBAR120")
    s = native.Sim.from_workload(w, "f32")
    s.set_tile(*tile)
    s.step(40)
    p0, u0 = s.get_fields()
    s.step(1)
    gp, gu = s.get_fields()
    g = np.zeros(p0.shape, np.int16)
    op, ou = O.step(oracle_params(w), w.rots, g, p0.astype(np.float64), u0.astype(np.float64), 1)
    assert max_abs(_phi(gp), _phi(op)) < 2e-6
    assert max_abs(gu, ou) < 5e-6
