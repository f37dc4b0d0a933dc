"""GPU parity of the two-kernel form of the step (Sec. 3.3.1: a psi kernel,
then a U kernel; pf_params.kernels = PF_TWO_KERNELS) through the C-ABI.

The psi kernel stores psi' and d psi/dt in device memory; the U kernel reads
d psi/dt back and applies the T0 update of Eq. PF_b.  Checks:
  * FP64 against the oracle's T0 step: 1e-12 relative per step, three 2D
    schemes, ragged grids with several grains, and over several steps;
  * the same values as the fused T0 step: the rate is the same arithmetic,
    stored and reloaded at the field precision, so the two forms agree bit for
    bit in FP32 (explicitly rounded packed operations), alone and in a group
    replayed from CUDA graphs, and to round-off in FP64 (where the compiler
    may contract a product and a sum into an FMA in one kernel and not in the
    other: 1e-15 relative per step);
  * frozen temperature with periodic x (the same kernel variant) against the
    oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import oracle_params, rel_err

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


def state(seed, nx, ny, scheme):
    rng = np.random.default_rng(seed)
    w = synth.free_dendrite_2d(nx, ny=ny, scheme=scheme, eps4=0.05)
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, 3)
    return w, psi, U, g, rots


def gpu_sim(N, w, prec, g, rots, psi, U, kernels, stream=None, **kw):
    p = N.make_params(2, w.nx, w.ny, 1, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, w.scheme, prec,
                      max_grains=rots.shape[0], time_level=N.PF_T0, kernels=kernels, **kw)
    s = N.Sim(p, stream=stream)
    s.set_grains(rots)
    s.set_grain_index(g)
    s.set_fields(psi, U)
    return s


@pytest.mark.parametrize("nx,ny", [(131, 47), (64, 64), (5, 9)])
@pytest.mark.parametrize("scheme", SCHEMES_2D)
def test_fp64_matches_oracle(native, scheme, nx, ny):
    w, psi, U, g, rots = state(61, nx, ny, scheme)
    s = gpu_sim(native, w, "f64", g, rots, psi, U, native.PF_TWO_KERNELS)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, time_level=O.T0), rots, g, psi, U, 1)
    assert rel_err(gp, op) < 1e-12 and rel_err(gu, ou) < 1e-12
    s.step(7)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, time_level=O.T0), rots, g, psi, U, 8)
    assert rel_err(gp, op) < 8e-12 and rel_err(gu, ou) < 8e-12


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("scheme", SCHEMES_2D)
def test_equals_fused_t0_bit_for_bit(native, scheme, prec):
    w, psi, U, g, rots = state(62, 190, 83, scheme)
    if prec == "f32":
        psi, U = psi.astype(np.float32), U.astype(np.float32)
    out = {}
    for kernels in (native.PF_FUSED, native.PF_TWO_KERNELS):
        s = gpu_sim(native, w, prec, g, rots, psi, U, kernels)
        s.set_tile(64, 1, 19)
        s.step(6)
        out[kernels] = s.get_fields()
        s.close()
    for a, b in zip(out[native.PF_FUSED], out[native.PF_TWO_KERNELS]):
        if prec == "f32":
            assert np.array_equal(a, b)  # explicitly rounded FP32 operations: bit for bit
        else:  # the compiler may contract a FP64 product and sum differently in the two kernels
            assert rel_err(a, b) < 6e-15


def test_group_graph_equals_alone(native):
    import torch
    st = torch.cuda.Stream()
    w, psi, U, g, rots = state(63, 150, 70, "SBAR21")
    alone = gpu_sim(native, w, "f32", g, rots, psi.astype(np.float32), U.astype(np.float32), native.PF_FUSED,
                    stream=st)
    alone.step(35)
    a = alone.get_fields()
    two = gpu_sim(native, w, "f32", g, rots, psi.astype(np.float32), U.astype(np.float32), native.PF_TWO_KERNELS,
                  stream=st)
    other = native.Sim.from_workload(synth.free_dendrite_2d(90), "f32", stream=st)
    grp = native.Group(2, native.Group.work_items(two) + native.Group.work_items(other), stream=st)
    grp.add(two)
    grp.add(other)
    grp.step(35, use_graph=True)
    grp.close()
    b = two.get_fields()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_frozen_gradient_periodic_matches_oracle(native):
    rng = np.random.default_rng(64)
    w = synth.directional_2d(96, 61, 20.0, "SBAR21", Vp=0.3, lT=60.0)
    w.yT = 61 * w.h * 0.4
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, 2)
    s = gpu_sim(native, w, "f64", g, rots, psi, U, native.PF_TWO_KERNELS, bc_x=native.PF_BC_PERIODIC,
                thermal=native.PF_FROZEN_GRADIENT, Vp=w.Vp, lT=w.lT, yT=w.yT)
    s.set_step(11)
    s.step(3)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, step=11, time_level=O.T0), rots, g, psi, U, 3)
    assert rel_err(gp, op) < 3e-12 and rel_err(gu, ou) < 3e-12
