"""GPU parity of the compensated FP32 state (precision PF_F32C: FP32
arithmetic, psi and U stored as FP32 pairs hi + lo) against the FP64 oracle.

One step from an FP64 state.  The state is carried to about 2^-48 relative,
so what remains is the FP32 rounding of the rates: psi' - psi = dt dpsi/dt
with dpsi/dt accurate to a few FP32 ulps of its largest term (|L| up to
~1e2 at the seam of two discs of the random states, giving dt * 1e2 * 6e-8
~ 1e-7 in psi there and less in phi), and U' - U whose terms are each
accurate to a few FP32 ulps of themselves (|delta phi| <= 0.05 per step, the
diffusion term <= 0.2 |U| in one step).  Bounds: max|d phi| 2e-7 and
max|d U| 2e-7, ten times below the one-step bounds of the FP32 fields (2e-6,
5e-6), which are set by the FP32 rounding of the stored state and of phi'.

Checkpoint: FP64 fields in, FP64 fields out, to the pair's 2^-48 relative
precision.  Solute: conserved to 1e-9 relative over 100 steps (the addition
theorem's delta phi differs from the next step's phi' - phi by the FP32
rounding of tanh, ~1e-7 per interface cell and step with random sign).
Batching: a compensated member gives bit-identical results alone and in a
mixed group replayed from a CUDA graph.
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


def gpu_sim(N, w, scheme, prec, g, rots, psi, U, stream=None):
    p = N.make_params(2, w.nx, w.ny, 1, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, scheme, prec,
                      max_grains=rots.shape[0])
    s = N.Sim(p, stream=stream)
    s.set_grains(rots)
    s.set_grain_index(g)
    s.set_fields(psi, U)
    return s


def _phi(p):
    return np.tanh(np.asarray(p, np.float64) / math.sqrt(2))


def test_checkpoint_keeps_fp64_values(native):
    w, psi, U, g, rots = make_state(7, 130, 70)
    s = gpu_sim(native, w, "SBAR21", "f32c", g, rots, psi, U)
    gp, gu = s.get_fields()
    assert gp.dtype == np.float64
    assert rel_err(gp, psi) < 1e-14 and rel_err(gu, U) < 1e-14


@pytest.mark.parametrize("scheme", SCHEMES_2D)
def test_one_step_matches_oracle(native, scheme):
    w, psi, U, g, rots = make_state(3, 200, 131)
    s = gpu_sim(native, w, scheme, "f32c", g, rots, psi, U)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, scheme), rots, g, psi, U, 1)
    dphi, du = max_abs(_phi(gp), _phi(op)), max_abs(gu, ou)
    print(f"f32c one step {scheme}: max|dphi| {dphi:.3e} max|dU| {du:.3e}")
    assert dphi < 2e-7
    assert du < 2e-7


@pytest.mark.parametrize("scheme", SCHEMES_2D)
def test_ragged_tiles_and_sweeps(native, scheme):
    w, psi, U, g, rots = make_state(4, 125, 47)
    outs = []
    for sweep in (8, 17, 64):
        s = gpu_sim(native, w, scheme, "f32c", g, rots, psi, U)
        s.set_tile(64, 1, sweep)
        s.step(3)
        outs.append(s.get_fields())
        s.close()
    op, ou = O.step(oracle_params(w, scheme), rots, g, psi, U, 3)
    for gp, gu in outs:
        assert max_abs(_phi(gp), _phi(op)) < 3 * 2e-7 and max_abs(gu, ou) < 3 * 2e-7


def test_solute_conserved(native):
    w = synth.free_dendrite_2d(96)
    s = native.Sim.from_workload(w, "f32c")
    c0 = s.observe(0)["solute"]
    s.step(100)
    c1 = s.observe(0)["solute"]
    assert abs(c1 - c0) / abs(c0) < 1e-9, (c0, c1)


def test_alone_equals_in_mixed_group(native):
    import torch
    st = torch.cuda.Stream()
    w = synth.free_dendrite_2d(150, theta_deg=20.0)
    alone = native.Sim.from_workload(w, "f32c", stream=st)
    alone.step(40)
    a = alone.get_fields()
    mem = [native.Sim.from_workload(w, "f32c", stream=st),
           native.Sim.from_workload(synth.free_dendrite_2d(90), "f32", stream=st),
           native.Sim.from_workload(synth.free_dendrite_2d(70), "f64", stream=st)]
    grp = native.Group(3, sum(native.Group.work_items(m) for m in mem), stream=st)
    for m in mem:
        grp.add(m)
    grp.step(40, use_graph=True)
    grp.close()
    b = mem[0].get_fields()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_rejected_outside_its_scope(native):
    for kw in (dict(dim=3, nz=16, scheme="SBAR120", dt=0.015), dict(thermal=native.PF_FROZEN_GRADIENT, lT=100.0),
               dict(bc_x=native.PF_BC_PERIODIC), dict(time_level=native.PF_T0)):
        d = dict(dim=2, nx=32, ny=32, scheme="SBAR21", precision="f32c")
        d.update(kw)
        assert native.required_bytes(native.make_params(**d)) == 0, kw
    s = native.Sim.from_workload(synth.free_dendrite_2d(40), "f32c")
    with pytest.raises(native.PfError):
        s.shift_frame(2)
