"""GPU parity of the T0 time level (pure forward Euler of Eq. PF_b with the
chain-rule d phi/dt; Sec. 2.1, 3.3.1) through the C-ABI against the FP64
oracle, for the five schemes (2D: the variant instantiation of the fused
kernel; 3D: a run-time switch), FP64 per step and over several steps, FP32
within the one-step tolerances, and T0 and T1 members stepped in one group."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import max_abs, oracle_params, rel_err

pytestmark = pytest.mark.gpu

CASES = [("SBAR21", 2), ("S21", 2), ("S10", 2), ("SBAR120", 3), ("S100", 3)]


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    return N


def state(dim, scheme, seed=6):
    rng = np.random.default_rng(seed)
    if dim == 2:
        w = synth.free_dendrite_2d(131, ny=47, scheme=scheme)
    else:
        w = synth.free_dendrite_3d(45, scheme=scheme)
        w.ny, w.nz = 23, 21
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, 3)
    return w, psi, U, g, rots


def gpu_sim(N, w, prec, g, rots, psi, U, time_level, stream=None):
    p = N.make_params(w.dim, w.nx, w.ny, w.nz, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, w.scheme, prec,
                      max_grains=rots.shape[0], time_level=time_level)
    s = N.Sim(p, stream=stream)
    s.set_grains(rots)
    s.set_grain_index(g)
    s.set_fields(psi, U)
    return s


@pytest.mark.parametrize("scheme,dim", CASES)
def test_fp64_t0_matches_oracle(native, scheme, dim):
    w, psi, U, g, rots = state(dim, scheme)
    s = gpu_sim(native, w, "f64", g, rots, psi, U, native.PF_T0)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, time_level=O.T0), rots, g, psi, U, 1)
    assert rel_err(gp, op) < 1e-12 and rel_err(gu, ou) < 1e-12
    s.step(5)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, time_level=O.T0), rots, g, psi, U, 6)
    assert rel_err(gp, op) < 6e-12 and rel_err(gu, ou) < 6e-12


@pytest.mark.parametrize("scheme,dim", CASES)
def test_fp32_t0_one_step(native, scheme, dim):
    w, psi, U, g, rots = state(dim, scheme, seed=7)
    psi32, U32 = psi.astype(np.float32), U.astype(np.float32)
    s = gpu_sim(native, w, "f32", g, rots, psi32, U32, native.PF_T0)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, time_level=O.T0), rots, g, psi32.astype(np.float64), U32.astype(np.float64), 1)
    assert max_abs(np.tanh(gp.astype(np.float64) / math.sqrt(2)), np.tanh(op / math.sqrt(2))) < 2e-6
    assert max_abs(gu, ou) < 5e-6


def test_group_mixes_time_levels(native):
    import torch
    st = torch.cuda.Stream()
    runs = []
    for i, tl in enumerate((native.PF_T0, native.PF_T1, native.PF_T0)):
        w, psi, U, g, rots = state(2, "SBAR21", seed=20 + i)
        runs.append((w, psi, U, g, rots, tl, gpu_sim(native, w, "f64", g, rots, psi, U, tl, stream=st)))
    grp = native.Group(3, sum(native.Group.work_items(r[-1]) for r in runs), stream=st)
    for r in runs:
        grp.add(r[-1])
    grp.step(34, use_graph=True)
    grp.close()
    for w, psi, U, g, rots, tl, s in runs:
        gp, gu = s.get_fields()
        op, ou = O.step(oracle_params(w, time_level=tl), rots, g, psi, U, 34)
        assert rel_err(gp, op) < 34e-12 and rel_err(gu, ou) < 34e-12
