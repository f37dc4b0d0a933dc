"""GPU parity of S_{2,1}'s standard anti-trapping term with the magnitude floor
of reading R-A21G (App. B), on states where the floor acts, and the run that
needs it.

* Rough states: a random interface state with noise of 0.4 W added inside the
  band |psi| < 3, so that the 21-point |grad psi| falls below half of the
  two-point slope at many flux points.  FP64 against the oracle: 1e-12
  relative per step; FP32 from an FP32-representable state with the
  tolerances of the smooth one-step test (phi 2e-6, U 5e-6) scaled by 4 for
  the larger rates of a rough field.
* The isothermal runs of Sec. 4.3.2 (781^2, h/W = 1.2, W/d0* = 16,
  eps4 = 0.014, 20 345 steps): without the floor the FP32 S_{2,1} run at
  alpha0 = 0 diverges near step 18 500 from a local maximum of psi inside the
  interface; with it every cell stays finite and the crystal keeps growing.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import max_abs, oracle_params, rel_err
from tests.test_gpu_step2d import gpu_sim, make_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    return N


def rough_state(seed, nx, ny):
    w, psi, U, g, rots = make_state(seed, nx, ny)
    rng = np.random.default_rng(seed + 1000)
    psi = psi + (np.abs(psi) < 3) * rng.normal(scale=0.4, size=psi.shape)
    return w, psi, U, g, rots


def floored_x_faces(psi, h):
    """Interior x faces where the 21-point |grad psi| is below half of the
    two-point slope (where the floor acts)."""
    ny, nx = psi.shape
    n = 0
    for j in range(2, ny - 2):
        for i in range(2, nx - 3):
            if abs(psi[j, i]) >= 3:
                continue
            g = O.appb_grad(psi, i, j, 0, h)
            if math.hypot(g[0], g[1]) < 0.5 * abs(psi[j, i + 1] - psi[j, i]) / h:
                n += 1
    return n


def test_rough_state_exercises_the_floor():
    w, psi, _, _, _ = rough_state(5, 70, 40)
    assert floored_x_faces(psi, w.h) >= 10


@pytest.mark.parametrize("steps", [1, 8])
def test_fp64_rough_state_matches_oracle(native, steps):
    w, psi, U, g, rots = rough_state(5, 197, 96)
    s = gpu_sim(native, w, "S21", "f64", g, rots, psi, U)
    s.step(steps)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, "S21"), rots, g, psi, U, steps)
    assert rel_err(gp, op) < steps * 1e-12
    assert rel_err(gu, ou) < steps * 1e-12


def test_fp32_rough_state_matches_oracle(native):
    w, psi, U, g, rots = rough_state(6, 200, 131)
    psi32, U32 = psi.astype(np.float32), U.astype(np.float32)
    s = gpu_sim(native, w, "S21", "f32", g, rots, psi32, U32)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, "S21"), rots, g, psi32.astype(np.float64), U32.astype(np.float64), 1)
    phi_g = np.tanh(gp.astype(np.float64) / math.sqrt(2))
    phi_o = np.tanh(op / math.sqrt(2))
    assert max_abs(phi_g, phi_o) < 8e-6
    assert max_abs(gu, ou) < 2e-5


def test_paper_isothermal_s21_run_stays_finite(native):
    w = synth.paper_isothermal_2d(0.0, "S21")
    s = native.Sim.from_workload(w, "f32")
    done = 0
    while done < w.steps:
        k = min(5000, w.steps - done)
        s.step(k)
        done += k
        o = s.observe(0, allow_nonfinite=True)
        assert o["nonfinite"] == 0, f"non-finite cells by step {done}"
    assert o["found"] and o["solid_fraction"] > 0.02
