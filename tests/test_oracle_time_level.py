"""Pins of the oracle's T0 time level (pure forward Euler of Eq. PF_b as
printed: d phi/dt by the chain rule (1 - phi^2)/sqrt2 dpsi/dt, phi^n on the
left-hand side; Sec. 2.1 and 3.3.1) against what forward Euler fixes,
independently of how the right-hand side is evaluated:
- one T0 step is exactly linear in dt: U(2 dt) - U = 2 (U(dt) - U);
- T0 and T1 (delta phi, phi') differ by O(dt^2) per step, so the T0 rate is
  the dt -> 0 limit of the T1 increment;
- T0 does not conserve the solute exactly: its drift over a fixed time is
  first order in dt, while T1 conserves it to round-off."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import oracle_params

CASES = [("SBAR21", 2), ("S21", 2), ("S10", 2), ("SBAR120", 3), ("S100", 3)]


def state(dim, scheme, seed=4):
    rng = np.random.default_rng(seed)
    if dim == 2:
        w = synth.free_dendrite_2d(28, ny=22, scheme=scheme)
    else:
        w = synth.free_dendrite_3d(14, scheme=scheme)
        w.ny, w.nz = 13, 12
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, 2)
    return w, psi, U, g, rots


@pytest.mark.parametrize("scheme,dim", CASES)
def test_t0_step_is_linear_in_dt(scheme, dim):
    w, psi, U, g, rots = state(dim, scheme)
    dt = w.dt * 0.25
    p1 = oracle_params(w, time_level=O.T0, dt=dt)
    p2 = oracle_params(w, time_level=O.T0, dt=2 * dt)
    a_psi, a_U = O.step(p1, rots, g, psi, U, 1)
    b_psi, b_U = O.step(p2, rots, g, psi, U, 1)
    for x0, a, b in ((psi, a_psi, b_psi), (U, a_U, b_U)):
        da, db = a - x0, b - x0
        assert np.max(np.abs(db - 2 * da)) <= 1e-12 * np.max(np.abs(db))


@pytest.mark.parametrize("scheme,dim", CASES)
def test_t0_and_t1_agree_to_second_order(scheme, dim):
    w, psi, U, g, rots = state(dim, scheme)
    diffs, incs = [], []
    for dt in (w.dt * 0.25, w.dt * 0.125):
        _, u0 = O.step(oracle_params(w, time_level=O.T0, dt=dt), rots, g, psi, U, 1)
        _, u1 = O.step(oracle_params(w, time_level=O.T1, dt=dt), rots, g, psi, U, 1)
        diffs.append(np.max(np.abs(u0 - u1)))
        incs.append(np.max(np.abs(u1 - U)))
    ratio = diffs[0] / diffs[1]
    assert 3.4 < ratio < 4.6, ratio              # O(dt^2) difference
    assert diffs[0] < 0.1 * incs[0]              # much smaller than the O(dt) increment


def test_t0_solute_drift_is_first_order():
    w, psi, U, g, rots = state(2, "SBAR21")
    p = oracle_params(w)

    def solute(ps, u):
        return O.observe(p, rots, np.zeros((1, 3)) + 1.0, g, ps, u)["solute"]

    c0 = solute(psi, U)
    drift = {}
    for tl in (O.T0, O.T1):
        for dt, n in ((w.dt * 0.5, 20), (w.dt * 0.25, 40)):
            ps, u = O.step(oracle_params(w, time_level=tl, dt=dt), rots, g, psi, U, n)
            drift[(tl, n)] = abs(solute(ps, u) - c0) / abs(c0)
    assert drift[(O.T1, 20)] < 1e-13 and drift[(O.T1, 40)] < 1e-13
    assert drift[(O.T0, 20)] > 1e-7
    r = drift[(O.T0, 20)] / drift[(O.T0, 40)]
    assert 1.6 < r < 2.4, r
