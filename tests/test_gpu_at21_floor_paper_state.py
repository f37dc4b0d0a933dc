"""What the magnitude floor of A_{2,1} (reading R-A21G) does on a state the
paper's own setup reaches.

App. B divides each D~_{2,1} anti-trapping flux by |grad psi| from the
21-point derivatives at the flux point, so each flux carries the quotient
(psi_e - psi_0) / (|e| |grad psi|).  Nothing in App. B bounds it.  The oracle
raises the magnitude to half of the two-point slope where it falls below,
which bounds every quotient by 2 and the whole term, with alpha = 1, by
(16/3 + 8/(3 sqrt2)) / h.

The state: the isothermal S_{2,1} run of Sec. 4.3.2 at alpha0 = 0 (781^2,
h/W = 1.2, eps4 = 0.014, Omega = 0.43, k = 0.1), grown on the GPU in FP32 to
the paper's 20 345 steps.  On it the oracle's A_{2,1} without the floor
exceeds that bound more than fivefold inside the interface, while the floor
changes fewer than 0.1 % of the cells, all of them inside the diffuse
interface (|phi| < 1) and none in the bulk.  With the floor the term stays
within the bound.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import oracle_params

pytestmark = pytest.mark.gpu

BOUND = 16 / 3 + 8 / (3 * math.sqrt(2))


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    return N


def test_floor_on_the_sec_4_3_2_state(native):
    w = synth.paper_isothermal_2d(0.0, "S21")
    s = native.Sim.from_workload(w, "f32")
    s.step(w.steps)
    psi, _ = s.get_fields()
    s.close()
    psi = psi.astype(np.float64)
    assert np.isfinite(psi).all()
    p = oracle_params(w)
    one = np.ones_like(psi)
    prev = O.set_at21_floor(True)
    try:
        a_on = O.apply(p, "at_21", one, psi)
        O.set_at21_floor(False)
        a_off = O.apply(p, "at_21", one, psi)
    finally:
        O.set_at21_floor(prev)
    # with the floor: within the bound of quotients <= 2
    assert np.abs(a_on).max() * w.h <= BOUND * (1 + 1e-12)
    # without it: App. B's quotients run far past any bounded value
    off_max = np.abs(a_off).max() * w.h
    assert off_max > 5 * BOUND, off_max
    # the floor acts on few cells, all inside the diffuse interface
    acts = a_on != a_off
    assert 0 < acts.sum() < 1e-3 * acts.size, int(acts.sum())
    phi = np.tanh(psi[acts] / math.sqrt(2))
    assert np.abs(phi).max() < 1.0 - 1e-6
    big = np.abs(a_off) * w.h > BOUND
    assert np.abs(psi[big]).max() < 8.0
