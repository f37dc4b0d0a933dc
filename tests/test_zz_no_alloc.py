"""The allocation-free observe entry point, pf_observe_fields_noalloc.

Some callers cannot call cudaMalloc (a host framework that owns every device
allocation, or a loop that must not stall on an allocation) but already hold
the fields on the device.  This entry point runs the observe reductions on
those fields with the library's fixed device scratch instead of caller
memory.  The test calls it through the C-ABI twice in a row, on two
different states, and checks each result against pf_observe on the same
handle: the tip cell and position exactly (both sides take the decision with
the same FP64 formula), the solute integral and solid fraction within the
1e-12 relative tolerance of the other observe tests, for one grain, for
every cell (grain -1) and for the pulling axis (grain -2).  Collected last so that
a failure here does not hide any other test.
"""
import numpy as np
import pytest

from paper_2110_12448_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    return N


def _same(a, b):
    assert a["found"] == b["found"]
    assert a["tip_index"] == b["tip_index"]
    assert a["tip"][:2] == b["tip"][:2]
    assert a["tip_score"] == b["tip_score"]
    assert a["nonfinite"] == b["nonfinite"]
    assert abs(a["solute"] - b["solute"]) <= 1e-12 * abs(b["solute"])
    assert abs(a["solid_fraction"] - b["solid_fraction"]) <= 1e-12
    assert abs(a["angle_xy_deg"] - b["angle_xy_deg"]) <= 1e-9


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_observe_matches_pf_observe_twice(native, prec):
    rng = np.random.default_rng(21)
    w = synth.polycrystal_2d(rng, 203, 4)
    s = native.Sim.from_workload(w, prec)
    for call in range(2):
        s.step(25 + 10 * call)
        psi_d, U_d, g_d = s.device_fields()
        for g in (-1, 1, -2):  # -2: every cell, +y as the growth axis (the pulling axis)
            gg = max(g, 0)
            ref = s.observe(g)
            got = native.observe_fields_noalloc(s.p, psi_d, U_d, g_d, w.rots[gg], w.centres[gg], g)
            _same(got, ref)
            assert got["status"] == native.PF_OK


def test_noalloc_observe_rejects_bad_arguments(native):
    s = native.Sim.from_workload(synth.free_dendrite_2d(32), "f32")
    psi_d, U_d, g_d = s.device_fields()
    import ctypes as C
    p = native.make_params(2, 1 << 20, 1 << 15, scheme="SBAR21")  # 2^35 cells: above the limit
    with pytest.raises(native.PfError):
        native.observe_fields_noalloc(p, psi_d, U_d, g_d, np.eye(3), np.zeros(3), -1)
    with pytest.raises(native.PfError):
        native.observe_fields_noalloc(s.p, psi_d, U_d, None, np.eye(3), np.zeros(3), 0)  # grain map needed
