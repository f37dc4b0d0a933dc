"""pf_group_observe: the observe reductions of every member of a group with one
synchronisation give exactly what pf_observe gives on the same members run
alone (FP32, FP64 and compensated members; tip cell and position, solute,
solid fraction, and the tip velocity from the previous group observation)."""
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


def test_group_observe_equals_observe_alone(native):
    import torch
    st = torch.cuda.Stream()
    ws = [(synth.free_dendrite_2d(120, theta_deg=10.0), "f32"), (synth.free_dendrite_2d(90, theta_deg=25.0), "f64"),
          (synth.free_dendrite_2d(100, theta_deg=40.0), "f32c")]
    alone = [native.Sim.from_workload(w, p, stream=st) for w, p in ws]
    ref = []
    for s in alone:
        s.step(30)
        s.observe(0)
        s.step(20)
        ref.append(s.observe(0))
    mem = [native.Sim.from_workload(w, p, stream=st) for w, p in ws]
    grp = native.Group(3, sum(native.Group.work_items(m) for m in mem), stream=st)
    for m in mem:
        grp.add(m)
    grp.step(30, use_graph=False)
    grp.observe(0)
    grp.step(20, use_graph=False)
    got = grp.observe(0)
    grp.close()
    for a, b in zip(got, ref):
        assert a["found"] == b["found"] == 1
        assert a["tip_index"] == b["tip_index"] and a["tip"] == b["tip"]
        assert a["solute"] == b["solute"] and a["solid_fraction"] == b["solid_fraction"]
        assert a["v_tip"] == b["v_tip"] and a["v_tip"] > 0
        assert a["step"] == b["step"] == 50


def test_group_observe_rejects_a_grain_some_member_lacks(native):
    rng = np.random.default_rng(5)
    a = native.Sim.from_workload(synth.polycrystal_2d(rng, 96, 3), "f32")
    b = native.Sim.from_workload(synth.free_dendrite_2d(64), "f32")
    grp = native.Group(2, native.Group.work_items(a) + native.Group.work_items(b))
    grp.add(a)
    grp.add(b)
    with pytest.raises(native.PfError):
        grp.observe(2)  # b has one grain
    assert len(grp.observe(-1)) == 2
    grp.close()
