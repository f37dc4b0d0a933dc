"""A batch split over several groups on their own streams (batch.Batch)
gives every instance exactly the state it reaches in one group on one stream:
the instances are independent and each group launch computes the same
arithmetic.  Checked bit for bit in FP32 after graph-replayed runs with
observes in between, with the observe records in workload order, also with
the groups at temporal-blocking depth 2 (two steps per band wavefront)."""
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


@pytest.mark.parametrize("n_streams", [1, 2, 3])
@pytest.mark.parametrize("tile", [(64, 1, 16), (64, 1, 16, 2, 2)])
def test_batch_equals_one_group(native, n_streams, tile):
    import torch
    from paper_2110_12448_gb300.batch import Batch
    ws = [synth.free_dendrite_2d(n, theta_deg=t) for n, t in ((96, 0.0), (130, 10.0), (70, 25.0), (111, 40.0))]
    st = torch.cuda.Stream()
    sims = [native.Sim.from_workload(w, "f32", stream=st) for w in ws]
    for s in sims:
        s.set_tile(64, 1, 16)
    g = native.Group(len(sims), sum(native.Group.work_items(s) for s in sims), stream=st)
    for s in sims:
        g.add(s)
    g.step(37, use_graph=True)
    g.step(3, use_graph=False)
    ref = [s.get_fields() for s in sims]
    ref_obs = g.observe(0)
    g.close()

    b = Batch(ws, "f32", n_streams=n_streams, tile=tile)
    assert len(b.groups) == min(n_streams, len(ws))
    assert all(g.depth()[2] == (tile[3] if len(tile) > 3 else 1) for g in b.groups)
    b.step(20, use_graph=True, stream=st)
    mid = b.observe(0)
    assert len(mid) == len(ws)
    b.step(17, use_graph=True, stream=st)
    b.step(3, use_graph=False, stream=st)
    assert b.steps_done == 40
    obs = b.observe(0)
    for s, (p0, u0), o, o0 in zip(b.members, ref, obs, ref_obs):
        p1, u1 = s.get_fields()
        assert np.array_equal(p0, p1) and np.array_equal(u0, u1)
        assert o["tip"] == o0["tip"] and o["solute"] == o0["solute"]
    b.close()
    for s in sims:
        s.close()


def test_autotune_under_two_streams(native):
    from paper_2110_12448_gb300 import autotune
    from paper_2110_12448_gb300.batch import Batch
    ws = [synth.free_dendrite_2d(160, theta_deg=t) for t in (0.0, 15.0, 30.0)]
    tile, times = autotune.tune(ws, "f32", steps=4, repeats=1, use_cache=False, n_streams=2)
    assert str(tuple(tile)) in times and all(t > 0 for t in times.values())
    b = Batch(ws, "f32", n_streams=2, tile=tile)
    b.step(5)
    assert b.steps_done == 5 and all(o["nonfinite"] == 0 for o in b.observe(0))
    b.close()


def test_empty_batch_rejected(native):
    from paper_2110_12448_gb300.batch import Batch
    with pytest.raises(ValueError):
        Batch([], "f32")


@pytest.mark.parametrize("n_streams", [2, 3])
def test_batch_equals_one_group_frozen_gradient(native, n_streams):
    """Frozen-temperature instances read their time from each group's step
    clock: split over several groups they still reach the same state."""
    import torch
    from paper_2110_12448_gb300.batch import Batch
    ws = [synth.directional_2d(96, 70, t, "SBAR21", Vp=0.3, lT=60.0) for t in (0.0, 20.0, 35.0)]
    st = torch.cuda.Stream()
    sims = [native.Sim.from_workload(w, "f32", stream=st) for w in ws]
    for s in sims:
        s.set_tile(64, 1, 16)
    g = native.Group(len(sims), sum(native.Group.work_items(s) for s in sims), stream=st)
    for s in sims:
        g.add(s)
    g.step(40, use_graph=True)
    ref = [s.get_fields() for s in sims]
    g.close()
    b = Batch(ws, "f32", n_streams=n_streams, tile=(64, 1, 16))
    b.step(24, use_graph=True, stream=st)
    b.step(16, use_graph=False, stream=st)
    for s, (p0, u0) in zip(b.members, ref):
        p1, u1 = s.get_fields()
        assert np.array_equal(p0, p1) and np.array_equal(u0, u1)
    b.close()
    for s in sims:
        s.close()
