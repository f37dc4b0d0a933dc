"""Degenerate calls through the C-ABI: an empty group, zero-step group runs,
seedless and invalid seed lists, and the all-liquid state of a handle that
was never seeded.  There psi is uniform: no gradients (the anisotropy guard
gives a_s = 1), phi = -1 exactly, so Eq. PF_a reduces to d psi/dt = sqrt2 phi
= -sqrt2 while phi stays -1, delta phi = 0 and Eq. PF_b leaves U unchanged."""
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


def test_empty_group(native):
    import torch
    st = torch.cuda.Stream()
    g = native.Group(4, 1000, stream=st)
    assert len(g) == 0
    g.step(10, use_graph=True)
    g.step(10, use_graph=False)
    assert g.observe(-1) == []
    g.close()


@pytest.mark.parametrize("prec", ["f32", "f64", "f32c"])
def test_group_zero_steps_changes_nothing(native, prec):
    import torch
    st = torch.cuda.Stream()
    s = native.Sim.from_workload(synth.free_dendrite_2d(70), prec, stream=st)
    a = s.get_fields()
    g = native.Group(1, native.Group.work_items(s), stream=st)
    g.add(s)
    g.step(0)
    b = s.get_fields()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    with pytest.raises(native.PfError):
        g.step(-1)
    g.close()
    s.close()


def test_seed_lists_rejected(native):
    w = synth.free_dendrite_2d(40)
    s = native.Sim.from_workload(w, "f64")
    a = s.get_fields()
    with pytest.raises(native.PfError):
        s.init_seeds(np.zeros((0, 4)), np.zeros(0, np.int16))  # no seeds
    with pytest.raises(native.PfError):
        s.init_seeds([[1.0, 1.0, 0.0, 2.0]], [5])  # grain beyond the table
    with pytest.raises(native.PfError):
        s.init_seeds([[np.nan, 1.0, 0.0, 2.0]], [0])
    b = s.get_fields()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    s.close()


@pytest.mark.parametrize("dim,prec", [(2, "f32"), (2, "f64"), (3, "f32"), (3, "f64")])
def test_unseeded_liquid_is_a_fixed_point(native, dim, prec):
    w = synth.free_dendrite_2d(48) if dim == 2 else synth.free_dendrite_3d(20)
    p = native.make_params(dim, w.nx, w.ny, w.nz, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, w.scheme, prec)
    s = native.Sim(p)
    s.set_grains(w.rots)
    a = s.get_fields()
    assert np.all(a[0] < -100) and np.all(a[1] == np.asarray(w.U0, a[1].dtype))
    s.step(3)
    b = s.get_fields()
    assert np.array_equal(a[1], b[1])
    expect = a[0].astype(np.float64) - 3 * w.dt * np.sqrt(2.0)
    tol = 1e-12 if prec == "f64" else 3 * 6.2e-5  # three FP32 roundings at |psi| ~ 1e3
    assert np.abs(b[0] - expect).max() <= tol
    assert np.ptp(b[0]) == 0  # still uniform
    o = s.observe(-1)
    assert o["found"] == 0 and o["nonfinite"] == 0 and o["solid_fraction"] == 0.0
    s.close()
