"""The 2D step's path for instances whose cells are all in grain 0 (the
instance record's one_grain flag): no grain rows are read and no
grain-boundary faces are recomputed, with the same arithmetic as the general
path.  Checked bit for bit against the general path, which a second grain
with the same crystal frame in one corner selects; and against the FP64
oracle when a grouped member's grain map changes between steps, so the group
must refresh the member's record."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    return N


def sim(N, w, prec, rots, g, psi, U, stream=None, tile=(64, 1, 16)):
    p = N.make_params(w.dim, w.nx, w.ny, w.nz, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, w.scheme, prec,
                      max_grains=4)
    s = N.Sim(p, stream=stream)
    s.set_grains(rots)
    s.set_grain_index(g)
    dt = np.float32 if prec == "f32" else np.float64
    s.set_fields(psi.astype(dt), U.astype(dt))
    s.set_tile(*tile)
    return s


@pytest.mark.parametrize("prec", ["f32", "f64", "f32c"])
@pytest.mark.parametrize("scheme", ["SBAR21", "S21", "S10"])
def test_one_grain_path_equals_general_path(native, prec, scheme):
    rng = np.random.default_rng(31)
    w = synth.free_dendrite_2d(133, ny=71, scheme=scheme)
    psi, U = synth.random_state(rng, w)
    _, rots = synth.random_grains(rng, w, 2)
    rots[1] = rots[0]  # grain 1: the same crystal frame
    g0 = np.zeros(psi.shape, np.int16)
    g1 = g0.copy()
    g1[1, 1] = 1  # selects the general path; its faces are recomputed in the same frame
    a = sim(native, w, prec, rots, g0, psi, U)
    b = sim(native, w, prec, rots, g1, psi, U)
    a.step(1)
    b.step(1)
    (pa, ua), (pb, ub) = a.get_fields(), b.get_fields()
    # the stencils of cells beyond the corner's neighbourhood never see grain 1
    far = np.ones(psi.shape, bool)
    far[:6, :6] = False
    assert np.array_equal(pa[far], pb[far]) and np.array_equal(ua[far], ub[far])
    a.close()
    b.close()


@pytest.mark.parametrize("scheme", ["SBAR21", "S21"])
def test_group_refreshes_a_member_whose_grains_change(native, scheme):
    import torch
    rng = np.random.default_rng(32)
    w = synth.free_dendrite_2d(131, ny=77, scheme=scheme)
    psi, U = synth.random_state(rng, w)
    g_multi, rots = synth.random_grains(rng, w, 3)
    g_one = np.zeros(psi.shape, np.int16)
    st = torch.cuda.Stream()
    s = sim(native, w, "f64", rots, g_one, psi, U, stream=st)
    other = sim(native, w, "f64", rots, g_multi, psi, U, stream=st)
    grp = native.Group(2, 2 * native.Group.work_items(s), stream=st)
    grp.add(s)
    grp.add(other)
    grp.step(3, use_graph=False)
    torch.cuda.synchronize()
    s.set_grain_index(g_multi)  # in the group: the group rebuilds the member's record
    grp.step(4, use_graph=False)
    grp.close()
    p = oracle_params(w)
    op, ou = O.step(p, rots, g_one, psi, U, 3)
    op, ou = O.step(p, rots, g_multi, op, ou, 4)
    gp, gu = s.get_fields()
    assert rel_err(gp, op) < 7e-12 and rel_err(gu, ou) < 7e-12
    s.close()
    other.close()
