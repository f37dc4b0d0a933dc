"""GPU checks of depth-2 temporal blocking (pf_group_set_depth): a group that
advances two steps per wavefront over bands gives, cell for cell, the same
arithmetic as one launch per step, so its fields equal the depth-1 group's
bit for bit, in FP32, FP64 and on the compensated FP32 state, 2D and 3D, for
ragged bands, odd step counts, odd starting parity, graph replay and mixed
classes; FP64 also against the oracle directly.  Groups that cannot step as wavefronts (frozen temperature,
two-kernel form) report depth 1 in effect and step as before."""
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


def states(dim, schemes, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i, sc in enumerate(schemes):
        if dim == 2:
            w = synth.free_dendrite_2d(131 + 37 * i, ny=83 + 29 * i, scheme=sc)
        else:
            w = synth.free_dendrite_3d(45 + 8 * i, scheme=sc)
            w.ny, w.nz = 23 + 4 * i, 37 + 9 * i
        psi, U = synth.random_state(rng, w)
        g, rots = synth.random_grains(rng, w, 3)
        out.append((w, psi, U, g, rots))
    return out


def run(N, cases, prec, tile, depth, band_sweeps, steps, use_graph, pre=0, extra=None):
    """Fields after `pre` depth-1 steps and then `steps` steps at the given depth."""
    import torch
    st = torch.cuda.Stream()
    sims = []
    for w, psi, U, g, rots in cases:
        p = N.make_params(w.dim, w.nx, w.ny, w.nz, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, w.scheme, prec,
                          max_grains=rots.shape[0], **(extra or {}))
        s = N.Sim(p, stream=st)
        s.set_grains(rots)
        s.set_grain_index(g)
        dt = np.float32 if prec == "f32" else np.float64
        s.set_fields(psi.astype(dt), U.astype(dt))
        s.set_tile(*tile)
        sims.append(s)
    grp = N.Group(len(sims), sum(N.Group.work_items(s) for s in sims), stream=st)
    for s in sims:
        grp.add(s)
    if pre:
        grp.step(pre, use_graph=False)
    grp.set_depth(depth, band_sweeps)
    eff = grp.depth()[2]
    grp.step(steps, use_graph=use_graph)
    grp.close()
    out = [s.get_fields() for s in sims]
    for s in sims:
        s.close()
    return out, eff


@pytest.mark.parametrize("prec", ["f32", "f64", "f32c"])
@pytest.mark.parametrize("band_sweeps", [1, 2, 5])
@pytest.mark.parametrize("steps,use_graph,pre", [(5, False, 0), (7, False, 1), (36, True, 0), (21, True, 1)])
def test_2d_depth2_equals_depth1(native, prec, band_sweeps, steps, use_graph, pre):
    cases = states(2, ["SBAR21", "SBAR21", "SBAR21"], seed=3)
    tile = (64, 1, 8)
    a, e1 = run(native, cases, prec, tile, 1, 1, steps, use_graph, pre)
    b, e2 = run(native, cases, prec, tile, 2, band_sweeps, steps, use_graph, pre)
    assert (e1, e2) == (1, 2)
    for (pa, ua), (pb, ub) in zip(a, b):
        assert np.array_equal(pa, pb) and np.array_equal(ua, ub)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_2d_mixed_classes_and_t0(native, prec):
    """S10, S21 and S-bar_21 members (three classes) at T0, bands of one
    shortest sweep and of three longer ones."""
    cases = states(2, ["S10", "S21", "SBAR21"], seed=4)
    extra = dict(time_level=native.PF_T0)
    for tile, bs in (((64, 1, 8), 1), ((64, 1, 12), 3)):
        a, _ = run(native, cases, prec, tile, 1, 1, 10, True, 0, extra)
        b, e = run(native, cases, prec, tile, 2, bs, 10, True, 0, extra)
        assert e == 2
        for (pa, ua), (pb, ub) in zip(a, b):
            assert np.array_equal(pa, pb) and np.array_equal(ua, ub)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("tile,band_sweeps", [((34, 10, 8), 1), ((34, 10, 9), 2), ((34, 18, 8), 3)])
def test_3d_depth2_equals_depth1(native, prec, tile, band_sweeps):
    if prec == "f64" and tile[1] == 18:
        pytest.skip("tile needs more shared memory than a block may have in FP64")
    cases = states(3, ["SBAR120", "S100"], seed=5)
    a, _ = run(native, cases, prec, tile, 1, 1, 6, False)
    b, e = run(native, cases, prec, tile, 2, band_sweeps, 6, False)
    assert e == 2
    for (pa, ua), (pb, ub) in zip(a, b):
        assert np.array_equal(pa, pb) and np.array_equal(ua, ub)


def test_depth2_matches_oracle_fp64(native):
    cases = states(2, ["SBAR21", "S21"], seed=6) + states(3, ["SBAR120"], seed=7)
    for c in cases:
        tile = (64, 1, 8) if c[0].dim == 2 else (34, 10, 8)
        (got,), e = run(native, [c], "f64", tile, 2, 2, 6, False)
        assert e == 2
        w, psi, U, g, rots = c
        op, ou = O.step(oracle_params(w), rots, g, psi, U, 6)
        assert rel_err(got[0], op) < 6e-12 and rel_err(got[1], ou) < 6e-12


def test_ineligible_groups_step_at_depth1(native):
    """Frozen temperature (one step clock per launch) and the two-kernel form
    keep depth 1."""
    cases = states(2, ["SBAR21"], seed=8)
    w = cases[0][0]
    thermal = dict(thermal=1, Vp=0.01, lT=1000.0, yT=0.3 * w.ny * w.h)
    a, _ = run(native, cases, "f32", (64, 1, 8), 1, 1, 5, False, extra=thermal)
    b, e = run(native, cases, "f32", (64, 1, 8), 2, 1, 5, False, extra=thermal)
    assert e == 1 and all(np.array_equal(x, y) for p, q in zip(a, b) for x, y in zip(p, q))
    _, e = run(native, cases, "f32", (64, 1, 8), 2, 1, 4, False,
               extra=dict(time_level=native.PF_T0, kernels=native.PF_TWO_KERNELS))
    assert e == 1


def test_set_depth_validates(native):
    import torch
    st = torch.cuda.Stream()
    grp = native.Group(1, 16, stream=st)
    for bad in ((0, 1), (3, 1), (2, 0)):
        with pytest.raises(native.PfError):
            grp.set_depth(*bad)
    grp.set_depth(2, 4)
    assert grp.depth() == (2, 4, 1)  # no members: nothing steps as a wavefront
    grp.close()


def _sims(N, cases, prec, tiles, st):
    sims = []
    for (w, psi, U, g, rots), tile in zip(cases, tiles):
        p = N.make_params(w.dim, w.nx, w.ny, w.nz, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, w.scheme, prec,
                          max_grains=rots.shape[0])
        s = N.Sim(p, stream=st)
        s.set_grains(rots)
        s.set_grain_index(g)
        dt = np.float32 if prec == "f32" else np.float64
        s.set_fields(psi.astype(dt), U.astype(dt))
        s.set_tile(*tile)
        sims.append(s)
    return sims


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_2d_and_3d_classes_with_different_band_counts(native, prec):
    """A 2D and a 3D member in one depth-2 group: the classes have different
    band counts (the 2D member 11 one-sweep bands, the 3D member 5), and each
    band launch skips the classes that have no items in it."""
    import torch
    cases = states(2, ["SBAR21"], seed=9) + states(3, ["SBAR120"], seed=10)
    tiles = [(64, 1, 8), (34, 10, 8)]
    out = []
    for depth in (1, 2):
        st = torch.cuda.Stream()
        sims = _sims(native, cases, prec, tiles, st)
        grp = native.Group(2, sum(native.Group.work_items(s) for s in sims), stream=st)
        for s in sims:
            grp.add(s)
        grp.set_depth(depth, 1)
        assert grp.depth()[2] == depth
        grp.step(20, use_graph=True)
        grp.step(3, use_graph=False)
        grp.close()
        out.append([s.get_fields() for s in sims])
        for s in sims:
            s.close()
    for (pa, ua), (pb, ub) in zip(*out):
        assert np.array_equal(pa, pb) and np.array_equal(ua, ub)


def test_depth_survives_membership_changes(native):
    """The depth setting holds when members leave and join; a thermal member
    joining turns the wavefronts off, and its leaving turns them back on."""
    import torch
    cases = states(2, ["SBAR21", "SBAR21"], seed=12)
    st = torch.cuda.Stream()
    a, b = _sims(native, cases, "f32", [(64, 1, 8)] * 2, st)
    grp = native.Group(3, native.Group.work_items(a) + 2 * native.Group.work_items(b), stream=st)
    grp.set_depth(2, 3)
    grp.add(a)
    grp.add(b)
    assert grp.depth() == (2, 3, 2)
    grp.step(4, use_graph=False)
    grp.remove(b)
    assert grp.depth() == (2, 3, 2)
    w = cases[0][0]
    pt = native.make_params(w.dim, w.nx, w.ny, w.nz, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, w.scheme, "f32",
                            thermal=1, Vp=0.01, lT=1000.0, yT=0.3 * w.ny * w.h)
    t = native.Sim(pt, stream=st)
    t.set_fields(cases[0][1].astype(np.float32), cases[0][2].astype(np.float32))
    t.set_tile(64, 1, 8)
    grp.add(t)
    assert grp.depth() == (2, 3, 1)
    grp.step(2, use_graph=False)
    grp.remove(t)
    assert grp.depth() == (2, 3, 2)
    grp.step(2, use_graph=False)
    grp.close()
    # a alone at depth 1 for the same 8 steps
    (ref,), _ = run(native, cases[:1], "f32", (64, 1, 8), 1, 1, 8, False)
    got = a.get_fields()
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    for s in (a, b, t):
        s.close()
