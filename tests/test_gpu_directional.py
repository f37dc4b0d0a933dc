"""GPU parity of directional solidification (frozen temperature along +y,
Eqs. Thermal_F1/_F2 in Eq. PF_a; periodic x, Sec. 4.2) through the C-ABI
against the FP64 oracle: one and many steps for the three 2D schemes on ragged
and odd widths, the time origin of later steps, batched groups replayed from
CUDA graphs (the device step clock), mixed thermal / isothermal members, FP32
within the one-step tolerances, and the pulled planar front's steady state."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import max_abs, oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    return N


def ds_state(seed, nx, ny, scheme="SBAR21", n_grains=3, lT=60.0, Vp=0.3):
    rng = np.random.default_rng(seed)
    w = synth.directional_2d(nx, ny, 20.0, scheme, Vp=Vp, lT=lT)
    w.yT = ny * w.h * 0.4
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, n_grains)
    w.rots = rots
    return w, psi, U, g, rots


def gpu_sim(N, w, prec, g, rots, psi, U, step=0, stream=None):
    p = N.make_params(2, w.nx, w.ny, 1, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, w.scheme, prec,
                      max_grains=rots.shape[0], bc_x=w.bc_x, thermal=w.thermal, Vp=w.Vp, lT=w.lT, yT=w.yT)
    s = N.Sim(p, stream=stream)
    s.set_grains(rots)
    s.set_grain_index(g)
    s.set_fields(psi, U)
    s.set_step(step)
    return s


@pytest.mark.parametrize("nx", [64, 131, 190])
@pytest.mark.parametrize("scheme", ["SBAR21", "S21", "S10"])
def test_fp64_one_step_matches_oracle(native, scheme, nx):
    w, psi, U, g, rots = ds_state(1, nx, 47, scheme)
    s = gpu_sim(native, w, "f64", g, rots, psi, U, step=37)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, step=37), rots, g, psi, U, 1)
    assert rel_err(gp, op) < 1e-12 and rel_err(gu, ou) < 1e-12


@pytest.mark.parametrize("scheme", ["SBAR21", "S10"])
def test_fp64_many_steps(native, scheme):
    w, psi, U, g, rots = ds_state(2, 97, 41, scheme)
    s = gpu_sim(native, w, "f64", g, rots, psi, U, step=5)
    s.step(7)
    s.step(5)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, step=5), rots, g, psi, U, 12)
    assert rel_err(gp, op) < 12e-12 and rel_err(gu, ou) < 12e-12


def test_group_graph_clock(native):
    # two frozen-gradient members at different steps and one isothermal member,
    # 40 steps in a group (two graph replays of 16 plus single launches)
    cases = []
    for i, (nx, step) in enumerate([(70, 0), (64, 123)]):
        w, psi, U, g, rots = ds_state(10 + i, nx, 33)
        cases.append((w, psi, U, g, rots, step))
    wi = synth.free_dendrite_2d(48, 10.0)
    rng = np.random.default_rng(7)
    psi_i, U_i = synth.random_state(rng, wi)
    import torch
    st = torch.cuda.Stream()
    sims = [gpu_sim(native, w, "f64", g, rots, psi, U, step, stream=st) for w, psi, U, g, rots, step in cases]
    si = native.Sim.from_workload(wi, "f64", stream=st)
    si.set_fields(psi_i, U_i)
    grp = native.Group(3, sum(native.Group.work_items(s) for s in sims + [si]), stream=st)
    for s in sims + [si]:
        grp.add(s)
    grp.step(3, use_graph=False)
    grp.step(37, use_graph=True)
    grp.close()
    for s, (w, psi, U, g, rots, step) in zip(sims, cases):
        gp, gu = s.get_fields()
        op, ou = O.step(oracle_params(w, step=step), rots, g, psi, U, 40)
        assert rel_err(gp, op) < 40e-12 and rel_err(gu, ou) < 40e-12
        assert s.steps_done == step + 40
    gp, gu = si.get_fields()
    op, ou = O.step(oracle_params(wi), wi.rots, np.zeros(wi.shape, np.int16), psi_i, U_i, 40)
    assert rel_err(gp, op) < 40e-12 and rel_err(gu, ou) < 40e-12


@pytest.mark.parametrize("scheme", ["SBAR21", "S21", "S10"])
def test_fp32_one_step(native, scheme):
    w, psi, U, g, rots = ds_state(3, 131, 40, scheme)
    psi32, U32 = psi.astype(np.float32), U.astype(np.float32)
    s = gpu_sim(native, w, "f32", g, rots, psi32, U32, step=11)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, step=11), rots, g, psi32.astype(np.float64), U32.astype(np.float64), 1)
    assert max_abs(np.tanh(gp.astype(np.float64) / math.sqrt(2)), np.tanh(op / math.sqrt(2))) < 2e-6
    assert max_abs(gu, ou) < 5e-6


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_pulled_planar_front_tracks_the_isotherm(native, prec):
    # same setting as the oracle pin: V W / D = 0.016, the front must move at Vp
    # on the isotherm with U = 0 in the new solid
    nx, ny = 64, 220
    w = synth.directional_2d(nx, ny, 0.0, "SBAR21", Vp=0.1, lT=150.0, amp=0.0)
    w.eps4 = 0.0
    s = native.Sim.from_workload(w, prec)

    def front():
        psi, U = s.get_fields()
        col = psi[:, 5].astype(np.float64)
        j = int(np.nonzero((col[:-1] >= 0) & (col[1:] < 0))[0][0])
        return (j + col[j] / (col[j] - col[j + 1])) * w.h, j, U

    s.step(5000)
    y1, _, _ = front()
    s.step(5000)
    y2, j2, U = front()
    t = 10000 * w.dt
    assert abs((y2 - y1) / (5000 * w.dt) - w.Vp) <= 0.01 * w.Vp
    assert abs(y2 - (w.yT + w.Vp * t)) < 0.25
    assert np.max(np.abs(U[j2 - 12])) < 0.01


def test_group_on_legacy_stream_launches_directly(native):
    # graphs need a capturable stream: on the legacy default stream the group
    # falls back to direct launches and stays exact
    w, psi, U, g, rots = ds_state(21, 64, 33)
    s = gpu_sim(native, w, "f64", g, rots, psi, U, 9)
    grp = native.Group(1, native.Group.work_items(s))
    grp.add(s)
    grp.step(20, use_graph=True)
    grp.close()
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, step=9), rots, g, psi, U, 20)
    assert rel_err(gp, op) < 20e-12 and rel_err(gu, ou) < 20e-12


# ---- 3D: frozen gradient along +y, periodic x, mirror y and z ----

def ds_state3(seed, nx, ny, nz, scheme, lT=60.0, Vp=0.3):
    rng = np.random.default_rng(seed)
    w = synth.free_dendrite_3d(nx, scheme=scheme)
    w.ny, w.nz = ny, nz
    w.bc_x, w.thermal, w.Vp, w.lT, w.yT = 1, 1, Vp, lT, ny * w.h * 0.4
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, 2)
    w.rots = rots
    return w, psi, U, g, rots


def gpu_sim3(N, w, prec, g, rots, psi, U, step=0, stream=None):
    p = N.make_params(3, w.nx, w.ny, w.nz, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, w.scheme, prec,
                      max_grains=rots.shape[0], bc_x=w.bc_x, thermal=w.thermal, Vp=w.Vp, lT=w.lT, yT=w.yT)
    s = N.Sim(p, stream=stream)
    s.set_grains(rots)
    s.set_grain_index(g)
    s.set_fields(psi, U)
    s.set_step(step)
    return s


@pytest.mark.parametrize("shape", [(64, 21, 19), (37, 29, 17)])
@pytest.mark.parametrize("scheme", ["SBAR120", "S100"])
def test_fp64_3d_matches_oracle(native, scheme, shape):
    w, psi, U, g, rots = ds_state3(31, *shape, scheme)
    s = gpu_sim3(native, w, "f64", g, rots, psi, U, step=17)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, step=17), rots, g, psi, U, 1)
    assert rel_err(gp, op) < 1e-12 and rel_err(gu, ou) < 1e-12
    s.step(4)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, step=17), rots, g, psi, U, 5)
    assert rel_err(gp, op) < 5e-12 and rel_err(gu, ou) < 5e-12


@pytest.mark.parametrize("scheme", ["SBAR120", "S100"])
def test_fp32_3d_one_step(native, scheme):
    w, psi, U, g, rots = ds_state3(32, 45, 23, 18, scheme)
    psi32, U32 = psi.astype(np.float32), U.astype(np.float32)
    s = gpu_sim3(native, w, "f32", g, rots, psi32, U32, step=3)
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, step=3), rots, g, psi32.astype(np.float64), U32.astype(np.float64), 1)
    assert max_abs(np.tanh(gp.astype(np.float64) / math.sqrt(2)), np.tanh(op / math.sqrt(2))) < 2e-6
    assert max_abs(gu, ou) < 5e-6


def test_group_graph_clock_3d(native):
    import torch
    st = torch.cuda.Stream()
    w, psi, U, g, rots = ds_state3(33, 40, 22, 16, "SBAR120")
    s = gpu_sim3(native, w, "f64", g, rots, psi, U, step=50, stream=st)
    grp = native.Group(1, native.Group.work_items(s), stream=st)
    grp.add(s)
    grp.step(35, use_graph=True)
    grp.close()
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, step=50), rots, g, psi, U, 35)
    assert rel_err(gp, op) < 35e-12 and rel_err(gu, ou) < 35e-12


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_shift_frame_moves_state_and_keeps_temperature(native, prec):
    """pf_shift_frame: cell (x, y) takes (x, y + m), bit for bit; the top m
    rows are melt: psi continues the last row minus h per row (bit for bit), U
    continues the steady far field U0 + (U_last - U0) exp(-Vp k h / D) (to
    rounding), the grain index is copied; and
    the next step equals the oracle's step on the shifted state with the
    isotherm yT moved down by m h (FP64: 1e-12 relative)."""
    w, psi, U, g, rots = ds_state(21, 90, 53)
    if prec == "f32":
        psi, U = psi.astype(np.float32), U.astype(np.float32)
    s = gpu_sim(native, w, prec, g, rots, psi, U, step=41)
    s.step(3)
    p3, u3 = s.get_fields()
    g3 = s.get_grain_index()
    m = 7
    s.shift_frame(m)
    p4, u4 = s.get_fields()
    g4 = s.get_grain_index()
    assert np.array_equal(p4[:-m], p3[m:]) and np.array_equal(u4[:-m], u3[m:]) and np.array_equal(g4[:-m], g3[m:])
    steps_up = np.arange(1, m + 1)[:, None] * w.h
    want_top = (p3[-1].astype(np.float64)[None, :] - steps_up).astype(p3.dtype)
    assert np.array_equal(p4[-m:], want_top)
    ks = np.arange(1, m + 1)[:, None]
    want_u = w.U0 + (u3[-1].astype(np.float64)[None, :] - w.U0) * np.exp(-w.Vp * w.h / w.D * ks)
    assert np.abs(u4[-m:] - want_u).max() <= (1e-14 if prec == "f64" else 1e-6)
    assert np.array_equal(g4[-m:], np.repeat(g3[-1:], m, axis=0))
    assert s.steps_done == 44
    if prec == "f64":
        s.step(1)
        gp, gu = s.get_fields()
        op, ou = O.step(oracle_params(w, step=44, yT=w.yT - m * w.h), rots, g4, p4, u4, 1)
        assert rel_err(gp, op) < 1e-12 and rel_err(gu, ou) < 1e-12


def test_shift_frame_keeps_growth_angle(native):
    """The grains' reference points move with the frame: the growth angle of
    a grain and of the pulling axis is unchanged by a shift, and the tip sits
    m h lower in the moved frame (planar front with sine modes near the bottom
    of the box, so the shifted rows hold no interface)."""
    w = synth.directional_2d(96, 120, 20.0, "SBAR21", Vp=0.1, lT=500.0)
    s = native.Sim.from_workload(w, "f64")
    s.step(10)
    before = {g: s.observe(g) for g in (0, -2)}
    m = 5
    s.shift_frame(m)
    for g, b in before.items():
        a = s.observe(g)
        assert a["found"] == b["found"] == 1
        assert abs(a["tip"][1] - (b["tip"][1] - m * w.h)) <= 1e-9
        assert abs(a["tip"][0] - b["tip"][0]) <= 1e-12
        assert abs(a["angle_xy_deg"] - b["angle_xy_deg"]) <= 1e-9, (g, a["angle_xy_deg"], b["angle_xy_deg"])


@pytest.mark.parametrize("scheme", ["SBAR120", "S100"])
def test_shift_frame_3d_frozen_gradient(native, scheme):
    """3D pf_shift_frame with a frozen temperature: the top m rows of U
    continue the steady far field U0 + (U_last - U0) exp(-Vp k h / D) in every
    z plane, psi the signed distance; the next step equals the oracle's on the
    shifted state with the isotherm yT moved down by m h (FP64, 1e-12)."""
    w, psi, U, g, rots = ds_state3(34, 20, 26, 12, scheme, lT=80.0, Vp=0.2)
    s = gpu_sim3(native, w, "f64", g, rots, psi, U, step=13)
    s.step(2)
    p3, u3 = s.get_fields()  # [z, y, x]
    g3 = s.get_grain_index()
    m = 4
    s.shift_frame(m)
    p4, u4 = s.get_fields()
    g4 = s.get_grain_index()
    assert np.array_equal(p4[:, :-m], p3[:, m:]) and np.array_equal(u4[:, :-m], u3[:, m:])
    assert np.array_equal(g4[:, :-m], g3[:, m:])
    ks = np.arange(1, m + 1)[None, :, None]
    assert np.array_equal(p4[:, -m:], p3[:, -1:] - ks * w.h)
    want_u = w.U0 + (u3[:, -1:] - w.U0) * np.exp(-w.Vp * w.h / w.D * ks)
    assert np.abs(u4[:, -m:] - want_u).max() <= 1e-14
    s.step(1)
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w, step=15, yT=w.yT - m * w.h), rots, g4, p4, u4, 1)
    assert rel_err(gp, op) < 1e-12 and rel_err(gu, ou) < 1e-12


def test_shift_frame_3d_and_invalid_calls(native):
    w = synth.free_dendrite_3d(24, steps=1)
    w.nx, w.ny, w.nz = 20, 26, 12
    w.seeds = np.array([[10.0, 10.0, 5.0, 4.0]])
    s = native.Sim.from_workload(w, "f32")
    s.step(2)
    p0, u0 = s.get_fields()  # [z, y, x]
    s.shift_frame(5)
    p1, u1 = s.get_fields()
    assert np.array_equal(p1[:, :-5, :], p0[:, 5:, :]) and np.array_equal(u1[:, :-5, :], u0[:, 5:, :])
    assert np.array_equal(u1[:, -5:, :], np.repeat(u0[:, -1:, :], 5, axis=1))  # isothermal: a copy
    for bad in (0, -1, w.ny):
        with pytest.raises(native.PfError):
            s.shift_frame(bad)
    g = native.Group(2, native.Group.work_items(s))
    g.add(s)
    with pytest.raises(native.PfError):
        s.shift_frame(1)  # a group member: PF_ERR_STATE
    g.close()


def test_moving_frame_keeps_the_pulled_planar_front(native):
    """The pulled planar front of the oracle pin (V W / D = 0.016, Vp = 0.1,
    lT = 150, front on its isotherm, 4 cells wide like the pin: with lT above
    the diffusion length D/V = 63 W a wider front is constitutionally
    unstable), FP64, for the pin's 1e4 steps, once in a static box and once in
    a box shifted back by pf_shift_frame whenever the front passes 32 W: the
    two fronts agree in the lab frame within 0.05 W, stay within 0.25 W of the
    isotherm yT + Vp t, and the tip speed along the pulling axis
    (pf_observe(-2)) stays within 2% of Vp across the shifts.  A shift that
    would put F1 = 1 - (1-k) zeta below 0.05 on the grid is refused and moves
    nothing."""
    nx, ny, h, dt = 4, 220, 0.8, 0.02
    k, lam = 0.15, 10.0
    D = 0.6267 * lam
    Vp, lT, yT = 0.1, 150.0, 30.0
    y = (np.arange(ny) * h)[:, None] * np.ones((1, nx))
    eta = y - yT
    psi = -eta
    U = np.where(eta < 0, 0.0, -1.0 + np.exp(-Vp * np.maximum(eta, 0) / D))
    p = native.make_params(2, nx, ny, 1, h, dt, k, 0.0, lam, D, -1.0, "SBAR21", "f64", bc_x=native.PF_BC_PERIODIC,
                           thermal=native.PF_FROZEN_GRADIENT, Vp=Vp, lT=lT, yT=yT)
    lab = {}
    for moving in (False, True):
        s = native.Sim(p)
        s.set_fields(psi, U)
        s.observe(-2)
        off, shifts, speeds = 0.0, 0, []
        for chunk in range(10):
            s.step(1000)
            o = s.observe(-2)
            if chunk >= 1:
                speeds.append(o["v_tip"])
            lab[moving] = o["tip"][1] + off  # lab position, taken before any shift of this chunk
            if moving and o["tip"][1] > 32.0:
                rows = int(round((o["tip"][1] - 30.0) / h))
                s.shift_frame(rows)
                off += rows * h
                shifts += 1
        t = s.steps_done * dt
        assert abs(lab[moving] - (yT + Vp * t)) < 0.25
        assert max(abs(v - Vp) for v in speeds) < 0.02 * Vp, speeds
        if moving:
            assert shifts >= 3
            before = s.get_fields()
            with pytest.raises(native.PfError):
                s.shift_frame(100)  # zeta at the top would reach 1.5: F1 < 0
            after = s.get_fields()
            assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert abs(lab[True] - lab[False]) < 0.05
