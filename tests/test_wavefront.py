"""Host checks of depth-2 temporal blocking (no GPU).

Explicit Euler (Sec. 3.3.1) makes level n+1 a function of level n alone, with
a psi stencil reach of two rows (planes) and one for U and the grain.  A group
at depth 2 advances two steps as one wavefront over bands along the sweep
axis, in the order pf_wavefront_order returns, with the two levels in the
same ping-pong buffers as at depth 1.  These tests take that order from the
C-ABI library (host only) and replay it with the FP64 oracle: each launch
(level, band) is one oracle step of the whole source buffer, of which only the
band's rows are written into the destination buffer.  The intermediate buffer
starts as NaN, so a row read before it is written shows up, and a level-n row
read after its band was overwritten by level n+2 gives a wrong value.  The
result must equal two plain oracle steps bit for bit, for ragged band heights
down to the two-row minimum; a planted out-of-order schedule must not."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import native, synth
from tests.helpers import oracle_params


def order(n_bands):
    return native.wavefront_order(n_bands)


@pytest.mark.parametrize("k", [1, 2, 3, 7])
def test_order_covers_every_band_twice_in_dependency_order(k):
    seq = order(k)
    assert len(seq) == 2 * k
    assert sorted(seq) == sorted([(0, b) for b in range(k)] + [(1, b) for b in range(k)])
    pos = {e: i for i, e in enumerate(seq)}
    for b in range(k):
        # step n+2 on band b reads level n+1 on bands b-1 .. b+1 and writes
        # level n+2 over level n of band b, which steps n+1 on b-1 .. b+1 read
        for nb in (b - 1, b, b + 1):
            if 0 <= nb < k:
                assert pos[(1, b)] > pos[(0, nb)]
        # ... and it runs right after the band below it was written (L2 reuse)
        if b + 1 < k:
            assert pos[(1, b)] == pos[(0, b + 1)] + 1


def test_order_rejects_invalid_arguments():
    import ctypes as C
    L = native.lib()
    a = (C.c_int * 4)()
    assert L.pf_wavefront_order(0, a, a, 4) == native.PF_ERR_INVALID
    assert L.pf_wavefront_order(2, None, None, 4) == native.PF_ERR_INVALID
    assert L.pf_wavefront_order(2, a, a, -1) == native.PF_ERR_INVALID
    assert L.pf_wavefront_order(5, None, None, 0) == 10  # size query


def replay(p, rots, g, psi, U, rows, band_rows, seq):
    """Two steps by the (level, band) launches of seq over bands of band_rows
    rows along axis 0 of the field arrays (y in 2D, z in 3D)."""
    X = [psi.copy(), U.copy()]
    Y = [np.full_like(psi, np.nan), np.full_like(U, np.nan)]
    for lvl, b in seq:
        src, dst = (X, Y) if lvl == 0 else (Y, X)
        full = O.step(p, rots, g, src[0], src[1], 1)
        lo, hi = b * band_rows, min((b + 1) * band_rows, rows)
        for f in range(2):
            dst[f][lo:hi] = full[f][lo:hi]
    return X


def case(dim, scheme, seed):
    rng = np.random.default_rng(seed)
    if dim == 2:
        w = synth.free_dendrite_2d(21, ny=37, scheme=scheme)
    else:
        w = synth.free_dendrite_3d(11, scheme=scheme)
        w.ny, w.nz = 9, 17
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, 3)
    return w, psi, U, g, rots


@pytest.mark.parametrize("dim,scheme", [(2, "SBAR21"), (2, "S21"), (2, "S10"), (3, "SBAR120"), (3, "S100")])
@pytest.mark.parametrize("band_rows", [2, 3, 5, 8])
def test_wavefront_equals_two_steps(dim, scheme, band_rows):
    w, psi, U, g, rots = case(dim, scheme, 11 + band_rows)
    p = oracle_params(w)
    rows = psi.shape[0]
    k = -(-rows // band_rows)
    want = O.step(p, rots, g, psi, U, 2)
    got = replay(p, rots, g, psi, U, rows, band_rows, order(k))
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_wavefront_equals_two_steps_t0():
    w, psi, U, g, rots = case(2, "SBAR21", 5)
    p = oracle_params(w, time_level=O.T0)
    want = O.step(p, rots, g, psi, U, 2)
    got = replay(p, rots, g, psi, U, psi.shape[0], 4, order(-(-psi.shape[0] // 4)))
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


@pytest.mark.parametrize("bad", ["late_first_step", "one_row_band"])
def test_planted_schedule_mistakes_are_caught(bad):
    """The replay is strong enough to reject a schedule that violates the
    dependencies: step n+2 on a band before step n+1 on the band after it, and
    bands thinner than the psi halo."""
    w, psi, U, g, rots = case(2, "SBAR21", 3)
    p = oracle_params(w)
    rows = psi.shape[0]
    want = O.step(p, rots, g, psi, U, 2)
    if bad == "late_first_step":
        band_rows = 4
        k = -(-rows // band_rows)
        seq = [(0, b) for b in range(1)] + [(1, 0)] + [(0, b) for b in range(1, k)] + [(1, b) for b in range(1, k)]
    else:
        # one-row bands: step n+2 on band b reads level n+1 two rows away, in
        # band b+2, not written yet
        band_rows = 1
        seq = order(rows)
    got = replay(p, rots, g, psi, U, rows, band_rows, seq)
    assert not (np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]))
