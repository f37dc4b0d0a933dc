"""The physical claim of Sec. 4.3.2 on the GPU path: isotropic schemes keep
the growth direction of a 2D free dendrite on the crystal axis, the
anisotropic S_{1,0} does not when W and h are large.

The growth angle alpha is measured as in the paper, by tracking the tip: the
direction of the tip's displacement over the second half of the run.
* The isothermal setup of Sec. 4.3.2 (781^2, h/W = 1.2, W/d0* = 16,
  eps4 = 0.014, 20 345 steps), alpha0 = 30 deg: S_{1,0}'s lattice anisotropy
  turns the tip more than 6 deg toward the grid diagonal (measured +11 deg),
  while S-bar_{2,1} stays within 2.5 deg (measured +0.6) and S_{2,1} within
  4 deg (measured +2.3).
* 3D (Sec. 6.2.2): see test_3d_paper_setup_growth_angle.
* A resolved dendrite (h/W = 0.8, the workloads' physics, 768^2, 12 000 steps)
  with S-bar_{2,1} at alpha0 = 15 and 40 deg: alpha within 1 deg of alpha0
  (measured 0.06 and 0.42) and sigma* = 2 D d0* / (rho^2 V) the same at both
  angles within 15% (measured 9%).
"""
import math

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


def tracked(N, w):
    """(alpha by tip tracking over the second half, sigma*) after w.steps."""
    s = N.Sim.from_workload(w, "f32")
    half = w.steps // 2
    s.step(half)
    t1 = s.observe(0)["tip"]
    s.step(w.steps - half - 1000)
    s.observe(0)
    s.step(1000)
    o = s.observe(0)
    assert o["found"] and o["nonfinite"] == 0
    t2 = o["tip"]
    alpha = math.degrees(math.atan2(-(t2[0] - t1[0]), t2[1] - t1[1]))
    sigma = s.tip_radius(o, 0)["sigma_star"]
    s.close()
    return alpha, sigma


@pytest.mark.parametrize("scheme,lo,hi", [("S10", 6.0, 20.0), ("SBAR21", -2.5, 2.5), ("S21", -4.0, 4.0)])
def test_paper_setup_growth_angle(native, scheme, lo, hi):
    w = synth.paper_isothermal_2d(30.0, scheme)
    alpha, _ = tracked(native, w)
    assert lo < alpha - 30.0 < hi, (scheme, alpha)


def test_resolved_isotropic_dendrite_is_rotation_invariant(native):
    res = {}
    for theta in (15.0, 40.0):
        w = synth.free_dendrite_2d(768, theta, "SBAR21", steps=12000)
        res[theta] = tracked(native, w)
        assert abs(res[theta][0] - theta) < 1.0, (theta, res[theta])
    s15, s40 = res[15.0][1], res[40.0][1]
    assert abs(s15 - s40) / max(s15, s40) < 0.15, res


def test_3d_paper_setup_growth_angle(native):
    """Sec. 6.2.2 in a reduced cube (192^3, 15 000 of the ~30 500 steps; the
    paper's 9.6e4 d0* cube does not fit one GPU), crystal turned by
    alpha0 = 15 deg about z: S_{1,0,0} turns the tip more than 12 deg toward
    the grid diagonal (measured +22), S-bar_{1,2,0} stays within 8 deg
    (measured -6; +0.5 at the paper's full time in a 320^3 cube)."""
    dev = {}
    for scheme in ("S100", "SBAR120"):
        w = synth.paper_isothermal_3d(15.0, scheme, n=192, steps=15000)
        dev[scheme] = tracked(native, w)[0] - 15.0
    assert dev["S100"] > 12.0, dev
    assert abs(dev["SBAR120"]) < 8.0, dev
