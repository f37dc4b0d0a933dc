"""Bounds battery for the checked build (run by test_gpu_bounds.py in a
subprocess with PF_LIBRARY pointing at the -DPF_BOUNDS_CHECK library): tiny,
odd and ragged grids for every scheme, precision and variant (isothermal with
mirror walls, frozen gradient with periodic x, T0), single handles and
graph-replayed groups (with the group observe), both 3D tiles, observe and
the tip radius; the compensated FP32 state and the two-kernel form in 2D.
Prints the failure count and the first failing source line."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2110_12448_gb300 import native as N  # noqa: E402
from paper_2110_12448_gb300 import synth  # noqa: E402

VARIANTS = [dict(), dict(bc_x=1, thermal=1, Vp=0.3, lT=60.0), dict(time_level=1)]
TWO_KERNELS = dict(time_level=1, kernels=1)


def run_case(dim, scheme, prec, shape, var, tile=None, group=False, stream=None):
    rng = np.random.default_rng(sum(shape) + len(var))
    if dim == 2:
        w = synth.free_dendrite_2d(shape[0], ny=shape[1], scheme=scheme)
    else:
        w = synth.free_dendrite_3d(shape[0], scheme=scheme)
        w.ny, w.nz = shape[1], shape[2]
    for k, v in var.items():
        setattr(w, k, v)
    if var.get("thermal"):
        w.yT = w.ny * w.h * 0.4
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, 2)
    p = N.make_params(dim, w.nx, w.ny, w.nz, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, scheme, prec,
                      max_grains=2, bc_x=var.get("bc_x", 0), thermal=var.get("thermal", 0), Vp=var.get("Vp", 0.0),
                      lT=var.get("lT", 1.0), yT=w.yT, time_level=var.get("time_level", 0),
                      kernels=var.get("kernels", 0))
    s = N.Sim(p, stream=stream)
    s.set_grains(rots)
    s.set_grain_index(g)
    s.set_fields(psi, U)
    if tile:
        s.set_tile(*tile)
    if group:
        grp = N.Group(1, N.Group.work_items(s), stream=stream)
        grp.add(s)
        grp.step(18, use_graph=True)
        grp.observe(0, allow_nonfinite=True)
        grp.close()
    else:
        s.step(3)
    ob = s.observe(0, allow_nonfinite=True)
    if ob["found"]:
        try:
            s.tip_radius(ob, 0)
        except N.PfError:
            pass  # a tip on the grain centre has no growth axis
    s.close()


def main():
    torch.cuda.set_device(0)
    st = torch.cuda.Stream()
    cases = 0
    for prec in ("f32", "f64"):
        for scheme in ("SBAR21", "S21", "S10"):
            for shape in [(4, 4), (5, 9), (61, 7), (64, 5), (131, 47), (190, 33)]:
                for var in VARIANTS:
                    run_case(2, scheme, prec, shape, var, stream=st)
                    cases += 1
            run_case(2, scheme, prec, (70, 21), VARIANTS[1], group=True, stream=st)
            cases += 1
            for shape in [(4, 4), (5, 9), (61, 7), (131, 47)]:
                run_case(2, scheme, prec, shape, TWO_KERNELS, stream=st)
                cases += 1
            run_case(2, scheme, prec, (70, 21), TWO_KERNELS, group=True, stream=st)
            cases += 1
        for scheme in ("SBAR120", "S100"):
            for shape in [(4, 4, 4), (5, 9, 4), (31, 15, 7), (37, 29, 17)]:
                for var in VARIANTS:
                    for tile in ([(34, 10, 8)] if prec == "f64" else [(34, 10, 8), (34, 18, 16)]):
                        run_case(3, scheme, prec, shape, var, tile=tile, stream=st)
                        cases += 1
            run_case(3, scheme, prec, (33, 17, 9), VARIANTS[1], group=True, stream=st)
            cases += 1
    for scheme in ("SBAR21", "S21", "S10"):  # the compensated FP32 state
        for shape in [(4, 4), (5, 9), (61, 7), (64, 5), (131, 47)]:
            run_case(2, scheme, "f32c", shape, VARIANTS[0], stream=st)
            cases += 1
        run_case(2, scheme, "f32c", (70, 21), VARIANTS[0], group=True, stream=st)
        cases += 1
    torch.cuda.synchronize()
    res = N.debug_bounds()
    print(json.dumps({"cases": cases, "checked": res is not None, "failures": None if res is None else res[0],
                      "first_line": None if res is None else res[1]}))


if __name__ == "__main__":
    main()
