"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a temporary copy of oracle/pf_oracle.c
(never in the committed file), builds it, and runs the pin suites
(test_oracle_symbols.py, test_oracle_step.py, test_oracle_tip_radius.py,
test_oracle_directional.py, test_oracle_time_level.py) against that build through the ORACLE_LIB override: at least one pin must
fail."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pf_oracle.c")

# (name, text to find, replacement): each a mistake someone could make
# The 2D and 3D rates spell the frozen-temperature terms alike; each thermal
# mutation is applied inside one rate's block (its own comment and the three
# lines below it), so that it hits exactly one of them.
_THERMAL_BODY = (
    "        double zeta = (j * h - q->yT - q->Vp * t) / q->lT;\n"
    "        double F1 = 1.0 - (1.0 - q->k) * zeta, F2 = u + zeta;\n"
    "        return ((L + N + SQ2 * (ph - q->lambda * (1.0 - ph * ph) * F2)) / (ac * ac) - SQ2 * ph * G) / F1;\n")
THERMAL_BLOCKS = {
    "2d": "        /* Eq. PF_a with the frozen-temperature functions F1, F2 */\n" + _THERMAL_BODY,
    "3d": "        /* Eq. PF_a with the frozen-temperature functions F1, F2 (pulling along +y) */\n" + _THERMAL_BODY,
}
MUTATIONS = [
    ("lap21_weights_swapped", "return (2.0 / 3.0) * lap_10(f, i, j, h) + (1.0 / 3.0) * lap_01(f, i, j, h);",
     "return (1.0 / 3.0) * lap_10(f, i, j, h) + (2.0 / 3.0) * lap_01(f, i, j, h);"),
    ("lap01_prefactor", "- 4.0 * V2(f, i, j)) /\n           (2.0 * h * h);", "- 4.0 * V2(f, i, j)) /\n           (1.0 * h * h);"),
    ("grad01_prefactor", "return (a * a + b * b) / (8.0 * h * h);", "return (a * a + b * b) / (4.0 * h * h);"),
    ("flux10_drops_corner_mean",
     "w = V2(a, i + dx, j) + V2(a, i, j) + abar2(a, i, j, dx, 1) + abar2(a, i, j, dx, -1);",
     "w = V2(a, i + dx, j) + V2(a, i, j) + 2.0 * abar2(a, i, j, dx, 1);"),
    ("flux11_wrong_neighbour", "return w / (4.0 * SQ2 * h) * (V2(b, i + dx, j + dy) - V2(b, i, j));",
     "return w / (4.0 * SQ2 * h) * (V2(b, i + dx, j) - V2(b, i, j));"),
    ("div21_weights", "return (2.0 / 3.0) * div_10(a, b, i, j, h) + (1.0 / 3.0) * div_01(a, b, i, j, h);",
     "return 0.5 * div_10(a, b, i, j, h) + 0.5 * div_01(a, b, i, j, h);"),
    ("flux100_nn_weight", "double ab = 0.25 * near + (1.0 / 16.0) * nn;", "double ab = 0.25 * near + (1.0 / 32.0) * nn;"),
    ("flux110_weights", "double ab = (3.0 / 16.0) * near + (1.0 / 32.0) * nn;",
     "double ab = (1.0 / 4.0) * near + (0.0) * nn;"),
    ("lap010_prefactor", "return (s - 12.0 * F3(f, 0, 0, 0)) / (4.0 * h * h);", "return (s - 12.0 * F3(f, 0, 0, 0)) / (2.0 * h * h);"),
    ("aniso_rotation_transposed", "for (int q = 0; q < dim; ++q) gc[p] += R[q * 3 + p] * g[q];",
     "for (int q = 0; q < dim; ++q) gc[p] += R[p * 3 + q] * g[q];"),
    ("aniso_cubic_coefficient", "double a = 1.0 - 3.0 * eps4 + 4.0 * eps4 * s4 / (r2 * r2);",
     "double a = 1.0 - 2.0 * eps4 + 4.0 * eps4 * s4 / (r2 * r2);"),
    ("aniso_derivative_sign", "double da = 16.0 * eps4 * (gc[p] * gc[p] * gc[p] / (r2 * r2) - gc[p] * s4 / (r2 * r2 * r2));",
     "double da = 16.0 * eps4 * (gc[p] * gc[p] * gc[p] / (r2 * r2) + gc[p] * s4 / (r2 * r2 * r2));"),
    ("mirror_off_by_one", "if (i < 0) i = -1 - i;", "if (i < 0) i = -i;"),
    ("update_uses_old_phi", "(1.0 + k - (1.0 - k) * phn);", "(1.0 + k - (1.0 - k) * (phn - *PA(&Pdphi, i, j, kk)));"),
    ("antitrapping_sign", "tmp[c] = u + (dt * (q->D * Dterm + Aterm)", "tmp[c] = u + (dt * (q->D * Dterm - Aterm)"),
    ("antitrapping_alpha_dt", "Palpha.v[c] = (1.0 + (1.0 - k) * PU.v[c]) * Pdphi.v[c] / (SQ2 * dt);",
     "Palpha.v[c] = (1.0 + (1.0 - k) * PU.v[c]) * Pdphi.v[c] / (2.0 * dt);"),
    ("source_lambda_sign", "return (L + N + SQ2 * (ph - q->lambda * (1.0 - ph * ph) * u)) / (ac * ac) - SQ2 * ph * G;\n}\n\nstatic double dpsi_dt_3d",
     "return (L + N + SQ2 * (ph + q->lambda * (1.0 - ph * ph) * u)) / (ac * ac) - SQ2 * ph * G;\n}\n\nstatic double dpsi_dt_3d"),
    ("G_term_dropped_3d", "return (L + N + SQ2 * (ph - q->lambda * (1.0 - ph * ph) * u)) / (ac * ac) - SQ2 * ph * G;\n}\n\nstatic int check_params",
     "return (L + N + SQ2 * (ph - q->lambda * (1.0 - ph * ph) * u)) / (ac * ac);\n}\n\nstatic int check_params"),
    ("appb_coefficient", "double dn = (35.0 / 24.0) * ((B(1, 1) - B(0, -1)) - (B(0, 1) - B(1, -1))) / (2.0 * h) -\n                (1.0 / 8.0)",
     "double dn = (35.0 / 48.0) * ((B(1, 1) - B(0, -1)) - (B(0, 1) - B(1, -1))) / (2.0 * h) -\n                (1.0 / 8.0)"),
    ("tip_interpolation", "double frac = ps / (ps - pn);", "double frac = pn / (pn - ps);"),
    ("solute_weight", "sol += (1.0 + k - (1.0 - k) * ph) * (1.0 + (1.0 - k) * u) / 2.0;",
     "sol += (1.0 + k + (1.0 - k) * ph) * (1.0 + (1.0 - k) * u) / 2.0;"),
    ("init_radius_sign", "double v = seeds[4 * s + 3] - sqrt(dx * dx + dy * dy + dz * dz);",
     "double v = seeds[4 * s + 3] + sqrt(dx * dx + dy * dy + dz * dz);"),
    ("tip_radius_fit_factor", "rho = 0.5 * (s4 / st);", "rho = (s4 / st);"),
    ("tip_radius_interp_swapped", "f[1] * ((1.0 - f[0]) * TRV(0, 1, 0) + f[0] * TRV(1, 1, 0));\n    if",
     "f[1] * ((1.0 - f[0]) * TRV(1, 1, 0) + f[0] * TRV(0, 1, 0));\n    if"),
    ("tip_radius_crossing", "dt * (prev / (prev - v))", "dt * (v / (prev - v))"),
    ("tip_radius_no_window", "        w = rho;\n", "        w = w;\n"),
    ("tip_radius_combination_3d", "2.0 / (1.0 / rx + 1.0 / rz)", "0.5 * (rx + rz)"),
    ("tip_radius_transverse_axis", "ex[0] = ez[1] * epar[2] - ez[2] * epar[1];", "ex[0] = ez[1] * epar[2] + ez[2] * epar[1];"),
    *[(f"thermal_{name}_{dim}", blk, blk.replace(old, new)) for dim, blk in THERMAL_BLOCKS.items() for name, old, new in [
        ("F1_dropped",
         "return ((L + N + SQ2 * (ph - q->lambda * (1.0 - ph * ph) * F2)) / (ac * ac) - SQ2 * ph * G) / F1;",
         "return ((L + N + SQ2 * (ph - q->lambda * (1.0 - ph * ph) * F2)) / (ac * ac) - SQ2 * ph * G);"),
        ("F2_sign", "double F1 = 1.0 - (1.0 - q->k) * zeta, F2 = u + zeta;",
         "double F1 = 1.0 - (1.0 - q->k) * zeta, F2 = u - zeta;"),
        ("F1_sign", "double F1 = 1.0 - (1.0 - q->k) * zeta, F2 = u + zeta;",
         "double F1 = 1.0 + (1.0 - q->k) * zeta, F2 = u + zeta;"),
        ("pulling_sign", "double zeta = (j * h - q->yT - q->Vp * t) / q->lT;",
         "double zeta = (j * h - q->yT + q->Vp * t) / q->lT;"),
        ("row_offset", "double zeta = (j * h - q->yT - q->Vp * t) / q->lT;",
         "double zeta = ((j + 1) * h - q->yT - q->Vp * t) / q->lT;"),
    ]],
    ("thermal_clock_frozen", "dpsi_dt_2d(q, &Ppsi, &Pphi, &PU, &Pg, rot, i, j, q->t0 + (double)s * dt)",
     "dpsi_dt_2d(q, &Ppsi, &Pphi, &PU, &Pg, rot, i, j, q->t0)"),
    ("t0_chain_rule_factor", "Pdphi.v[c] = dt * (1.0 - ph * ph) / SQ2 * Pnew.v[c];",
     "Pdphi.v[c] = dt * (1.0 - ph * ph) * Pnew.v[c];"),
    ("t0_without_1_minus_phi2", "Pdphi.v[c] = dt * (1.0 - ph * ph) / SQ2 * Pnew.v[c];",
     "Pdphi.v[c] = dt / SQ2 * Pnew.v[c];"),
    ("t0_uses_new_phi", "                Pnew.v[c] = ph; /* phi^n on the left-hand side */",
     "                Pnew.v[c] = tanh((Ppsi.v[c] + dt * Pnew.v[c]) / SQ2);"),
    ("at21_floor_dropped_face",
     "        if (g_at21_floor) m = fmax(m, 0.5 * fabs(V2(b, i + dx, j + dy) - V2(b, i, j)) / h);\n", ""),
    ("at21_floor_dropped_corner",
     "        if (g_at21_floor) m = fmax(m, 0.5 * fabs(V2(b, i + dx, j + dy) - V2(b, i, j)) / (SQ2 * h));\n", ""),
    ("at21_floor_factor", "if (g_at21_floor) m = fmax(m, 0.5 * fabs(V2(b, i + dx, j + dy) - V2(b, i, j)) / h);",
     "if (g_at21_floor) m = fmax(m, 2.0 * fabs(V2(b, i + dx, j + dy) - V2(b, i, j)) / h);"),
    ("observe_pulling_axis_as_x", "    if (g == -2) d[1] = 1.0;", "    if (g == -2) d[0] = 1.0;"),
    ("at_std2_no_normalisation", "((V2(b, i + dx, j + dy) - V2(b, i, j)) / h) / sqrt(m2);",
     "((V2(b, i + dx, j + dy) - V2(b, i, j)) / h);"),
    ("at_std3_one_sided_alpha", "s += 0.5 * (F3(a, e[0], e[1], e[2]) + F3(a, 0, 0, 0)) * ((F3(b,",
     "s += F3(a, 0, 0, 0) * ((F3(b,"),
    ("lap120_weights", "(1.0 / 3.0) * lap_100(f, i, j, k, h) + (2.0 / 3.0) * lap_010(f, i, j, k, h)",
     "(2.0 / 3.0) * lap_100(f, i, j, k, h) + (1.0 / 3.0) * lap_010(f, i, j, k, h)"),
    ("psi_update_half_dt", "psin[c] = psi[c] + dt * r;", "psin[c] = psi[c] + 0.5 * dt * r;"),
    ("U_denominator_sign", "(1.0 + (1.0 - k) * u) * dph) / (1.0 + k - (1.0 - k) * phn);",
     "(1.0 + (1.0 - k) * u) * dph) / (1.0 + k + (1.0 - k) * phn);"),
    ("G_term_dropped_2d",
     "    return (L + N + SQ2 * (ph - q->lambda * (1.0 - ph * ph) * u)) / (ac * ac) - SQ2 * ph * G;\n}\n\n"
     "static double dpsi_dt_3d(",
     "    return (L + N + SQ2 * (ph - q->lambda * (1.0 - ph * ph) * u)) / (ac * ac);\n}\n\nstatic double dpsi_dt_3d("),
    ("growth_axis_lowest_y", "            if (yc > best) {", "            if (-yc > best) {"),
    ("periodic_x_as_mirror", "if (bc == OR_BC_PERIODIC_X) return axis == 0 ? OR_BC_PERIODIC : OR_BC_MIRROR;",
     "if (bc == OR_BC_PERIODIC_X) return OR_BC_MIRROR;"),
]


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(source, name, old, new):
    assert source.count(old) == 1, f"mutation {name}: anchor text not found exactly once"
    mutated = source.replace(old, new)
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "pf_oracle_mut.c")
        lib = os.path.join(d, "liboracle_mut.so")
        open(src, "w").write(mutated)
        subprocess.run(["gcc", "-std=c11", "-O1", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", lib, src,
                        "-lm"], check=True)
        env = dict(os.environ, ORACLE_LIB=lib, OMP_NUM_THREADS="2")
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_symbols.py"),
                            os.path.join(ROOT, "tests", "test_oracle_step.py"),
                            os.path.join(ROOT, "tests", "test_oracle_tip_radius.py"),
                            os.path.join(ROOT, "tests", "test_oracle_directional.py"),
                            os.path.join(ROOT, "tests", "test_oracle_time_level.py"),
                            os.path.join(ROOT, "tests", "test_oracle_at21_guard.py")],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"mutation {name} survived every pin:\n{r.stdout[-2000:]}"
