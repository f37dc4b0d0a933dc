/*
 * pf_oracle.c -- plain FP64 CPU oracle of the explicit time step of the
 * quantitative binary-alloy phase-field model with the isotropic finite
 * differences of Ji, Molavi Tabrizi & Karma (arXiv:2110.12448).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or helper with
 * the CUDA library; the two implement the same equations independently.
 *
 * Structure: whole-grid passes in the order the paper states them.
 *   pass 0  copy psi, U, grain into padded arrays with ghost cells
 *           (cell-centred mirror = no-flux walls, or periodic for tests)
 *   pass 1  phi = tanh(psi / sqrt 2)                                 (Eq. 1)
 *   pass 2  d psi/dt from Eq. PF_a for every cell, psi' = psi + dt dpsi/dt
 *   pass 3  phi' and delta phi everywhere (ghosts mirrored from psi')
 *   pass 4  U' from Eq. PF_b in conservative form for every cell
 *
 * Operators (all lengths in units of W, lattice spacing h):
 *   L_{1,0}, L_{0,1}, L_{2,1}               Eqs. 2D_L10, 2D_L01, 2D_L21
 *   D~_{1,0}, D~_{0,1}, D~_{2,1}            Eqs. divergence_10/_11, flux_10/_11
 *   G_{1,0}, G_{0,1}, G_{2,1}               App. A, Eqs. Grad_10, Grad_11
 *   A_{2,1} (standard anti-trapping)        App. B
 *   L, D~, G on <100>, <110>, <111> shells  Sec. 5, Eqs. 3D_L100-3D_L111,
 *                                           divergence_100-_111, Grad_100-_111
 *   S_{1,0}, S_{1,0,0} divergences          <10>/<100> fluxes with a two-point
 *                                           face mean of alpha (the paper cites
 *                                           Tourret 2015/2017 without a formula)
 *   anisotropy                              Eq. anis_function, cubic form in 3D
 *
 * Readings of points where the paper is silent are listed in the design
 * notes of the repository (R-ANISO, R-BC, T1, R-GUARD, R-INIT, R-GRAIN,
 * R-ROT, R-TIP, R-S10, R-A21, G-144).
 *
 * Parity pins: every operator is pinned by its printed Fourier symbol, exact
 * polynomial reproduction or reduction identities; the step by the planar
 * fixed point, exact solute conservation, Fourier-mode decay and lattice
 * symmetry; observe by closed-form fields.  The S_{1,0}/S_{1,0,0} divergence
 * and anti-trapping forms are pinned only by reduction, conservation and
 * convergence checks: "parity unpinned" against the paper, which does not
 * print them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OR_S10 0
#define OR_S21 1
#define OR_SBAR21 2
#define OR_S100 3
#define OR_SBAR120 4

#define OR_BC_MIRROR 0
#define OR_BC_PERIODIC 1
#define OR_BC_PERIODIC_X 2 /* periodic in x, cell-centred mirror in y (and z) */

/* thermal = 0: isothermal (F1 = 1, F2 = U, Sec. 2.1).  thermal = 1: frozen
 * temperature for directional solidification along +y (Eqs. Thermal_F1,
 * Thermal_F2): zeta = (y - yT - Vp t) / lT, F1 = 1 - (1-k) zeta, F2 = U +
 * zeta, with y = j h and t = t0 + s dt at step s of a call. */
typedef struct {
    int dim, nx, ny, nz;
    int scheme, bc;
    double h, dt, k, eps4, lambda, D;
    int thermal, time_level;
    double Vp, lT, yT, t0;
} or_params;

/* time_level 0 = T1 (default): U' uses phi' and delta phi = phi' - phi;
 * time_level 1 = T0: pure forward Euler of Eq. PF_b as printed, d phi/dt =
 * (1 - phi^2) / sqrt2 d psi/dt (chain rule) in the source and the
 * anti-trapping term, phi^n on the left-hand side. */
#define OR_T1 0
#define OR_T0 1

static const double SQ2 = 1.41421356237309504880;
static const double SQ3 = 1.73205080756887729353;

/* ------------------------------------------------------------------------- */
/* padded fields: 2 ghost layers on each side of each axis (z only in 3D)    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz, dim;
    int sx, sy;      /* padded strides */
    int oz;          /* z offset (2 in 3D, 0 in 2D) */
    double* v;
} pad_t;

/* boundary rule of axis `axis` under the parameter bc */
static int axis_bc(int bc, int axis) {
    if (bc == OR_BC_PERIODIC_X) return axis == 0 ? OR_BC_PERIODIC : OR_BC_MIRROR;
    return bc;
}

static int map_index(int i, int n, int bc) {
    if (bc == OR_BC_PERIODIC) return ((i % n) + n) % n;
    /* cell-centred mirror: -1 -> 0, -2 -> 1, n -> n-1, n+1 -> n-2 */
    while (i < 0 || i >= n) {
        if (i < 0) i = -1 - i;
        if (i >= n) i = 2 * n - 1 - i;
    }
    return i;
}

static int pad_alloc(pad_t* p, const or_params* q) {
    p->nx = q->nx; p->ny = q->ny; p->nz = q->dim == 3 ? q->nz : 1; p->dim = q->dim;
    p->sx = q->nx + 4; p->sy = q->ny + 4; p->oz = q->dim == 3 ? 2 : 0;
    size_t n = (size_t)p->sx * p->sy * (p->nz + 2 * p->oz);
    p->v = (double*)calloc(n, sizeof(double));
    return p->v ? 0 : -1;
}

static inline double* PA(const pad_t* p, int i, int j, int k) {
    return p->v + ((size_t)(k + p->oz) * p->sy + (size_t)(j + 2)) * p->sx + (size_t)(i + 2);
}
#define V2(p, i, j) (*PA((p), (i), (j), 0))
#define V3(p, i, j, k) (*PA((p), (i), (j), (k)))

/* fill interior from src and ghosts by the boundary rule */
static void pad_fill(pad_t* p, const double* src, int bc) {
    int zl = p->dim == 3 ? -2 : 0, zh = p->dim == 3 ? p->nz + 2 : 1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = zl; k < zh; ++k)
        for (int j = -2; j < p->ny + 2; ++j)
            for (int i = -2; i < p->nx + 2; ++i) {
                int ii = map_index(i, p->nx, axis_bc(bc, 0)), jj = map_index(j, p->ny, axis_bc(bc, 1));
                int kk = p->dim == 3 ? map_index(k, p->nz, axis_bc(bc, 2)) : 0;
                *PA(p, i, j, k) = src[((size_t)kk * p->ny + jj) * p->nx + ii];
            }
}

/* ------------------------------------------------------------------------- */
/* 2D operators at cell (i,j); Sec. 3 and Appendices A, B                     */
/* ------------------------------------------------------------------------- */

/* Eq. 2D_L10: <10> shell */
static double lap_10(const pad_t* f, int i, int j, double h) {
    return (V2(f, i + 1, j) + V2(f, i - 1, j) + V2(f, i, j + 1) + V2(f, i, j - 1) - 4.0 * V2(f, i, j)) / (h * h);
}
/* Eq. 2D_L01: <11> shell, spacing sqrt(2) h */
static double lap_01(const pad_t* f, int i, int j, double h) {
    return (V2(f, i + 1, j + 1) + V2(f, i - 1, j + 1) + V2(f, i + 1, j - 1) + V2(f, i - 1, j - 1) - 4.0 * V2(f, i, j)) /
           (2.0 * h * h);
}
/* Eq. 2D_L21: weights 2/3 on <10>, 1/3 on <11> (Eq. tau_2D) */
static double lap_21(const pad_t* f, int i, int j, double h) {
    return (2.0 / 3.0) * lap_10(f, i, j, h) + (1.0 / 3.0) * lap_01(f, i, j, h);
}

/* App. A, Eq. Grad_10 */
static double grad2_10(const pad_t* f, int i, int j, double h) {
    double a = V2(f, i + 1, j) - V2(f, i - 1, j), b = V2(f, i, j + 1) - V2(f, i, j - 1);
    return (a * a + b * b) / (4.0 * h * h);
}
/* App. A, Eq. Grad_11 */
static double grad2_01(const pad_t* f, int i, int j, double h) {
    double a = V2(f, i + 1, j + 1) - V2(f, i - 1, j - 1), b = V2(f, i + 1, j - 1) - V2(f, i - 1, j + 1);
    return (a * a + b * b) / (8.0 * h * h);
}
static double grad2_21(const pad_t* f, int i, int j, double h) {
    return (2.0 / 3.0) * grad2_10(f, i, j, h) + (1.0 / 3.0) * grad2_01(f, i, j, h);
}

/* alpha-bar at the off-lattice corner (i + sx/2, j + sy/2): mean of the four
 * surrounding lattice values (text after Eq. flux_10) */
static double abar2(const pad_t* a, int i, int j, int sx, int sy) {
    return 0.25 * (V2(a, i, j) + V2(a, i + sx, j) + V2(a, i, j + sy) + V2(a, i + sx, j + sy));
}

/* Eq. flux_10: <10> flux from (i,j) towards (i+dx, j+dy), outward positive */
static double flux_10(const pad_t* a, const pad_t* b, int i, int j, int dx, int dy, double h) {
    double w;
    if (dx != 0)
        w = V2(a, i + dx, j) + V2(a, i, j) + abar2(a, i, j, dx, 1) + abar2(a, i, j, dx, -1);
    else
        w = V2(a, i, j + dy) + V2(a, i, j) + abar2(a, i, j, 1, dy) + abar2(a, i, j, -1, dy);
    return w / (4.0 * h) * (V2(b, i + dx, j + dy) - V2(b, i, j));
}
/* Eq. divergence_10 */
static double div_10(const pad_t* a, const pad_t* b, int i, int j, double h) {
    return (flux_10(a, b, i, j, 1, 0, h) + flux_10(a, b, i, j, -1, 0, h) + flux_10(a, b, i, j, 0, 1, h) +
            flux_10(a, b, i, j, 0, -1, h)) /
           h;
}
/* Eq. flux_11: <11> flux towards (i+dx, j+dy) */
static double flux_11(const pad_t* a, const pad_t* b, int i, int j, int dx, int dy, double h) {
    double w = V2(a, i + dx, j + dy) + V2(a, i, j) + V2(a, i, j + dy) + V2(a, i + dx, j);
    return w / (4.0 * SQ2 * h) * (V2(b, i + dx, j + dy) - V2(b, i, j));
}
/* Eq. divergence_11 */
static double div_01(const pad_t* a, const pad_t* b, int i, int j, double h) {
    return (flux_11(a, b, i, j, 1, 1, h) + flux_11(a, b, i, j, -1, 1, h) + flux_11(a, b, i, j, 1, -1, h) +
            flux_11(a, b, i, j, -1, -1, h)) /
           (SQ2 * h);
}
static double div_21(const pad_t* a, const pad_t* b, int i, int j, double h) {
    return (2.0 / 3.0) * div_10(a, b, i, j, h) + (1.0 / 3.0) * div_01(a, b, i, j, h);
}

/* S_{1,0} divergence (reading R-S10): <10> fluxes with a two-point face mean */
static double div_std_2d(const pad_t* a, const pad_t* b, int i, int j, double h) {
    static const int d[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    double s = 0.0;
    for (int q = 0; q < 4; ++q) {
        int dx = d[q][0], dy = d[q][1];
        s += 0.5 * (V2(a, i + dx, j + dy) + V2(a, i, j)) * (V2(b, i + dx, j + dy) - V2(b, i, j)) / h;
    }
    return s / h;
}

/* face gradient of b at the <10> face between (i,j) and (i+dx, j+dy):
 * normal component = two-point difference, transverse = four-point mean of
 * the centred differences on both sides (the <10> shell used for the O(eps4)
 * terms, reading R-ANISO) */
static void face_grad_2d(const pad_t* b, int i, int j, int dx, int dy, double h, double g[2]) {
    if (dx != 0) {
        int i1 = i + dx;
        g[0] = (V2(b, i1, j) - V2(b, i, j)) / h * (double)dx; /* d/dx, sign-corrected */
        g[1] = (V2(b, i1, j + 1) + V2(b, i, j + 1) - V2(b, i1, j - 1) - V2(b, i, j - 1)) / (4.0 * h);
    } else {
        int j1 = j + dy;
        g[0] = (V2(b, i + 1, j1) + V2(b, i + 1, j) - V2(b, i - 1, j1) - V2(b, i - 1, j)) / (4.0 * h);
        g[1] = (V2(b, i, j1) - V2(b, i, j)) / h * (double)dy;
    }
}

/* S_{1,0} anti-trapping divergence (reading R-S10): <10> fluxes of
 * alpha grad(b)/|grad b| with a two-point alpha and the face gradient */
static double at_std_2d(const pad_t* a, const pad_t* b, int i, int j, double h, double guard2) {
    static const int d[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    double s = 0.0;
    for (int q = 0; q < 4; ++q) {
        int dx = d[q][0], dy = d[q][1];
        double g[2];
        face_grad_2d(b, i, j, dx, dy, h, g);
        double m2 = g[0] * g[0] + g[1] * g[1];
        if (m2 * h * h < guard2) continue;
        s += 0.5 * (V2(a, i + dx, j + dy) + V2(a, i, j)) * ((V2(b, i + dx, j + dy) - V2(b, i, j)) / h) / sqrt(m2);
    }
    return s / h;
}

/* App. B: |grad b| at the <10> face point (i + 1/2, j) and, by the 90-degree
 * rotation the appendix prescribes, at (i, j + 1/2).  B(p, q) reads b at
 * origin + p along the face normal and q along the face tangent. */
static double bt(const pad_t* b, int i, int j, int tr, int p, int q) {
    return tr ? V2(b, i + q, j + p) : V2(b, i + p, j + q);
}
static double gradmag_face_2d(const pad_t* b, int i, int j, int tr, double h) {
#define B(p, q) bt(b, i, j, tr, (p), (q))
    double dn = (35.0 / 24.0) * ((B(1, 1) - B(0, -1)) - (B(0, 1) - B(1, -1))) / (2.0 * h) -
                (1.0 / 8.0) * ((B(2, 1) - B(-1, -1)) - (B(-1, 1) - B(2, -1))) / (6.0 * h) -
                (1.0 / 3.0) * ((B(1, 2) - B(0, -2)) - (B(0, 2) - B(1, -2))) / (2.0 * h);
    double dt = (35.0 / 24.0) * ((B(1, 1) - B(0, -1)) + (B(0, 1) - B(1, -1))) / (4.0 * h) -
                (1.0 / 8.0) * ((B(2, 1) - B(-1, -1)) + (B(-1, 1) - B(2, -1))) / (4.0 * h) -
                (1.0 / 3.0) * ((B(1, 2) - B(0, -2)) + (B(0, 2) - B(1, -2))) / (8.0 * h);
#undef B
    return sqrt(dn * dn + dt * dt);
}
/* App. B: |grad b| at the corner (i + 1/2, j + 1/2) */
static double gradmag_corner_2d(const pad_t* b, int i, int j, double h) {
#define B(p, q) V2(b, i + (p), j + (q))
    double dx = (5.0 / 4.0) * ((B(1, 1) - B(0, 0)) - (B(0, 1) - B(1, 0))) / (2.0 * h) -
                (1.0 / 8.0) * ((B(2, 1) - B(-1, 0)) - (B(-1, 1) - B(2, 0))) / (6.0 * h) -
                (1.0 / 8.0) * ((B(1, 2) - B(0, -1)) - (B(0, 2) - B(1, -1))) / (2.0 * h);
    double dy = (5.0 / 4.0) * ((B(1, 1) - B(0, 0)) + (B(0, 1) - B(1, 0))) / (2.0 * h) -
                (1.0 / 8.0) * ((B(2, 1) - B(-1, 0)) + (B(-1, 1) - B(2, 0))) / (2.0 * h) -
                (1.0 / 8.0) * ((B(1, 2) - B(0, -1)) + (B(0, 2) - B(1, -1))) / (6.0 * h);
#undef B
    return sqrt(dx * dx + dy * dy);
}
/* exported for the App. B exactness pin: derivative pair at a face or corner */
int or_appb_grad(const double* field, int nx, int ny, int i, int j, int kind, double h, double out[2]) {
    or_params q = {2, nx, ny, 1, 0, OR_BC_PERIODIC, h, 0, 0, 0, 0, 0};
    pad_t b;
    if (pad_alloc(&b, &q)) return -1;
    pad_fill(&b, field, OR_BC_PERIODIC);
    double d0, d1;
    if (kind == 0 || kind == 1) {
        int tr = kind;
#define B(p, q) bt(&b, i, j, tr, (p), (q))
        d0 = (35.0 / 24.0) * ((B(1, 1) - B(0, -1)) - (B(0, 1) - B(1, -1))) / (2.0 * h) -
             (1.0 / 8.0) * ((B(2, 1) - B(-1, -1)) - (B(-1, 1) - B(2, -1))) / (6.0 * h) -
             (1.0 / 3.0) * ((B(1, 2) - B(0, -2)) - (B(0, 2) - B(1, -2))) / (2.0 * h);
        d1 = (35.0 / 24.0) * ((B(1, 1) - B(0, -1)) + (B(0, 1) - B(1, -1))) / (4.0 * h) -
             (1.0 / 8.0) * ((B(2, 1) - B(-1, -1)) + (B(-1, 1) - B(2, -1))) / (4.0 * h) -
             (1.0 / 3.0) * ((B(1, 2) - B(0, -2)) + (B(0, 2) - B(1, -2))) / (8.0 * h);
#undef B
        /* (normal, tangent) -> (x, y) */
        out[0] = tr ? d1 : d0;
        out[1] = tr ? d0 : d1;
    } else {
#define B(p, q) V2(&b, i + (p), j + (q))
        d0 = (5.0 / 4.0) * ((B(1, 1) - B(0, 0)) - (B(0, 1) - B(1, 0))) / (2.0 * h) -
             (1.0 / 8.0) * ((B(2, 1) - B(-1, 0)) - (B(-1, 1) - B(2, 0))) / (6.0 * h) -
             (1.0 / 8.0) * ((B(1, 2) - B(0, -1)) - (B(0, 2) - B(1, -1))) / (2.0 * h);
        d1 = (5.0 / 4.0) * ((B(1, 1) - B(0, 0)) + (B(0, 1) - B(1, 0))) / (2.0 * h) -
             (1.0 / 8.0) * ((B(2, 1) - B(-1, 0)) + (B(-1, 1) - B(2, 0))) / (2.0 * h) -
             (1.0 / 8.0) * ((B(1, 2) - B(0, -1)) + (B(0, 2) - B(1, -1))) / (6.0 * h);
#undef B
        out[0] = d0;
        out[1] = d1;
    }
    free(b.v);
    return 0;
}

/* App. B: standard anti-trapping A_{2,1}: the D~_{2,1} fluxes of
 * alpha grad(b) with |grad b| from the 21-point derivatives at each flux
 * point (reading R-A21).  Each flux carries the quotient
 * (b_e - b_0) / (|e| |grad b|), the component of the unit normal along the
 * flux direction e; where the 21-point magnitude is less than half of the
 * two-point slope |b_e - b_0| / |e| (a quotient above 2, which occurs only
 * where grad b has no direction, e.g. at a local extremum of psi inside the
 * interface) the magnitude is raised to that half (reading R-A21G). */
/* The floor of reading R-A21G is on unless a test turns it off (to show
 * what App. B's form does without it); or_set_at21_floor returns the
 * previous setting. */
static int g_at21_floor = 1;
int or_set_at21_floor(int on) {
    int old = g_at21_floor;
    g_at21_floor = on != 0;
    return old;
}
static double at_21(const pad_t* a, const pad_t* b, int i, int j, double h, double guard2) {
    double s10 = 0.0, s11 = 0.0;
    /* <10> fluxes: (dx,dy) and the face whose App. B origin gives that point */
    static const int d10[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    for (int q = 0; q < 4; ++q) {
        int dx = d10[q][0], dy = d10[q][1];
        double m;
        if (dx != 0)
            m = gradmag_face_2d(b, dx > 0 ? i : i - 1, j, 0, h);
        else
            m = gradmag_face_2d(b, i, dy > 0 ? j : j - 1, 1, h);
        if (g_at21_floor) m = fmax(m, 0.5 * fabs(V2(b, i + dx, j + dy) - V2(b, i, j)) / h);
        if (m * m * h * h < guard2) continue;
        s10 += flux_10(a, b, i, j, dx, dy, h) / m;
    }
    static const int d11[4][2] = {{1, 1}, {-1, 1}, {1, -1}, {-1, -1}};
    for (int q = 0; q < 4; ++q) {
        int dx = d11[q][0], dy = d11[q][1];
        double m = gradmag_corner_2d(b, dx > 0 ? i : i - 1, dy > 0 ? j : j - 1, h);
        if (g_at21_floor) m = fmax(m, 0.5 * fabs(V2(b, i + dx, j + dy) - V2(b, i, j)) / (SQ2 * h));
        if (m * m * h * h < guard2) continue;
        s11 += flux_11(a, b, i, j, dx, dy, h) / m;
    }
    return (2.0 / 3.0) * s10 / h + (1.0 / 3.0) * s11 / (SQ2 * h);
}

/* ------------------------------------------------------------------------- */
/* 3D operators at cell (i,j,k); Sec. 5 and App. A                            */
/* ------------------------------------------------------------------------- */
#define F3(f, di, dj, dk) V3((f), i + (di), j + (dj), k + (dk))

static double lap_100(const pad_t* f, int i, int j, int k, double h) { /* Eq. 3D_L100 */
    double s = F3(f, 1, 0, 0) + F3(f, -1, 0, 0) + F3(f, 0, 1, 0) + F3(f, 0, -1, 0) + F3(f, 0, 0, 1) + F3(f, 0, 0, -1);
    return (s - 6.0 * F3(f, 0, 0, 0)) / (h * h);
}
static double lap_010(const pad_t* f, int i, int j, int k, double h) { /* Eq. 3D_L110 */
    double s = 0.0;
    for (int a = -1; a <= 1; a += 2)
        for (int b = -1; b <= 1; b += 2) s += F3(f, a, b, 0) + F3(f, a, 0, b) + F3(f, 0, a, b);
    return (s - 12.0 * F3(f, 0, 0, 0)) / (4.0 * h * h);
}
static double lap_001(const pad_t* f, int i, int j, int k, double h) { /* Eq. 3D_L111 */
    double s = 0.0;
    for (int a = -1; a <= 1; a += 2)
        for (int b = -1; b <= 1; b += 2)
            for (int c = -1; c <= 1; c += 2) s += F3(f, a, b, c);
    return (s - 8.0 * F3(f, 0, 0, 0)) / (4.0 * h * h);
}
static double lap_120(const pad_t* f, int i, int j, int k, double h) { /* Eq. tau_3D with (1,2,0) */
    return (1.0 / 3.0) * lap_100(f, i, j, k, h) + (2.0 / 3.0) * lap_010(f, i, j, k, h);
}

static double grad2_100(const pad_t* f, int i, int j, int k, double h) { /* Eq. Grad_100 */
    double a = F3(f, 1, 0, 0) - F3(f, -1, 0, 0), b = F3(f, 0, 1, 0) - F3(f, 0, -1, 0), c = F3(f, 0, 0, 1) - F3(f, 0, 0, -1);
    return (a * a + b * b + c * c) / (4.0 * h * h);
}
static double grad2_010(const pad_t* f, int i, int j, int k, double h) { /* Eq. Grad_110 */
    double t[6] = {F3(f, 1, 1, 0) - F3(f, -1, -1, 0), F3(f, 1, -1, 0) - F3(f, -1, 1, 0),
                   F3(f, 1, 0, 1) - F3(f, -1, 0, -1), F3(f, -1, 0, 1) - F3(f, 1, 0, -1),
                   F3(f, 0, 1, 1) - F3(f, 0, -1, -1), F3(f, 0, -1, 1) - F3(f, 0, 1, -1)};
    double s = 0.0;
    for (int q = 0; q < 6; ++q) s += t[q] * t[q];
    return s / (16.0 * h * h);
}
/* Eq. Grad_111 with the prefactor 1/(16 h^2) (reading G-144: the printed
 * 1/(144 h^2) does not reproduce |grad psi|^2 for a linear psi) */
static double grad2_001(const pad_t* f, int i, int j, int k, double h) {
    double t[4] = {F3(f, 1, 1, 1) - F3(f, -1, -1, -1), F3(f, 1, 1, -1) - F3(f, -1, -1, 1),
                   F3(f, 1, -1, 1) - F3(f, -1, 1, -1), F3(f, -1, 1, 1) - F3(f, 1, -1, -1)};
    double s = 0.0;
    for (int q = 0; q < 4; ++q) s += t[q] * t[q];
    return s / (16.0 * h * h);
}
static double grad2_120(const pad_t* f, int i, int j, int k, double h) {
    return (1.0 / 3.0) * grad2_100(f, i, j, k, h) + (2.0 / 3.0) * grad2_010(f, i, j, k, h);
}

/* <100> flux towards unit offset e (one nonzero component of +-1):
 * alpha-bar = 1/4 (two nearest) + 1/16 (eight next-nearest) */
static double flux_100(const pad_t* a, const pad_t* b, int i, int j, int k, const int e[3], double h) {
    double near = F3(a, 0, 0, 0) + F3(a, e[0], e[1], e[2]);
    double nn = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        if (e[ax] != 0) continue;
        for (int s = -1; s <= 1; s += 2) {
            int t[3] = {0, 0, 0};
            t[ax] = s;
            nn += F3(a, t[0], t[1], t[2]) + F3(a, e[0] + t[0], e[1] + t[1], e[2] + t[2]);
        }
    }
    double ab = 0.25 * near + (1.0 / 16.0) * nn;
    return ab * (F3(b, e[0], e[1], e[2]) - F3(b, 0, 0, 0)) / h;
}
static double div_100(const pad_t* a, const pad_t* b, int i, int j, int k, double h) { /* Eq. divergence_100 */
    double s = 0.0;
    for (int ax = 0; ax < 3; ++ax)
        for (int sg = -1; sg <= 1; sg += 2) {
            int e[3] = {0, 0, 0};
            e[ax] = sg;
            s += flux_100(a, b, i, j, k, e, h);
        }
    return s / h;
}
/* <110> flux towards d = e1 + e2 (two nonzero components):
 * alpha-bar = 3/16 (four nearest) + 1/32 (eight next-nearest) */
static double flux_110(const pad_t* a, const pad_t* b, int i, int j, int k, const int d[3], double h) {
    int ax3 = d[0] == 0 ? 0 : (d[1] == 0 ? 1 : 2);
    int e1[3] = {0, 0, 0}, e2[3] = {0, 0, 0};
    int first = 1;
    for (int ax = 0; ax < 3; ++ax) {
        if (ax == ax3) continue;
        if (first) { e1[ax] = d[ax]; first = 0; }
        else e2[ax] = d[ax];
    }
    double near = F3(a, 0, 0, 0) + F3(a, e1[0], e1[1], e1[2]) + F3(a, e2[0], e2[1], e2[2]) + F3(a, d[0], d[1], d[2]);
    double nn = 0.0;
    for (int s = -1; s <= 1; s += 2) {
        int t[3] = {0, 0, 0};
        t[ax3] = s;
        nn += F3(a, t[0], t[1], t[2]) + F3(a, e1[0] + t[0], e1[1] + t[1], e1[2] + t[2]) +
              F3(a, e2[0] + t[0], e2[1] + t[1], e2[2] + t[2]) + F3(a, d[0] + t[0], d[1] + t[1], d[2] + t[2]);
    }
    double ab = (3.0 / 16.0) * near + (1.0 / 32.0) * nn;
    return ab * (F3(b, d[0], d[1], d[2]) - F3(b, 0, 0, 0)) / (SQ2 * h);
}
static double div_010(const pad_t* a, const pad_t* b, int i, int j, int k, double h) { /* Eq. divergence_110 */
    double s = 0.0;
    for (int ax3 = 0; ax3 < 3; ++ax3)
        for (int s1 = -1; s1 <= 1; s1 += 2)
            for (int s2 = -1; s2 <= 1; s2 += 2) {
                int d[3] = {0, 0, 0}, c = 0;
                for (int ax = 0; ax < 3; ++ax) {
                    if (ax == ax3) continue;
                    d[ax] = c == 0 ? s1 : s2;
                    ++c;
                }
                s += flux_110(a, b, i, j, k, d, h);
            }
    return s / (2.0 * SQ2 * h);
}
/* <111> flux: alpha-bar = mean over the eight corners of the cube spanned */
static double div_001(const pad_t* a, const pad_t* b, int i, int j, int k, double h) { /* Eq. divergence_111 */
    double s = 0.0;
    for (int sx = -1; sx <= 1; sx += 2)
        for (int sy = -1; sy <= 1; sy += 2)
            for (int sz = -1; sz <= 1; sz += 2) {
                double ab = 0.0;
                for (int cx = 0; cx <= 1; ++cx)
                    for (int cy = 0; cy <= 1; ++cy)
                        for (int cz = 0; cz <= 1; ++cz) ab += F3(a, cx * sx, cy * sy, cz * sz);
                ab *= 0.125;
                s += ab * (F3(b, sx, sy, sz) - F3(b, 0, 0, 0)) / (SQ3 * h);
            }
    return s * SQ3 / (4.0 * h);
}
static double div_120(const pad_t* a, const pad_t* b, int i, int j, int k, double h) {
    return (1.0 / 3.0) * div_100(a, b, i, j, k, h) + (2.0 / 3.0) * div_010(a, b, i, j, k, h);
}

/* S_{1,0,0} divergence: <100> fluxes with a two-point face mean (R-S10) */
static double div_std_3d(const pad_t* a, const pad_t* b, int i, int j, int k, double h) {
    double s = 0.0;
    for (int ax = 0; ax < 3; ++ax)
        for (int sg = -1; sg <= 1; sg += 2) {
            int e[3] = {0, 0, 0};
            e[ax] = sg;
            s += 0.5 * (F3(a, e[0], e[1], e[2]) + F3(a, 0, 0, 0)) * (F3(b, e[0], e[1], e[2]) - F3(b, 0, 0, 0)) / h;
        }
    return s / h;
}

/* face gradient at the <100> face towards e: normal two-point difference,
 * transverse four-point means of centred differences (R-ANISO) */
static void face_grad_3d(const pad_t* b, int i, int j, int k, const int e[3], double h, double g[3]) {
    for (int ax = 0; ax < 3; ++ax) {
        if (e[ax] != 0) {
            g[ax] = (F3(b, e[0], e[1], e[2]) - F3(b, 0, 0, 0)) / h * (double)e[ax];
        } else {
            int t[3] = {0, 0, 0};
            t[ax] = 1;
            g[ax] = (F3(b, e[0] + t[0], e[1] + t[1], e[2] + t[2]) + F3(b, t[0], t[1], t[2]) -
                     F3(b, e[0] - t[0], e[1] - t[1], e[2] - t[2]) - F3(b, -t[0], -t[1], -t[2])) /
                    (4.0 * h);
        }
    }
}
static double at_std_3d(const pad_t* a, const pad_t* b, int i, int j, int k, double h, double guard2) {
    double s = 0.0;
    for (int ax = 0; ax < 3; ++ax)
        for (int sg = -1; sg <= 1; sg += 2) {
            int e[3] = {0, 0, 0};
            e[ax] = sg;
            double g[3];
            face_grad_3d(b, i, j, k, e, h, g);
            double m2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
            if (m2 * h * h < guard2) continue;
            s += 0.5 * (F3(a, e[0], e[1], e[2]) + F3(a, 0, 0, 0)) * ((F3(b, e[0], e[1], e[2]) - F3(b, 0, 0, 0)) / h) /
                 sqrt(m2);
        }
    return s / h;
}

/* ------------------------------------------------------------------------- */
/* anisotropy: a_s(n) for cubic symmetry in the grain's crystal frame         */
/* ------------------------------------------------------------------------- */
/* R (row-major 3x3) maps crystal coordinates to lab coordinates; the crystal
 * components of a lab vector g are R^T g.  In the crystal frame
 *   a_s = 1 - 3 eps4 + 4 eps4 sum_i n_i^4,
 * which in 2D equals 1 + eps4 cos 4(theta - alpha0) of Eq. anis_function.
 * J = a_s^2 g + |g|^2 a_s d a_s / d g is the gradient with respect to g of
 * a_s^2 |g|^2 / 2, so that the first three terms of Eq. PF_a are div J.
 * Returns a_s; writes (J - g) in lab coordinates.  Below the guard |g|^2 h^2
 * < guard2 the normal is undefined: a_s = 1 and J - g = 0 (reading R-GUARD). */
double or_aniso(int dim, const double R[9], double eps4, const double g[3], double h, double guard2, double jmg[3]) {
    double gc[3] = {0, 0, 0};
    for (int p = 0; p < dim; ++p)
        for (int q = 0; q < dim; ++q) gc[p] += R[q * 3 + p] * g[q];
    double r2 = 0.0, s4 = 0.0;
    for (int p = 0; p < dim; ++p) {
        r2 += gc[p] * gc[p];
        s4 += gc[p] * gc[p] * gc[p] * gc[p];
    }
    for (int p = 0; p < 3; ++p) jmg[p] = 0.0;
    if (r2 * h * h < guard2) return 1.0;
    double a = 1.0 - 3.0 * eps4 + 4.0 * eps4 * s4 / (r2 * r2);
    double jc[3];
    for (int p = 0; p < dim; ++p) {
        double da = 16.0 * eps4 * (gc[p] * gc[p] * gc[p] / (r2 * r2) - gc[p] * s4 / (r2 * r2 * r2));
        jc[p] = a * a * gc[p] + r2 * a * da - gc[p];
    }
    for (int p = 0; p < dim; ++p) {
        double s = 0.0;
        for (int q = 0; q < dim; ++q) s += R[p * 3 + q] * jc[q];
        jmg[p] = s;
    }
    return a;
}

/* ------------------------------------------------------------------------- */
/* one time step                                                              */
/* ------------------------------------------------------------------------- */
static int is_iso(int scheme) { return scheme == OR_S21 || scheme == OR_SBAR21 || scheme == OR_SBAR120; }

static double guard_of(void) { return 1e-20; }

/* d psi / dt at one interior cell from Eq. PF_a (isothermal: F1 = 1, F2 = U).
 * grad2 / lap are the scheme's G and L; N = div(J - grad psi) on <10>/<100>
 * faces; a_c from the centred gradient. */
static double dpsi_dt_2d(const or_params* q, const pad_t* psi, const pad_t* phi, const pad_t* U, const pad_t* gr,
                         const double* rot, int i, int j, double t) {
    double h = q->h;
    const double* R = rot + 9 * (int)V2(gr, i, j);
    double L = is_iso(q->scheme) ? lap_21(psi, i, j, h) : lap_10(psi, i, j, h);
    double G = is_iso(q->scheme) ? grad2_21(psi, i, j, h) : grad2_10(psi, i, j, h);
    double gc[3] = {(V2(psi, i + 1, j) - V2(psi, i - 1, j)) / (2.0 * h), (V2(psi, i, j + 1) - V2(psi, i, j - 1)) / (2.0 * h), 0};
    double tmp[3];
    double ac = or_aniso(2, R, q->eps4, gc, h, guard_of(), tmp);
    static const int d[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    double N = 0.0;
    for (int f = 0; f < 4; ++f) {
        double g[3] = {0, 0, 0}, jmg[3];
        face_grad_2d(psi, i, j, d[f][0], d[f][1], h, g);
        or_aniso(2, R, q->eps4, g, h, guard_of(), jmg);
        N += (d[f][0] != 0 ? jmg[0] * d[f][0] : jmg[1] * d[f][1]);
    }
    N /= h;
    double ph = V2(phi, i, j), u = V2(U, i, j);
    if (q->thermal) {
        /* Eq. PF_a with the frozen-temperature functions F1, F2 */
        double zeta = (j * h - q->yT - q->Vp * t) / q->lT;
        double F1 = 1.0 - (1.0 - q->k) * zeta, F2 = u + zeta;
        return ((L + N + SQ2 * (ph - q->lambda * (1.0 - ph * ph) * F2)) / (ac * ac) - SQ2 * ph * G) / F1;
    }
    return (L + N + SQ2 * (ph - q->lambda * (1.0 - ph * ph) * u)) / (ac * ac) - SQ2 * ph * G;
}

static double dpsi_dt_3d(const or_params* q, const pad_t* psi, const pad_t* phi, const pad_t* U, const pad_t* gr,
                         const double* rot, int i, int j, int k, double t) {
    double h = q->h;
    const double* R = rot + 9 * (int)V3(gr, i, j, k);
    double L = is_iso(q->scheme) ? lap_120(psi, i, j, k, h) : lap_100(psi, i, j, k, h);
    double G = is_iso(q->scheme) ? grad2_120(psi, i, j, k, h) : grad2_100(psi, i, j, k, h);
    double gc[3] = {(F3(psi, 1, 0, 0) - F3(psi, -1, 0, 0)) / (2.0 * h), (F3(psi, 0, 1, 0) - F3(psi, 0, -1, 0)) / (2.0 * h),
                    (F3(psi, 0, 0, 1) - F3(psi, 0, 0, -1)) / (2.0 * h)};
    double tmp[3];
    double ac = or_aniso(3, R, q->eps4, gc, h, guard_of(), tmp);
    double N = 0.0;
    for (int ax = 0; ax < 3; ++ax)
        for (int sg = -1; sg <= 1; sg += 2) {
            int e[3] = {0, 0, 0};
            e[ax] = sg;
            double g[3], jmg[3];
            face_grad_3d(psi, i, j, k, e, h, g);
            or_aniso(3, R, q->eps4, g, h, guard_of(), jmg);
            N += jmg[ax] * sg;
        }
    N /= h;
    double ph = F3(phi, 0, 0, 0), u = F3(U, 0, 0, 0);
    if (q->thermal) {
        /* Eq. PF_a with the frozen-temperature functions F1, F2 (pulling along +y) */
        double zeta = (j * h - q->yT - q->Vp * t) / q->lT;
        double F1 = 1.0 - (1.0 - q->k) * zeta, F2 = u + zeta;
        return ((L + N + SQ2 * (ph - q->lambda * (1.0 - ph * ph) * F2)) / (ac * ac) - SQ2 * ph * G) / F1;
    }
    return (L + N + SQ2 * (ph - q->lambda * (1.0 - ph * ph) * u)) / (ac * ac) - SQ2 * ph * G;
}

static int check_params(const or_params* q) {
    if (!q || (q->dim != 2 && q->dim != 3)) return -1;
    if (q->nx < 4 || q->ny < 4 || (q->dim == 3 && q->nz < 4)) return -1;
    if (q->dim == 2 && q->scheme > OR_SBAR21) return -1;
    if (q->dim == 3 && q->scheme != OR_S100 && q->scheme != OR_SBAR120) return -1;
    if (!(q->h > 0) || !(q->dt > 0)) return -1;
    if (q->thermal && !(q->lT > 0)) return -1;
    if (q->time_level != OR_T1 && q->time_level != OR_T0) return -1;
    return 0;
}

/* Advance psi, U (length nx*ny[*nz], x fastest) by nsteps explicit Euler
 * steps (Sec. 3.3.1).  grain holds per-cell indices into rot (n_grains 3x3
 * crystal-to-lab matrices, row-major).  If dpsi_out is given, it receives
 * d psi/dt of the last step.  Time levels follow reading T1: the U equation
 * uses phi^{n+1} on its left-hand side and delta phi = phi^{n+1} - phi^n for
 * d phi/dt; D uses phi^n and U^n, the anti-trapping term psi^n. */
int or_step(const or_params* q, int n_grains, const double* rot, const int16_t* grain, double* psi, double* U,
            long nsteps, double* dpsi_out) {
    if (check_params(q)) return -1;
    size_t N = (size_t)q->nx * q->ny * (q->dim == 3 ? q->nz : 1);
    for (size_t c = 0; c < N; ++c)
        if (grain[c] < 0 || grain[c] >= n_grains) return -2;
    pad_t Ppsi, Pphi, PU, Pg, Pnew, Pdphi, Palpha, Pomp;
    pad_t* all[] = {&Ppsi, &Pphi, &PU, &Pg, &Pnew, &Pdphi, &Palpha, &Pomp};
    for (int t = 0; t < 8; ++t)
        if (pad_alloc(all[t], q)) return -3;
    double* gd = (double*)malloc(N * sizeof(double));
    double* psin = (double*)malloc(N * sizeof(double));
    double* dpsi = (double*)malloc(N * sizeof(double));
    double* tmp = (double*)malloc(N * sizeof(double));
    for (size_t c = 0; c < N; ++c) gd[c] = (double)grain[c];
    pad_fill(&Pg, gd, q->bc);
    const double h = q->h, dt = q->dt, k = q->k, guard2 = guard_of();
    const int nz = q->dim == 3 ? q->nz : 1;
    size_t padN = (size_t)Ppsi.sx * Ppsi.sy * (nz + 2 * Ppsi.oz);

    for (long s = 0; s < nsteps; ++s) {
        /* pass 0 + 1: ghosts, phi = tanh(psi / sqrt 2) (Eq. 1) */
        pad_fill(&Ppsi, psi, q->bc);
        pad_fill(&PU, U, q->bc);
#pragma omp parallel for schedule(static)
        for (size_t c = 0; c < padN; ++c) Pphi.v[c] = tanh(Ppsi.v[c] / SQ2);
        /* pass 2: d psi/dt and psi' at every cell */
#pragma omp parallel for collapse(2) schedule(static)
        for (int kk = 0; kk < nz; ++kk)
            for (int j = 0; j < q->ny; ++j)
                for (int i = 0; i < q->nx; ++i) {
                    size_t c = ((size_t)kk * q->ny + j) * q->nx + i;
                    double r = q->dim == 2 ? dpsi_dt_2d(q, &Ppsi, &Pphi, &PU, &Pg, rot, i, j, q->t0 + (double)s * dt)
                                           : dpsi_dt_3d(q, &Ppsi, &Pphi, &PU, &Pg, rot, i, j, kk, q->t0 + (double)s * dt);
                    dpsi[c] = r;
                    psin[c] = psi[c] + dt * r;
                }
        /* pass 3: phi', delta phi with ghosts from psi' (T1), or the chain-rule
         * increment dt (1 - phi^2)/sqrt2 dpsi/dt with ghosts from dpsi/dt and
         * phi^n in place of phi' (T0) */
        if (q->time_level == OR_T0) {
            pad_fill(&Pnew, dpsi, q->bc);
#pragma omp parallel for schedule(static)
            for (size_t c = 0; c < padN; ++c) {
                double ph = Pphi.v[c];
                Pdphi.v[c] = dt * (1.0 - ph * ph) / SQ2 * Pnew.v[c];
                Pnew.v[c] = ph; /* phi^n on the left-hand side */
            }
        } else {
            pad_fill(&Pnew, psin, q->bc);
#pragma omp parallel for schedule(static)
            for (size_t c = 0; c < padN; ++c) {
                double phn = tanh(Pnew.v[c] / SQ2);
                Pdphi.v[c] = phn - Pphi.v[c];
                Pnew.v[c] = phn; /* Pnew now holds phi' */
            }
        }
        /* alpha of the U equation: 1 - phi (D term) in Pomp, and
         * (1 + (1-k) U) d phi/dt / sqrt 2 (anti-trapping) in Palpha */
#pragma omp parallel for schedule(static)
        for (size_t c = 0; c < padN; ++c) {
            Pomp.v[c] = 1.0 - Pphi.v[c];
            Palpha.v[c] = (1.0 + (1.0 - k) * PU.v[c]) * Pdphi.v[c] / (SQ2 * dt);
        }
        /* pass 4: U' (Eq. PF_b, conservative form of reading T1) */
#pragma omp parallel for collapse(2) schedule(static)
        for (int kk = 0; kk < nz; ++kk)
            for (int j = 0; j < q->ny; ++j)
                for (int i = 0; i < q->nx; ++i) {
                    size_t c = ((size_t)kk * q->ny + j) * q->nx + i;
                    double Dterm, Aterm;
                    if (q->dim == 2) {
                        switch (q->scheme) {
                            case OR_S10:
                                Dterm = div_std_2d(&Pomp, &PU, i, j, h);
                                Aterm = at_std_2d(&Palpha, &Ppsi, i, j, h, guard2);
                                break;
                            case OR_S21:
                                Dterm = div_21(&Pomp, &PU, i, j, h);
                                Aterm = at_21(&Palpha, &Ppsi, i, j, h, guard2);
                                break;
                            default:
                                Dterm = div_21(&Pomp, &PU, i, j, h);
                                Aterm = div_21(&Palpha, &Ppsi, i, j, h);
                                break;
                        }
                    } else {
                        if (q->scheme == OR_S100) {
                            Dterm = div_std_3d(&Pomp, &PU, i, j, kk, h);
                            Aterm = at_std_3d(&Palpha, &Ppsi, i, j, kk, h, guard2);
                        } else {
                            Dterm = div_120(&Pomp, &PU, i, j, kk, h);
                            Aterm = div_120(&Palpha, &Ppsi, i, j, kk, h);
                        }
                    }
                    double u = U[c];
                    double phn = *PA(&Pnew, i, j, kk), dph = *PA(&Pdphi, i, j, kk);
                    tmp[c] = u + (dt * (q->D * Dterm + Aterm) + (1.0 + (1.0 - k) * u) * dph) / (1.0 + k - (1.0 - k) * phn);
                }
        memcpy(psi, psin, N * sizeof(double));
        memcpy(U, tmp, N * sizeof(double));
    }
    if (dpsi_out && nsteps > 0) memcpy(dpsi_out, dpsi, N * sizeof(double));
    for (int t = 0; t < 8; ++t) free(all[t]->v);
    free(gd); free(psin); free(dpsi); free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* operator evaluation on a whole field (for the pins)                        */
/* ------------------------------------------------------------------------- */
enum {
    OP_LAP_10 = 0, OP_LAP_01, OP_LAP_21, OP_GRAD2_10, OP_GRAD2_01, OP_GRAD2_21,
    OP_DIV_10, OP_DIV_01, OP_DIV_21, OP_DIV_STD2, OP_AT_STD2, OP_AT_21,
    OP_LAP_100 = 20, OP_LAP_010, OP_LAP_001, OP_LAP_120, OP_GRAD2_100, OP_GRAD2_010, OP_GRAD2_001, OP_GRAD2_120,
    OP_DIV_100, OP_DIV_010, OP_DIV_001, OP_DIV_120, OP_DIV_STD3, OP_AT_STD3,
    OP_ANISO_N = 40
};

/* out[c] = op(a, b) at every cell; bc and h from q; rot/eps4 only for
 * OP_ANISO_N, which evaluates N = div(J - grad a) on the face shell with the
 * single rotation rot. */
int or_apply(const or_params* q, int op, const double* a, const double* b, const double* rot, double* out) {
    if (!q || (q->dim != 2 && q->dim != 3)) return -1;
    pad_t A, B;
    if (pad_alloc(&A, q) || pad_alloc(&B, q)) return -3;
    pad_fill(&A, a, q->bc);
    if (b) pad_fill(&B, b, q->bc);
    const double h = q->h, guard2 = guard_of();
    const int nz = q->dim == 3 ? q->nz : 1;
    int rc = 0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < q->ny; ++j)
            for (int i = 0; i < q->nx; ++i) {
                size_t c = ((size_t)k * q->ny + j) * q->nx + i;
                double v = 0.0;
                switch (op) {
                    case OP_LAP_10: v = lap_10(&A, i, j, h); break;
                    case OP_LAP_01: v = lap_01(&A, i, j, h); break;
                    case OP_LAP_21: v = lap_21(&A, i, j, h); break;
                    case OP_GRAD2_10: v = grad2_10(&A, i, j, h); break;
                    case OP_GRAD2_01: v = grad2_01(&A, i, j, h); break;
                    case OP_GRAD2_21: v = grad2_21(&A, i, j, h); break;
                    case OP_DIV_10: v = div_10(&A, &B, i, j, h); break;
                    case OP_DIV_01: v = div_01(&A, &B, i, j, h); break;
                    case OP_DIV_21: v = div_21(&A, &B, i, j, h); break;
                    case OP_DIV_STD2: v = div_std_2d(&A, &B, i, j, h); break;
                    case OP_AT_STD2: v = at_std_2d(&A, &B, i, j, h, guard2); break;
                    case OP_AT_21: v = at_21(&A, &B, i, j, h, guard2); break;
                    case OP_LAP_100: v = lap_100(&A, i, j, k, h); break;
                    case OP_LAP_010: v = lap_010(&A, i, j, k, h); break;
                    case OP_LAP_001: v = lap_001(&A, i, j, k, h); break;
                    case OP_LAP_120: v = lap_120(&A, i, j, k, h); break;
                    case OP_GRAD2_100: v = grad2_100(&A, i, j, k, h); break;
                    case OP_GRAD2_010: v = grad2_010(&A, i, j, k, h); break;
                    case OP_GRAD2_001: v = grad2_001(&A, i, j, k, h); break;
                    case OP_GRAD2_120: v = grad2_120(&A, i, j, k, h); break;
                    case OP_DIV_100: v = div_100(&A, &B, i, j, k, h); break;
                    case OP_DIV_010: v = div_010(&A, &B, i, j, k, h); break;
                    case OP_DIV_001: v = div_001(&A, &B, i, j, k, h); break;
                    case OP_DIV_120: v = div_120(&A, &B, i, j, k, h); break;
                    case OP_DIV_STD3: v = div_std_3d(&A, &B, i, j, k, h); break;
                    case OP_AT_STD3: v = at_std_3d(&A, &B, i, j, k, h, guard2); break;
                    case OP_ANISO_N: {
                        double N = 0.0;
                        for (int ax = 0; ax < q->dim; ++ax)
                            for (int sg = -1; sg <= 1; sg += 2) {
                                double g[3] = {0, 0, 0}, jmg[3];
                                if (q->dim == 2)
                                    face_grad_2d(&A, i, j, ax == 0 ? sg : 0, ax == 1 ? sg : 0, h, g);
                                else {
                                    int e[3] = {0, 0, 0};
                                    e[ax] = sg;
                                    face_grad_3d(&A, i, j, k, e, h, g);
                                }
                                or_aniso(q->dim, rot, q->eps4, g, h, guard2, jmg);
                                N += jmg[ax] * sg;
                            }
                        v = N / h;
                        break;
                    }
                    default: rc = -1;
                }
                out[c] = v;
            }
    free(A.v);
    free(B.v);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* initial condition (reading R-INIT / R-GRAIN)                               */
/* ------------------------------------------------------------------------- */
/* seeds: n_seeds records (x, y, z, r) in units of W; seed_grain: grain index
 * of each seed.  psi = max_s (r_s - |x - c_s|), the signed distance to the
 * union of the seed spheres; the grain of a cell is that of the seed
 * attaining the maximum (ties: lowest seed index); U = U0. */
int or_init_seeds(const or_params* q, double U0, int n_seeds, const double* seeds, const int16_t* seed_grain,
                  double* psi, double* U, int16_t* grain) {
    if (check_params(q) || n_seeds < 1) return -1;
    const int nz = q->dim == 3 ? q->nz : 1;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < q->ny; ++j)
            for (int i = 0; i < q->nx; ++i) {
                size_t c = ((size_t)k * q->ny + j) * q->nx + i;
                double x = i * q->h, y = j * q->h, z = q->dim == 3 ? k * q->h : 0.0;
                double best = -INFINITY;
                int bs = 0;
                for (int s = 0; s < n_seeds; ++s) {
                    double dx = x - seeds[4 * s], dy = y - seeds[4 * s + 1], dz = q->dim == 3 ? z - seeds[4 * s + 2] : 0.0;
                    double v = seeds[4 * s + 3] - sqrt(dx * dx + dy * dy + dz * dz);
                    if (v > best) { best = v; bs = s; }
                }
                psi[c] = best;
                U[c] = U0;
                grain[c] = seed_grain[bs];
            }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* observables (reading R-TIP; solute from Eq. Supersaturation)               */
/* ------------------------------------------------------------------------- */
/* out[0..2] tip position, out[3] tip score (projection on the growth axis),
 * out[4] solute integral sum (1+k-(1-k)phi)(1+(1-k)U)/2 h^d,
 * out[5] solid fraction sum (1+phi)/2 / N, out[6] number of non-finite cells,
 * out[7] tip found (1/0), out[8] linear index of the tip cell,
 * out[9] growth angle in the xy plane (degrees, counter-clockwise from +y),
 * out[10] angle out of the xy plane (degrees; 0 in 2D).
 * grain = -1 uses every cell with grain 0's centre and axes. */
int or_observe(const or_params* q, int n_grains, const double* rot, const double* centres, const int16_t* grain,
               const double* psi, const double* U, int g, double* out) {
    if (check_params(q) || g < -2 || g >= n_grains) return -1;
    const int nz = q->dim == 3 ? q->nz : 1, dim = q->dim;
    const int gg = g < 0 ? 0 : g;
    const double* R = rot + 9 * gg;
    const double* cg = centres + 3 * gg;
    /* growth axis: the crystal axis (+-column of R) with the largest
     * y component; ties keep the first in the order (+a0, -a0, +a1, ...).
     * g = -2: the pulling axis +y (the most advanced interface along y that
     * Sec. 4.3.3 and 6.2.3 track in directional solidification) */
    double d[3] = {0, 0, 0}, best = -INFINITY;
    if (g == -2) d[1] = 1.0;
    for (int a = 0; a < dim && g != -2; ++a)
        for (int s = 1; s >= -1; s -= 2) {
            double yc = s * R[1 * 3 + a];
            if (yc > best) {
                best = yc;
                for (int p = 0; p < 3; ++p) d[p] = p < dim ? s * R[p * 3 + a] : 0.0;
            }
        }
    /* lattice axis closest to d (largest |d_a|, ties lowest a), its sign */
    int ea = 0;
    for (int a = 1; a < dim; ++a)
        if (fabs(d[a]) > fabs(d[ea])) ea = a;
    int es = d[ea] >= 0 ? 1 : -1;
    double bestsc = -INFINITY, tip[3] = {NAN, NAN, NAN};
    long tipc = -1;
    double sol = 0.0, sf = 0.0, nonfin = 0.0;
    const double k = q->k;
    for (int kk = 0; kk < nz; ++kk)
        for (int j = 0; j < q->ny; ++j)
            for (int i = 0; i < q->nx; ++i) {
                size_t c = ((size_t)kk * q->ny + j) * q->nx + i;
                double ps = psi[c], u = U[c];
                if (!isfinite(ps) || !isfinite(u)) { nonfin += 1.0; continue; }
                double ph = tanh(ps / SQ2);
                sol += (1.0 + k - (1.0 - k) * ph) * (1.0 + (1.0 - k) * u) / 2.0;
                sf += (1.0 + ph) / 2.0;
                if (g >= 0 && grain[c] != g) continue;
                if (!(ps >= 0.0)) continue;
                int ii = i, jj = j, kq = kk;
                if (ea == 0) ii += es; else if (ea == 1) jj += es; else kq += es;
                if (ii < 0 || jj < 0 || kq < 0 || ii >= q->nx || jj >= q->ny || kq >= nz) continue;
                double pn = psi[((size_t)kq * q->ny + jj) * q->nx + ii];
                if (!(pn < 0.0)) continue;
                double frac = ps / (ps - pn);
                double p[3] = {i * q->h, j * q->h, dim == 3 ? kk * q->h : 0.0};
                p[ea] += es * frac * q->h;
                double sc = 0.0;
                for (int a = 0; a < dim; ++a) sc += (p[a] - cg[a]) * d[a];
                if (sc > bestsc) {
                    bestsc = sc;
                    tipc = (long)c;
                    for (int a = 0; a < 3; ++a) tip[a] = p[a];
                }
            }
    double hd = dim == 3 ? q->h * q->h * q->h : q->h * q->h;
    size_t N = (size_t)q->nx * q->ny * nz;
    out[0] = tip[0]; out[1] = tip[1]; out[2] = tip[2];
    out[3] = bestsc;
    out[4] = sol * hd;
    out[5] = sf / (double)N;
    out[6] = nonfin;
    out[7] = tipc >= 0 ? 1.0 : 0.0;
    out[8] = (double)tipc;
    if (tipc >= 0) {
        double rx = tip[0] - cg[0], ry = tip[1] - cg[1], rz = dim == 3 ? tip[2] - cg[2] : 0.0;
        out[9] = atan2(-rx, ry) * 180.0 / M_PI;
        out[10] = atan2(rz, sqrt(rx * rx + ry * ry)) * 180.0 / M_PI;
    } else {
        out[9] = NAN;
        out[10] = NAN;
    }
    return 0;
}

/* explicit-Euler stability bound on dt used by the library's parameter check:
 * the largest |symbol| h^2 of the scheme's Laplacian is 16/3 for L_{2,1} and
 * L_{1,2,0}, 8 for L_{1,0} and 12 for L_{1,0,0}; the liquid diffusivity D and
 * the psi mobility 1 bound the coefficients. */
double or_dt_max(const or_params* q) {
    double lam = is_iso(q->scheme) ? 16.0 / 3.0 : (q->dim == 2 ? 8.0 : 12.0);
    double c = q->D > 1.0 ? q->D : 1.0;
    return 2.0 * q->h * q->h / (lam * c);
}

/* ------------------------------------------------------------------------- */
/* tip radius (Sec. 3.3.2, Sec. 6.2.2; reading R-RHO)                         */
/* ------------------------------------------------------------------------- */
/* The paper takes the psi = 0 contour, rotates it by minus the measured
 * growth angle so that the growth direction becomes the vertical axis, and
 * fits the parabola y = y_tip - (x - x_tip)^2 / (2 rho) to the part of the
 * contour within one radius behind the tip; in 3D it fits rho_x in the plane
 * spanned by the growth axis and the in-plane transverse axis, rho_z in the
 * plane spanned by the growth axis and z, and combines 1/rho = (1/rho_x +
 * 1/rho_z) / 2.  Steps here:
 *   frame   e_par = axis / |axis|; 2D: e_x = (e_par_y, -e_par_x); 3D: e_z = z
 *           minus its e_par component, normalised (x instead when the axis is
 *           within 1e-6 of z), e_x = e_z cross e_par
 *   contour for each transverse axis e and s = j h (j = -TR_J..-1, 1..TR_J):
 *           march r(t) = (tip + s e) - t e_par, t = m h / 4, m = 0..TR_M, psi
 *           interpolated multilinearly between cell centres; the first m >= 1
 *           with psi >= 0 gives the crossing t_j by linear interpolation
 *           between samples m-1 and m.  No sample if psi >= 0 at m = 0, if r
 *           leaves [0, (n-1) h] on an axis, or if no crossing by m = TR_M.
 *   fit     c = sum t_j s^2 / sum s^4 over the samples with t_j <= w, rho =
 *           1 / (2 c); w = TR_M h / 4 in the first round, then the previous
 *           rho (one radius behind the tip); TR_ROUNDS rounds.
 * out[0] rho, out[1] rho_x, out[2] rho_z (NaN in 2D), out[3] samples in the
 * last x fit, out[4] samples in the last z fit.  A fit without samples, or
 * with c <= 0, gives NaN. */
#define TR_J 32
#define TR_M 160
#define TR_ROUNDS 4

static double interp_psi(const or_params* q, const double* psi, const double r[3], int* inside) {
    const int n[3] = {q->nx, q->ny, q->dim == 3 ? q->nz : 1};
    int i0[3];
    double f[3];
    *inside = 1;
    for (int a = 0; a < 3; ++a) {
        if (a == 2 && q->dim == 2) {
            i0[a] = 0;
            f[a] = 0.0;
            continue;
        }
        double u = r[a] / q->h;
        if (!(u >= 0.0) || u > (double)(n[a] - 1)) {
            *inside = 0;
            return 0.0;
        }
        int i = (int)floor(u);
        if (i > n[a] - 2) i = n[a] - 2;
        i0[a] = i;
        f[a] = u - (double)i;
    }
#define TRV(di, dj, dk) psi[((size_t)(i0[2] + (dk)) * q->ny + (i0[1] + (dj))) * q->nx + (i0[0] + (di))]
    double v0 = (1.0 - f[1]) * ((1.0 - f[0]) * TRV(0, 0, 0) + f[0] * TRV(1, 0, 0)) +
                f[1] * ((1.0 - f[0]) * TRV(0, 1, 0) + f[0] * TRV(1, 1, 0));
    if (q->dim == 2) return v0;
    double v1 = (1.0 - f[1]) * ((1.0 - f[0]) * TRV(0, 0, 1) + f[0] * TRV(1, 0, 1)) +
                f[1] * ((1.0 - f[0]) * TRV(0, 1, 1) + f[0] * TRV(1, 1, 1));
#undef TRV
    return (1.0 - f[2]) * v0 + f[2] * v1;
}

/* crossings t_j of the lines along transverse axis e; t[j] = NaN: no sample */
static void tip_contour(const or_params* q, const double* psi, const double tip[3], const double epar[3],
                        const double e[3], double t[2 * TR_J]) {
    const double dt = q->h / 4.0;
    for (int l = 0; l < 2 * TR_J; ++l) {
        const int j = l < TR_J ? l - TR_J : l - TR_J + 1; /* -TR_J..-1, 1..TR_J */
        const double s = (double)j * q->h;
        double base[3];
        for (int a = 0; a < 3; ++a) base[a] = tip[a] + s * e[a];
        t[l] = NAN;
        double prev = 0.0;
        for (int m = 0; m <= TR_M; ++m) {
            const double tm = (double)m * dt;
            double r[3];
            for (int a = 0; a < 3; ++a) r[a] = base[a] - tm * epar[a];
            int inside;
            const double v = interp_psi(q, psi, r, &inside);
            if (!inside) break;
            if (v >= 0.0) {
                if (m >= 1) t[l] = (double)(m - 1) * dt + dt * (prev / (prev - v));
                break;
            }
            prev = v;
        }
    }
}

static double tip_fit(const or_params* q, const double t[2 * TR_J], int* used) {
    double w = (double)TR_M * (q->h / 4.0), rho = NAN;
    *used = 0;
    for (int round = 0; round < TR_ROUNDS; ++round) {
        double st = 0.0, s4 = 0.0;
        int n = 0;
        for (int l = 0; l < 2 * TR_J; ++l) {
            const int j = l < TR_J ? l - TR_J : l - TR_J + 1;
            const double s = (double)j * q->h;
            if (!(t[l] <= w)) continue;
            st += t[l] * (s * s);
            s4 += (s * s) * (s * s);
            ++n;
        }
        *used = n;
        if (n == 0 || !(st > 0.0)) return NAN;
        rho = 0.5 * (s4 / st);
        w = rho;
    }
    return rho;
}

int or_tip_radius(const or_params* q, const double* psi, const double tip[3], const double axis[3], double* out) {
    if (check_params(q)) return -1;
    const int dim = q->dim;
    double epar[3] = {axis[0], axis[1], dim == 3 ? axis[2] : 0.0};
    const double na = sqrt(epar[0] * epar[0] + epar[1] * epar[1] + epar[2] * epar[2]);
    if (!(na > 0.0)) return -1;
    for (int a = 0; a < 3; ++a) epar[a] /= na;
    double ex[3], ez[3] = {0.0, 0.0, 0.0};
    if (dim == 2) {
        ex[0] = epar[1];
        ex[1] = -epar[0];
        ex[2] = 0.0;
    } else {
        double ref[3] = {0.0, 0.0, 1.0};
        if (fabs(epar[2]) > 1.0 - 1e-6) {
            ref[0] = 1.0;
            ref[2] = 0.0;
        }
        const double pr = ref[0] * epar[0] + ref[1] * epar[1] + ref[2] * epar[2];
        for (int a = 0; a < 3; ++a) ez[a] = ref[a] - pr * epar[a];
        const double nz = sqrt(ez[0] * ez[0] + ez[1] * ez[1] + ez[2] * ez[2]);
        for (int a = 0; a < 3; ++a) ez[a] /= nz;
        ex[0] = ez[1] * epar[2] - ez[2] * epar[1];
        ex[1] = ez[2] * epar[0] - ez[0] * epar[2];
        ex[2] = ez[0] * epar[1] - ez[1] * epar[0];
    }
    double t[2 * TR_J];
    int nx_used = 0, nz_used = 0;
    tip_contour(q, psi, tip, epar, ex, t);
    const double rx = tip_fit(q, t, &nx_used);
    double rz = NAN;
    if (dim == 3) {
        tip_contour(q, psi, tip, epar, ez, t);
        rz = tip_fit(q, t, &nz_used);
    }
    out[0] = dim == 2 ? rx : 2.0 / (1.0 / rx + 1.0 / rz);
    out[1] = rx;
    out[2] = rz;
    out[3] = (double)nx_used;
    out[4] = (double)nz_used;
    return 0;
}
