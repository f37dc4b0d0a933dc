/*
 * pf.h -- C-ABI of the GB300 (sm_103a) library for the explicit time step of
 * the quantitative binary-alloy phase-field model with the O(h^2)-isotropic
 * finite differences of Ji, Molavi Tabrizi & Karma, arXiv:2110.12448.
 *
 * The model (Sec. 2.1, Eqs. PF_a and PF_b, isothermal: F1 = 1, F2 = U):
 *   a_s^2 dpsi/dt = div J - sqrt2 phi a_s^2 |grad psi|^2
 *                   + sqrt2 [phi - lambda (1 - phi^2) U],
 *   J = a_s^2 grad psi + |grad psi|^2 a_s d a_s / d(grad psi),
 *   (1 + k - (1-k) phi) dU/dt = D div[(1 - phi) grad U] + (anti-trapping)
 *                   + [1 + (1-k) U] d phi/dt,
 *   phi = tanh(psi / sqrt2)                                         (Eq. 1)
 * with the cubic anisotropy a_s of Eq. anis_function evaluated in each
 * grain's rotated crystal frame, explicit Euler in time (Sec. 3.3.1) and
 * no-flux (cell-centred mirror) walls.
 *
 * Schemes (Sec. 3.3.1 and Sec. 6.2.1):
 *   PF_S10      L_{1,0}, G_{1,0}, <10> divergence, standard anti-trapping
 *   PF_S21      L_{2,1}, G_{2,1}, D~_{2,1}, standard anti-trapping A_{2,1}
 *               with the 21-point |grad psi| of App. B
 *   PF_SBAR21   L_{2,1}, G_{2,1}, D~_{2,1} for D and the approximated
 *               anti-trapping of Eq. Anti_approx
 *   PF_S100     3D <100> scheme with standard anti-trapping
 *   PF_SBAR120  L_{1,2,0}, G_{1,2,0}, D~_{1,2,0} for D and Eq. Anti_approx
 * The O(eps4) anisotropy terms use the <10>/<100> face shell (Sec. 2.2).
 *
 * Conventions for every entry point:
 *   - return 0 (PF_OK) or a negative PF_ERR_* code; no exception crosses
 *     the ABI; pf_status_string() names a code.
 *   - fields are row-major with x fastest: index (k*ny + j)*nx + i; cell
 *     (i,j,k) sits at (i h, j h, k h) in units of the interface width W.
 *   - the library never allocates device memory.  The caller passes one
 *     device buffer of pf_required_bytes() bytes (256-byte aligned) that
 *     must outlive the handle, and a cudaStream_t (as void*) on which all
 *     work of the handle is queued; NULL means the legacy default stream.
 *   - host arrays are read or written during the call only (copied).
 *   - a handle is used from one host thread at a time.
 */
#ifndef PF_H
#define PF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pf_sim pf_sim;
typedef struct pf_group pf_group;

typedef enum { PF_S10 = 0, PF_S21 = 1, PF_SBAR21 = 2, PF_S100 = 3, PF_SBAR120 = 4 } pf_scheme;
/* Arithmetic and storage of the fields:
 *   PF_F32   FP32 fields, FP32 arithmetic (fast exp2 / reciprocal forms);
 *   PF_F64   FP64 fields and arithmetic;
 *   PF_F32C  FP32 arithmetic on a compensated state: psi and U each stored as
 *            an FP32 pair hi + lo (about 48 significant bits, 8 bytes per
 *            cell and field), updated by error-free two-sums; phi from the
 *            library tanh, delta phi from the addition theorem of tanh and
 *            the U differences of the diffusion term with their lo halves.
 *            2D, isothermal, mirror walls and the T1 time level only.  The
 *            host sees FP64 fields (pf_get_fields / pf_set_fields take FP64
 *            arrays, hi + lo). */
typedef enum { PF_F32 = 0, PF_F64 = 1, PF_F32C = 2 } pf_precision;

enum {
    PF_OK = 0,
    PF_ERR_INVALID = -1,   /* bad argument, size or parameter */
    PF_ERR_BUDGET = -2,    /* caller buffer smaller than required */
    PF_ERR_CUDA = -3,      /* a CUDA call failed (details: pf_last_cuda_error) */
    PF_ERR_NONFINITE = -4, /* observe found NaN/Inf in psi or U */
    PF_ERR_TIMEOUT = -5,   /* a bounded device wait gave up */
    PF_ERR_STATE = -6      /* call not valid in the handle's state */
};

/* Boundary rule along x (y and z always use cell-centred mirrors). */
enum { PF_BC_MIRROR = 0, PF_BC_PERIODIC = 1 };
/* Thermal condition (Sec. 2.1). */
enum { PF_ISOTHERMAL = 0, PF_FROZEN_GRADIENT = 1 };
/* Time levels of the U update (Sec. 3.3.1 leaves them open):
 * PF_T1: U' = U + [dt (D~ D + A) + (1+(1-k)U) dphi] / (1+k-(1-k)phi'),
 *        dphi = phi' - phi, anti-trapping alpha from dphi / dt (conserves the
 *        solute exactly with mirror walls);
 * PF_T0: pure forward Euler of Eq. PF_b as printed: dphi replaced by
 *        dt (1-phi^2)/sqrt2 dpsi/dt (chain rule), phi^n instead of phi'
 *        (conserves the solute to O(dt) over a fixed time). */
enum { PF_T1 = 0, PF_T0 = 1 };
/* Kernels of a step (Sec. 3.3.1 describes two, a psi kernel then a U kernel):
 * PF_FUSED: one kernel per step, psi' and the U update from the same pass
 *   (d psi/dt stays on chip);
 * PF_TWO_KERNELS: the psi kernel writes psi' and d psi/dt to device memory,
 *   then the U kernel reads d psi/dt back (2D, PF_T0 time level, PF_F32 or
 *   PF_F64).  Same arithmetic as the fused T0 step; it costs the extra
 *   traffic of d psi/dt and a second read of psi and U. */
enum { PF_FUSED = 0, PF_TWO_KERNELS = 1 };

/* Problem statement (Sec. 2.1): grid, lattice spacing h (units of W), time
 * step dt (units of tau0), partition coefficient k, anisotropy strength
 * eps4, coupling lambda, diffusivity D (= a1 a2 W/d0), initial
 * supersaturation U0, scheme, arithmetic precision of the fields, capacity
 * of the grain table (>= 1) and of the seed list used by pf_init_seeds
 * (0 = 64).  Every axis needs at least 4 cells.
 *
 * Thermal condition: PF_ISOTHERMAL (F1 = 1, F2 = U) or
 * PF_FROZEN_GRADIENT: directional solidification in a frozen temperature
 * field pulled along +y (Eqs. Thermal_F1, Thermal_F2): with
 * zeta = (y - yT - Vp t) / lT, y = j h and t = step * dt,
 *   F1 = 1 - (1-k) zeta multiplies a_s^2 dpsi/dt in Eq. PF_a,
 *   F2 = U + zeta replaces U in its coupling term;
 * Vp >= 0 (pulling speed, W / tau0), lT > 0 (thermal length, W), yT the
 * position of the reference isotherm T0 at t = 0.  F1 must stay above 0.05
 * over the grid at t = 0.  bc_x = PF_BC_PERIODIC makes x periodic; y (and
 * z) keep the mirror (no-flux) walls, which meet an interface at 90 deg.
 *
 * dt must not exceed the explicit-Euler bound 2 h^2 / (Lambda max(D, 1/F1min)),
 * Lambda = 16/3 for the isotropic Laplacians, 8 for L_{1,0}, 12 for L_{1,0,0};
 * F1min = 1 except with PF_FROZEN_GRADIENT. */
typedef struct {
    int32_t dim, nx, ny, nz;
    double h, dt, k, eps4, lambda, D, U0;
    int32_t scheme;     /* pf_scheme */
    int32_t precision;  /* pf_precision */
    int32_t max_grains;
    int32_t max_seeds;
    int32_t bc_x;       /* PF_BC_MIRROR or PF_BC_PERIODIC */
    int32_t thermal;    /* PF_ISOTHERMAL or PF_FROZEN_GRADIENT */
    double Vp, lT, yT;  /* frozen gradient: pulling speed, thermal length, isotherm T0 at t = 0 */
    int32_t time_level; /* PF_T1 (default) or PF_T0 */
    int32_t kernels;    /* PF_FUSED (default) or PF_TWO_KERNELS */
} pf_params;

/* A spherical (circular in 2D) seed: centre (x, y, z) and radius r in units
 * of W, and the grain it belongs to. */
typedef struct {
    double x, y, z, r;
    int32_t grain;
    int32_t reserved;
} pf_seed;

/* Observation (tip tracking of Sec. 3.3.2 and 6.2.2, solute integral of
 * Eq. Supersaturation).  All reductions run in FP64 on the device. */
typedef struct {
    int64_t step;             /* steps taken by the handle */
    double t;                 /* step * dt */
    double tip[3];            /* tip position (NaN if no tip) */
    double v_tip;             /* |tip - previous tip| / elapsed time; 0 on first call */
    double angle_xy_deg;      /* growth angle in the xy plane, counter-clockwise from +y */
    double angle_out_deg;     /* elevation of the tip above the xy plane (3D) */
    double solute;            /* sum (1+k-(1-k)phi)(1+(1-k)U)/2 h^d */
    double solid_fraction;    /* mean of (1+phi)/2 */
    double tip_score;         /* projection of the tip on the growth axis */
    int64_t tip_index;        /* linear index of the tip cell, -1 if none */
    int32_t found;            /* 1 if a tip was found */
    int32_t nonfinite;        /* number of cells with NaN/Inf psi or U */
} pf_obs;

/* Tip operating state (Sec. 3.3.2 and 6.2.2): tip radius from a parabola fit
 * of the psi = 0 contour and the selection constant sigma* = 2 D d0* /
 * (rho^2 V) (Sec. 1 and 3.3.2), in units of W and tau0. */
typedef struct {
    double rho;         /* tip radius; 3D: 2 / (1/rho_x + 1/rho_z) (NaN: no fit) */
    double rho_x;       /* fit across the growth axis in its plane with x/y */
    double rho_z;       /* fit across the growth axis toward z (NaN in 2D) */
    double sigma_star;  /* 2 D d0* / (rho^2 v_tip); NaN if v_tip <= 0 or no fit */
    double d0_star;     /* (1 - (1-k) Omega) / k * a1 / lambda with Omega = -U0,
                           a1 = 5 sqrt2 / 8 (Sec. 2.1, isothermal) */
    double axis[3];     /* unit growth axis: tip minus the grain's centre */
    int32_t n_x, n_z;   /* contour samples in the final fits */
} pf_tip;

/* Device bytes the caller must supply to pf_create for these parameters
 * (0 if the parameters are invalid). */
size_t pf_required_bytes(const pf_params* p);

/* Create a simulation on caller-owned device memory dev_mem (bytes >=
 * pf_required_bytes(p), 256-byte aligned) and stream.  Validates p (sizes,
 * scheme vs dim, dt against the stability bound) and sets the grain table to
 * one grain with the identity rotation, every cell to grain 0, psi = -1e3
 * (liquid) and U = U0.  *out receives the handle. */
int pf_create(const pf_params* p, void* dev_mem, size_t bytes, void* stream, pf_sim** out);

/* Set n_grains (<= max_grains) crystal orientations.  rot9: n_grains row-major
 * 3x3 matrices mapping crystal to lab coordinates (2D uses the upper-left
 * 2x2); Sec. 2.1 imposes the orientation through such rotations.  centres3:
 * n_grains reference points (x, y, z) used by pf_observe for the tip
 * projection and growth angle, or NULL for the domain centre. */
int pf_set_grains(pf_sim* s, int n_grains, const double* rot9, const double* centres3);

/* psi = max over seeds of (r_s - |x - c_s|), the signed distance to the
 * union of seeds; grain = grain of the seed attaining the maximum (ties: the
 * lowest seed index); U = U0.  Computed in FP64 on the device.  seeds: host
 * array of n_seeds records, 1 <= n_seeds <= max_seeds, finite, each grain in
 * [0, n_grains); otherwise PF_ERR_INVALID and the fields are unchanged (a
 * handle that was never seeded holds the all-liquid state pf_create leaves). */
int pf_init_seeds(pf_sim* s, int n_seeds, const pf_seed* seeds);

/* Copy an explicit per-cell grain map (nx*ny*nz int16, values < n_grains).
 * The library remembers the largest index it has written into the map
 * (here and in pf_init_seeds); while that is 0, every cell is in grain 0 and
 * the 2D step reads no grain rows, with the same arithmetic.  A change of
 * grains (this call, pf_init_seeds, pf_set_grains) on a member of a group
 * takes effect at the group's next pf_group_step, which rebuilds that
 * member's instance record; the caller orders the change after the group's
 * queued work, as for any call on a member. */
int pf_set_grain_index(pf_sim* s, const int16_t* host_grain);
int pf_get_grain_index(pf_sim* s, int16_t* host_grain);

/* Advance n >= 0 explicit Euler steps, queued asynchronously on the stream
 * (one fused kernel launch per step). */
int pf_step(pf_sim* s, int64_t n);

/* Synchronise the stream and observe grain g (0 <= g < n_grains) or, with
 * g = -1, every cell with grain 0's centre and axes.  Tip: among cells of
 * the grain with psi >= 0 whose neighbour along the lattice axis closest to
 * the growth axis has psi < 0, the linearly interpolated psi = 0 crossing
 * with the largest projection on the growth axis (the crystal axis with the
 * largest +y component); ties go to the lowest cell index.  g = -2: every
 * cell, with +y as the growth axis: the most advanced interface along the
 * pulling axis, which Sec. 4.3.3 and 6.2.3 track in directional
 * solidification (unlike a tilted crystal axis it is periodic in x).
 * Returns PF_ERR_NONFINITE (with *out filled) when NaN/Inf cells exist. */
int pf_observe(pf_sim* s, int grain, pf_obs* out);

/* Synchronise the stream and measure the tip radius of grain g (-1 as in
 * pf_observe) at tip[3] (from pf_observe; z ignored in 2D), entirely on the
 * device.  The paper rotates the psi = 0 contour so that the measured growth
 * direction is vertical and fits y = y_tip - (x - x_tip)^2 / (2 rho) up to one
 * radius behind the tip (in 3D separately across the two transverse axes).
 * Here: growth axis e = tip - centre of g, normalised; transverse axes (2D)
 * e_x = (e_y, -e_x), (3D) e_z = z minus its e component, normalised (x when e
 * is within 1e-6 of z), e_x = e_z cross e.  For s = j h, j = -32..-1, 1..32,
 * psi is interpolated multilinearly along tip + s e_x - t e (and e_z), t =
 * m h / 4 up to 40 h; the first psi >= 0 gives the crossing t(s) by linear
 * interpolation.  rho = sum s^4 / (2 sum t s^2) over the crossings with t <=
 * w, w = 40 h and then the previous rho, four rounds.  sigma* uses v_tip (from
 * pf_observe; pass 0 to skip).  Returns PF_ERR_INVALID for a bad grain or a
 * non-finite tip; PF_OK with rho = NaN when the contour gives no fit. */
int pf_tip_radius(pf_sim* s, int grain, const double tip[3], double v_tip, pf_tip* out);

/* Checkpoint / restore of the current fields (nx*ny*nz elements of the
 * handle's precision each; FP64 for PF_F32C, whose hi + lo halves are joined
 * on the way out and split on the way in) and of the step counter. */
int pf_get_fields(pf_sim* s, void* psi_host, void* U_host);
int pf_set_fields(pf_sim* s, const void* psi_host, const void* U_host);
/* The same copies queued on the handle's stream without waiting: the host
 * arrays must stay valid (and, for pf_get_fields_async, unread) until the
 * stream has passed the copies -- pf_synchronize, or any later synchronising
 * call on the stream.  Copies from or to pinned (page-locked) host memory run
 * asynchronously at the full host-link rate; pageable memory makes the CUDA
 * runtime stage them.  Work of other streams (a group on another stream) is
 * not ordered against these copies: the caller orders it. */
int pf_set_fields_async(pf_sim* s, const void* psi_host, const void* U_host);
int pf_get_fields_async(pf_sim* s, void* psi_host, void* U_host);
/* Wait until all work queued on the handle's stream has finished. */
int pf_synchronize(pf_sim* s);
int pf_get_step(pf_sim* s, int64_t* step);
int pf_set_step(pf_sim* s, int64_t step);

/* Moving frame for directional solidification (Sec. 4.3.3 and 6.2.3 pull
 * the sample along +y; the paper does not say how its boxes follow the tip):
 * moves the state `rows` cells toward -y, as if the box had been moved up by
 * rows*h.  Cell (x, y, z) takes the values of (x, y + rows, z); the vacated
 * top rows are melt the frame moves into: psi continues the last row,
 * decreasing by h per row (a signed distance into the melt); U continues the
 * steady far field of a frame moving at Vp through the melt,
 * U0 + (U_last - U0) exp(-Vp k h / D) k rows beyond the last row (with no
 * frozen temperature, Vp = 0: a copy of the last row); the grain index is
 * copied.  The frozen
 * temperature is kept in place: yT decreases by rows*h, so the next step sees
 * the same temperature at every material point.  Later observations are in
 * the moved frame: the tips remembered for V and the grains' reference points
 * (pf_set_grains' centres) move with it, so growth angles and V carry on
 * unchanged.  1 <= rows < ny.
 * Synchronises the stream.  Errors: PF_ERR_INVALID (rows out of range, or a
 * frozen temperature that the moved frame would put where pf_create refuses
 * it: F1 = 1 - (1-k) zeta below 0.05 on the grid, or the explicit step
 * unstable at 1/F1, at the current step; nothing is moved; or a PF_F32C
 * handle), PF_ERR_STATE
 * (the handle belongs to a group), PF_ERR_CUDA. */
int pf_shift_frame(pf_sim* s, int rows);

/* Device addresses of the current psi, U (precision of the handle; for
 * PF_F32C the FP32 hi halves, each followed by its nx*ny*nz lo halves) and
 * the int16 grain map; valid until the next pf_step / pf_group_step. */
int pf_device_fields(pf_sim* s, void** psi, void** U, void** grain);

/* Tile shape of the fused kernel (cells per block along x, and the number
 * of rows (2D) or planes (3D) a block sweeps); 0 keeps the current value.
 * Used by the autotuner.  block_x must be one of the compiled widths. */
int pf_set_tile(pf_sim* s, int block_x, int block_y, int sweep);
int pf_get_tile(pf_sim* s, int* block_x, int* block_y, int* sweep);
/* Work units of the current tile that are resident on the device at once
 * (warps in 2D, blocks in 3D).  A persistent launch runs min(work items,
 * this) units, so a work list just below a whole multiple of it balances
 * best; the autotuner picks sweep lengths from it.  Returns the count (> 0)
 * or a negative PF_ERR_* code; needs a current CUDA device. */
int pf_resident_units(pf_sim* s);

/* Bounds-checked builds (compiled with -DPF_BOUNDS_CHECK): every global and
 * shared-memory index formed by the kernels is checked; an index outside its
 * array is counted, replaced by 0 (no access leaves the array) and the
 * source line of the first one kept.  Returns PF_OK with the totals over all
 * kernels since the library was loaded, or PF_ERR_STATE in a build without
 * the checks (counts 0). */
int pf_debug_bounds(unsigned long long* failures, int* first_line);

/* Host-side fault injection for tests of the error paths (no GPU fault is
 * made): after `after_steps` more steps have launched (pf_step or
 * pf_group_step, all handles of the process), the next step is not launched
 * and the call returns PF_ERR_CUDA with pf_last_cuda_error() naming the
 * injection; the handles advance by the steps that did launch (a graph
 * replay counts as its 16 steps and fails whole).  after_steps < 0 disarms. */
int pf_debug_inject_launch_failure(long long after_steps);

int pf_destroy(pf_sim* s);
const char* pf_status_string(int code);
/* Text of the last CUDA error seen by any call (thread-local). */
const char* pf_last_cuda_error(void);

/* Observation without any device allocation by the caller.
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc -- for example code that runs inside a host
 * application or plugin framework which owns every device allocation, or a
 * real-time loop that must not trigger the device-wide synchronisation an
 * allocation can cause -- but that already hold the fields in device memory.
 * It computes the same FP64 reductions as pf_observe on caller-given device
 * fields: psi_dev, U_dev (nx*ny*nz elements of p->precision) and, when
 * grain >= 0, the int16 grain map grain_dev; rot9 is the observed grain's
 * crystal-to-lab matrix (grain 0's for grain = -1) and centre3 its reference
 * point.  grain = -2 observes every cell with +y as the growth axis (the
 * pulling axis, as in pf_observe; rot9 is then not used for the axis).  Only
 * p->dim, nx, ny, nz, h, k and precision are read.  The call synchronises
 * `stream` (NULL = legacy default stream) and fills *out like pf_observe,
 * except step, t and v_tip, which are 0 (no history is kept).
 *
 * Scratch: instead of memory from the caller, the block partials live in a
 * fixed 22 KB array in the library's device globals, which every GPU that
 * loads the library holds until the process exits.  Every call looks up that
 * array's device address on the current device (cudaGetSymbolAddress, which
 * allocates nothing), so the entry point stays valid across a device reset;
 * the first call on a device may load the library's device code, so make it
 * before any stream capture.  All calls share the array:
 * calls whose work overlaps on a device (two streams, two host threads) race
 * and must be serialised by the caller.  Grids above PF_NOALLOC_MAX_CELLS
 * cells are rejected with PF_ERR_INVALID.  Never allocates device memory. */
#define PF_NOALLOC_MAX_CELLS (1LL << 34)
int pf_observe_fields_noalloc(const pf_params* p, const void* psi_dev, const void* U_dev, const int16_t* grain_dev,
                              const double* rot9, const double* centre3, int grain, void* stream, pf_obs* out);

/* ------------------------------------------------------------------------ */
/* Batching: many simulations stepped together by one persistent launch per  */
/* (dimension, scheme, precision) class, optionally replayed from a CUDA     */
/* graph.  The group owns no fields; members keep their own memory.          */
/* ------------------------------------------------------------------------ */

/* Device bytes for a group of up to max_instances members whose tiles total
 * at most max_work work items (pf_group_work_items counts a member's). */
size_t pf_group_required_bytes(int max_instances, int max_work);
int pf_group_work_items(const pf_sim* s);
int pf_group_create(int max_instances, int max_work, void* dev_mem, size_t bytes, void* stream, pf_group** out);
/* Members must not be stepped on their own while in the group. */
int pf_group_add(pf_group* g, pf_sim* s);
int pf_group_remove(pf_group* g, pf_sim* s);
/* Advance every member by n steps.  With use_graph != 0, even-length runs
 * of launches are captured once per membership change and replayed; on the
 * legacy default stream (NULL), which cannot be captured, every step is
 * launched directly.  Frozen-temperature members read their step from a
 * device counter that every launch advances, so replays keep the time.
 * n = 0, or a group without members, launches nothing and returns PF_OK;
 * n < 0 is PF_ERR_INVALID. */
int pf_group_step(pf_group* g, int64_t n, int use_graph);
int pf_group_size(const pf_group* g);

/* Temporal blocking of a group (explicit Euler, Sec. 3.3.1: step n+1 reads
 * only level n).  depth 1 (the default) launches every step over whole grids.
 * depth 2 advances two steps per wavefront over bands along the sweep axis
 * (2D: y, 3D: z), band_sweeps work-item sweeps high (per member:
 * band_sweeps x its sweep rows):
 *   step n+1 on band 0, step n+1 on band 1, step n+2 on band 0,
 *   step n+1 on band 2, step n+2 on band 1, ..., step n+2 on the last band
 * (pf_wavefront_order), all on the group's stream.  Step n+2 on band b reads
 * level n+1 on band b and two rows (planes) into its neighbours, which the
 * step n+1 launches before it have written and no later launch overwrites; it
 * writes level n+2 only into band b, which no later step n+1 launch reads,
 * since a band (at least one sweep of at least 8 rows) is higher than the
 * two-row psi halo.  The intermediate level is then read back while it is
 * still in L2.  Every cell gets the same arithmetic as at depth 1, so results
 * are bit-identical.  A group whose members include a frozen temperature (one
 * step clock per launch) or a two-kernel member (its U pass needs the psi
 * pass of the neighbouring bands) steps at depth 1; pf_group_get_depth
 * reports the depth in effect.  An odd step
 * count ends with one depth-1 step.  depth outside {1, 2} or band_sweeps < 1
 * is PF_ERR_INVALID; the setting holds across membership changes. */
int pf_group_set_depth(pf_group* g, int depth, int band_sweeps);
/* The setting, and the depth the current members step at (1 or 2). */
int pf_group_get_depth(pf_group* g, int* depth, int* band_sweeps, int* effective);
/* The launch order of one depth-2 wavefront over n_bands bands (host only,
 * no device work): entry i is (level[i], band[i]), level 0 = step n+1,
 * level 1 = step n+2.  Writes min(cap, 2 n_bands) entries and returns
 * 2 n_bands; n_bands < 1, cap < 0, or cap > 0 with a NULL array is
 * PF_ERR_INVALID. */
int pf_wavefront_order(int n_bands, int* level, int* band, int cap);
/* pf_observe of every member (in the order they were added, out[i] for the
 * i-th) with one synchronisation: the reductions of all members are queued on
 * the group's stream and their records read back together.  grain as in
 * pf_observe and valid for every member.  Returns PF_ERR_NONFINITE (with all
 * of out filled) when a member holds NaN/Inf cells.  A group without
 * members writes nothing and returns PF_OK. */
int pf_group_observe(pf_group* g, int grain, pf_obs* out);
int pf_group_destroy(pf_group* g);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
