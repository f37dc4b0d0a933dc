// pf_internal.cuh -- device-side records shared by the kernels and the C-ABI
// layer of the sm_103a phase-field library.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pf {

// Scheme identifiers (values of pf_scheme in include/pf.h).
enum : int { S10 = 0, S21 = 1, SBAR21 = 2, S100 = 3, SBAR120 = 4 };

// Derived per-instance constants (index into InstRec::cf / cd).
enum : int {
    C_IH = 0,    // 1/h
    C_I4H,       // 1/(4h)
    C_IH_HALF,   // 1/(2h)
    C_HH,        // h^2
    C_IH2,       // 1/h^2
    C_I6H2,      // 1/(6h^2)
    C_G10,       // (2/3)/(4h^2)
    C_G01,       // (1/3)/(8h^2)
    C_DT,        // dt
    C_K,         // k
    C_OMK,       // 1-k
    C_EPS,       // eps4
    C_LAM,       // lambda
    C_D,         // D
    C_ISQ2DT,    // 1/(sqrt2 dt)
    C_I4H2,      // 1/(4h^2)
    NC
};

// One simulation as the fused kernels see it.  psi/U hold the two time
// levels; the current level of an instance in a launch is
// parity_offset ^ launch_parity.
struct InstRec {
    void* psi[2];
    void* U[2];
    const int16_t* grain;  // per-cell grain index
    const void* rot;       // n_grains x 9, crystal -> lab, in the field precision
    void* rate;            // d psi/dt of the two-kernel form (nullptr when fused)
    int32_t nx, ny, nz, parity_offset;
    int32_t thermal;  // 1: frozen temperature along +y (2D)
    int32_t bcx;      // 1: periodic x (2D)
    int32_t tlevel;   // 1: T0 time level (pure forward Euler of Eq. PF_b)
    int32_t n_grains; // rows of the rotation table
    int32_t one_grain; // 1: every cell is in grain 0 (the grain map need not be read)
    int32_t pad_;
    double h, dt, k, eps4, lambda, D;
    // frozen temperature: zeta(row j, step n) = j zA - zB - n zC
    // (zA = h / lT, zB = yT / lT, zC = Vp dt / lT)
    double zA, zB, zC;
    // derived constants, filled on the host (no FP64 arithmetic in FP32 kernels)
    float cf[NC];
    double cd[NC];
};

// A unit of work: one block sweeps `ext` rows (2D) or planes (3D) starting
// at (x0, y0, z0) of instance `inst`.
struct WorkItem {
    int32_t inst, x0, y0, z0, ext, pad0, pad1, pad2;
};

// Guard on |grad psi|^2 h^2 below which the interface normal is undefined:
// a_s = 1, anisotropic flux 0, anti-trapping flux 0.
template <typename T> struct Guard;
template <> struct Guard<float> { static constexpr float v = 1e-12f; };
template <> struct Guard<double> { static constexpr double v = 1e-20; };

// Bounds-checked build (compile with -DPF_BOUNDS_CHECK): every global and
// shared-memory index the kernels form goes through PF_CHK(i, n).  An index
// outside [0, n) is counted, its source line kept (first one), and replaced
// by 0, so the access stays inside the array and nothing faults.  Each
// translation unit keeps its own record and exports a host reader; pf_debug_bounds() sums them.  The default build compiles the
// index unchanged.
#ifdef PF_BOUNDS_CHECK
static __device__ unsigned long long g_oob_count;
static __device__ int g_oob_line;
__device__ __forceinline__ long long pf_chk(long long i, long long n, int line) {
    if (i >= 0 && i < n) return i;
    atomicAdd(&g_oob_count, 1ull);
    atomicCAS(&g_oob_line, 0, line);
    return 0;
}
#define PF_CHK(i, n) ::pf::pf_chk((long long)(i), (long long)(n), __LINE__)
#define PF_BOUNDS_READER(name)                                                     \
    int name(unsigned long long* count, int* line) {                               \
        if (cudaMemcpyFromSymbol(count, g_oob_count, sizeof(*count)) != cudaSuccess) \
            return -1;                                                             \
        if (cudaMemcpyFromSymbol(line, g_oob_line, sizeof(*line)) != cudaSuccess)  \
            return -1;                                                             \
        return 0;                                                                  \
    }
#else
#define PF_CHK(i, n) (i)
#define PF_BOUNDS_READER(name) \
    int name(unsigned long long* count, int* line) { *count = 0; *line = 0; return 1; }
#endif
// host readers of the per-unit records (return 1 in an unchecked build)
int bounds_step2d(unsigned long long* count, int* line);
int bounds_step3d(unsigned long long* count, int* line);
int bounds_observe(unsigned long long* count, int* line);

// Cell-centred mirror of an index into [0, n): -1 -> 0, -2 -> 1, n -> n-1,
// n+1 -> n-2.  Values further out (never consumed) are clamped in range.
__device__ __forceinline__ int mirror_idx(int i, int n) {
    i = i < 0 ? -1 - i : i;
    i = i >= n ? 2 * n - 1 - i : i;
    i = i < 0 ? 0 : i;
    return i;
}

// Launchers (defined in step2d.cu / step3d.cu).  prec: 0 float, 1 double,
// 2 compensated float pairs (2D isothermal only; lo half right after the hi
// half of each level).
// Return false if (prec, scheme, block) has no compiled kernel.
// Step counter of the instances in a launch (only read for frozen-temperature
// instances): with clock == nullptr every instance is at step `step`;
// otherwise instance i is at step base[i] + *clock (groups: the clock is
// advanced on the device after every launch, so graph replays stay exact).
struct StepClock {
    const long long* clock;
    const long long* base;
    long long step;
};
// var: the 2D kernel variant: 0 isothermal, mirror walls, T1; 1 frozen
// temperature and/or periodic x (T1 or T0 read from the record); 2 isothermal,
// mirror walls, T0.  mode: 0 the fused step; 1, 2 the psi and U passes of the
// two-kernel form (T0 time level: variant 1 or 2, prec 0 or 1)
bool launch_step2d(int prec, int scheme, int bx, int grid, cudaStream_t st, const WorkItem* work, int n_work,
                   const InstRec* recs, int launch_parity, StepClock clk, int var, int mode = 0);
bool launch_step3d(int prec, int scheme, int bx, int by, int grid, cudaStream_t st, const WorkItem* work,
                   int n_work, const InstRec* recs, int launch_parity, StepClock clk);
// clock += 1 (one thread)
cudaError_t launch_tick(long long* clock, cudaStream_t st);
// Blocks of the fused kernel that fit on one SM (0 if not compiled); var as
// for launch_step2d
int occupancy_step2d(int prec, int scheme, int bx, int var, int mode = 0);
int occupancy_step3d(int prec, int scheme, int bx, int by);

// Observation / initialisation kernels (observe.cu).
struct ObsPartial {
    double solute, solid, score;
    long long tip_index;
    long long nonfinite;
    double tip[3];
    double pad;
};
struct ObsArgs {
    const void* psi;
    const void* U;
    const int16_t* grain;
    int prec, dim, nx, ny, nz, grain_filter;
    double h, k;
    double cg[3], d[3];
    int ea, es;
};
constexpr int OBS_BLOCKS = 304;  // 2 x 152 SMs
constexpr int OBS_THREADS = 256;
cudaError_t launch_observe(const ObsArgs& a, ObsPartial* partials, ObsPartial* result, cudaStream_t st);
// one observe job of a group: the arguments and the member's OBS_BLOCKS partials
struct ObsJob {
    ObsArgs a;
    ObsPartial* partials;
};
// the jobs (in device memory) of n members in one launch; results[m] for job m
cudaError_t launch_observe_multi(const ObsJob* jobs, int n, ObsPartial* results, cudaStream_t st);
// Device address of the library's fixed observe scratch on the current device.
cudaError_t noalloc_scratch(ObsPartial** partials, ObsPartial** result);

// Tip radius (Sec. 3.3.2, Sec. 6.2.2): contour lines and parabola fits on the
// device.  out[0..4] = rho, rho_x, rho_z, samples in the x fit, in the z fit;
// out[8..135] receive the contour crossings.
struct TipArgs {
    const void* psi;
    int prec, dim, nx, ny, nz;
    double h;
    double tip[3], axis[3];  // tip position and (unnormalised) growth axis
};
constexpr int TIP_THREADS = 128;  // 4 warps per block, one warp per contour line
cudaError_t launch_tip_radius(const TipArgs& a, double* out, cudaStream_t st);

struct SeedDev {
    double x, y, z, r;
    int32_t grain, pad;
};
cudaError_t launch_init_seeds(int prec, int dim, int nx, int ny, int nz, double h, double U0, const SeedDev* seeds,
                              int n_seeds, void* psi, void* U, int16_t* grain, cudaStream_t st);
cudaError_t launch_fill(int prec, void* p, double v, long long n, cudaStream_t st);
// compensated FP32 state: FP64 -> (hi, lo) and back
cudaError_t launch_split(const double* x, float* hi, float* lo, long long n, cudaStream_t st);
cudaError_t launch_join(const float* hi, const float* lo, double* x, long long n, cudaStream_t st);
// frame shift of one field toward -y (kind 0: float, 1: double, 2: int16 grain index); vacated
// rows, k beyond the last: mode 0 copy the last row, 1 continue it by a k, 3 a + (last - a) exp(-b k)
cudaError_t launch_shift_rows(int kind, const void* src, void* dst, int nx, int ny, int nz, int rows, int mode,
                              double a, double b, cudaStream_t st);

}  // namespace pf
