// observe.cu -- FP64 reductions (solute integral of Eq. Supersaturation,
// solid fraction, non-finite scan, tip tracking of Sec. 3.3.2 / 6.2.2) and
// the seed initialisation, for sm_103a.
//
// Reductions are deterministic: a fixed grid of OBS_BLOCKS blocks walks the
// cells grid-stride, each block reduces in a fixed tree order, and one block
// combines the partials in index order.  The tip candidate is chosen by the
// total order (larger projection, then smaller cell index), so it does not
// depend on the reduction order.  Candidate positions and projections are
// formed with explicitly rounded FP64 operations (no contraction) so that the
// choice is reproducible on any FP64 implementation of the same formula.
#include <cfloat>
#include <math_constants.h>

#include "pf_internal.cuh"

namespace pf {
namespace {

constexpr double SQ2 = 1.41421356237309504880;

__device__ __forceinline__ bool better(double s1, long long i1, double s2, long long i2) {
    // is (s1, i1) preferred over (s2, i2)?
    if (i2 < 0) return i1 >= 0;
    if (i1 < 0) return false;
    if (s1 > s2) return true;
    if (s1 < s2) return false;
    return i1 < i2;
}

__device__ __forceinline__ void combine(ObsPartial& a, const ObsPartial& b) {
    a.solute += b.solute;
    a.solid += b.solid;
    a.nonfinite += b.nonfinite;
    if (better(b.score, b.tip_index, a.score, a.tip_index)) {
        a.score = b.score;
        a.tip_index = b.tip_index;
        a.tip[0] = b.tip[0];
        a.tip[1] = b.tip[1];
        a.tip[2] = b.tip[2];
    }
}

// The partial of block `blk` of `nblk` walking the cells of one field pair;
// sh: OBS_THREADS records of shared memory.
template <typename T>
__device__ void observe_block(const ObsArgs& a, ObsPartial* __restrict__ partials, long long blk, long long nblk,
                              ObsPartial* sh) {
    const T* __restrict__ psi = static_cast<const T*>(a.psi);
    const T* __restrict__ U = static_cast<const T*>(a.U);
    const long long nx = a.nx, ny = a.ny, nz = a.dim == 3 ? a.nz : 1;
    const long long N = nx * ny * nz;
    ObsPartial acc;
    acc.solute = 0.0;
    acc.solid = 0.0;
    acc.nonfinite = 0;
    acc.score = -DBL_MAX;
    acc.tip_index = -1;
    acc.tip[0] = acc.tip[1] = acc.tip[2] = 0.0;
    acc.pad = 0.0;
    const double k = a.k, omk = 1.0 - a.k;
    // Away from the interface |psi| / sqrt2 >= 22.6 and tanh is +-1 to FP64
    // precision (both here and in C libraries that return +-1 from |x| = 22
    // on).  Those bulk cells contribute 1 + (1-k) U (liquid) or k (1 + (1-k) U)
    // (solid) to the solute sum and 0 or 1 to the solid sum: they are counted
    // and their U summed, and the terms formed once per thread.  Rows
    // are walked whole (one block per row, threads along x), so no cell index
    // is divided.  The bulk U is summed exactly in FP32 pairs (Knuth's
    // two-sum: hi + lo carries ~48 bits, more than the FP64 sum of these FP32
    // values keeps) rather than in FP64, whose conversions and adds run at
    // GB300's low FP64 rate; the non-finite test also runs in the field
    // precision.
    long long n_liq = 0, n_sol = 0;
    T sl_hi = T(0), sl_lo = T(0), ss_hi = T(0), ss_lo = T(0);
    auto acc2 = [](T& hi, T& lo, T v) {
        if constexpr (sizeof(T) == 4) {
            const T sm = hi + v, bb = sm - hi;
            lo += (hi - (sm - bb)) + (v - bb);
            hi = sm;
        } else {
            hi += v;  // FP64 fields: the plain FP64 sum
        }
    };
    const long long rows = ny * nz;
    // one cell: returns after the tip test (the bulk liquid returns early)
    auto cell = [&](long long i, long long j, long long kk, long long c, T pst, T ut) {
        if (!isfinite(pst) || !isfinite(ut)) {
            acc.nonfinite += 1;
            return;
        }
        if (fabs(pst) >= T(32)) {
            if (pst > T(0)) {
                n_sol += 1;
                acc2(ss_hi, ss_lo, ut);
            } else {
                n_liq += 1;
                acc2(sl_hi, sl_lo, ut);
                return;  // liquid: no tip candidate
            }
        } else {
            const double u = (double)ut;
            const double ph = tanh((double)pst / SQ2);
            acc.solute += (1.0 + k - omk * ph) * (1.0 + omk * u) / 2.0;
            acc.solid += (1.0 + ph) / 2.0;
        }
        if (a.grain_filter >= 0 && a.grain[c] != a.grain_filter) return;
        if (!(pst >= T(0))) return;
        long long ii = i, jj = j, kq = kk;
        if (a.ea == 0) ii += a.es;
        else if (a.ea == 1) jj += a.es;
        else kq += a.es;
        if (ii < 0 || jj < 0 || kq < 0 || ii >= nx || jj >= ny || kq >= nz) return;
        const T pnt = psi[PF_CHK((kq * ny + jj) * nx + ii, N)];
        if (!(pnt < T(0))) return;
        const double ps = (double)pst, pn = (double)pnt;
        const double frac = __ddiv_rn(ps, __dsub_rn(ps, pn));
        double p[3] = {__dmul_rn((double)i, a.h), __dmul_rn((double)j, a.h),
                       a.dim == 3 ? __dmul_rn((double)kk, a.h) : 0.0};
        p[a.ea] = __dadd_rn(p[a.ea], __dmul_rn((double)a.es * frac, a.h));
        double sc = 0.0;
        for (int q = 0; q < a.dim; ++q) sc = __dadd_rn(sc, __dmul_rn(__dsub_rn(p[q], a.cg[q]), a.d[q]));
        if (better(sc, c, acc.score, acc.tip_index)) {
            acc.score = sc;
            acc.tip_index = c;
            acc.tip[0] = p[0];
            acc.tip[1] = p[1];
            acc.tip[2] = p[2];
        }
    };
    // FP32 rows whose length is a multiple of 4 are read four cells at a time
    // (16-byte vector loads: more bytes in flight per thread); other rows cell
    // by cell.  The order of the per-thread sums differs between the two, not
    // the cells each block covers.
    const bool vec4 = sizeof(T) == 4 && (nx & 3) == 0 && ((uintptr_t)psi & 15) == 0 && ((uintptr_t)U & 15) == 0;
    for (long long row = blk; row < rows; row += nblk) {
        const long long j = row % ny, kk = row / ny;
        const long long base = row * nx;
        if (vec4) {
            for (long long i = 4 * (long long)threadIdx.x; i < nx; i += 4 * (long long)blockDim.x) {
                const float4 p4 = __ldg(reinterpret_cast<const float4*>(psi + PF_CHK(base + i, N)));
                const float4 u4 = __ldg(reinterpret_cast<const float4*>(U + PF_CHK(base + i, N)));
                cell(i, j, kk, base + i, (T)p4.x, (T)u4.x);
                cell(i + 1, j, kk, base + i + 1, (T)p4.y, (T)u4.y);
                cell(i + 2, j, kk, base + i + 2, (T)p4.z, (T)u4.z);
                cell(i + 3, j, kk, base + i + 3, (T)p4.w, (T)u4.w);
            }
        } else {
            for (long long i = threadIdx.x; i < nx; i += blockDim.x) cell(i, j, kk, base + i, psi[base + i], U[base + i]);
        }
    }
    const double u_liq = (double)sl_hi + (double)sl_lo, u_sol = (double)ss_hi + (double)ss_lo;
    acc.solute += ((double)n_liq + omk * u_liq) + k * ((double)n_sol + omk * u_sol);
    acc.solid += (double)n_sol;
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = OBS_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) combine(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blk] = sh[0];
}

template <typename T>
__global__ void __launch_bounds__(OBS_THREADS) k_observe(ObsArgs a, ObsPartial* __restrict__ partials) {
    __shared__ ObsPartial sh[OBS_THREADS];
    observe_block<T>(a, partials, blockIdx.x, gridDim.x, sh);
}

// All members of a group in one launch: blocks (x, m) walk member m's cells
// exactly as blocks x of k_observe would (same partials, same order).
__global__ void __launch_bounds__(OBS_THREADS) k_observe_multi(const ObsJob* __restrict__ jobs) {
    __shared__ ObsPartial sh[OBS_THREADS];
    const ObsJob& j = jobs[blockIdx.y];
    if (j.a.prec == 0)
        observe_block<float>(j.a, j.partials, blockIdx.x, gridDim.x, sh);
    else
        observe_block<double>(j.a, j.partials, blockIdx.x, gridDim.x, sh);
}

// Combine the block partials: thread t folds partials t, t + 256, ... in
// index order, then a fixed tree; deterministic for a fixed partial count.
__device__ void finish_block(const ObsPartial* __restrict__ partials, int n, ObsPartial* __restrict__ out,
                             ObsPartial* sh) {
    ObsPartial acc;
    acc.solute = 0.0;
    acc.solid = 0.0;
    acc.nonfinite = 0;
    acc.score = -DBL_MAX;
    acc.tip_index = -1;
    acc.tip[0] = acc.tip[1] = acc.tip[2] = 0.0;
    acc.pad = 0.0;
    for (int b = threadIdx.x; b < n; b += OBS_THREADS) combine(acc, partials[b]);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = OBS_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) combine(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

__global__ void __launch_bounds__(OBS_THREADS) k_observe_finish(const ObsPartial* __restrict__ partials, int n,
                                                                ObsPartial* __restrict__ out) {
    __shared__ ObsPartial sh[OBS_THREADS];
    finish_block(partials, n, out, sh);
}

// Block m combines member m's partials into out[m].
__global__ void __launch_bounds__(OBS_THREADS) k_observe_finish_multi(const ObsJob* __restrict__ jobs,
                                                                      ObsPartial* __restrict__ out) {
    __shared__ ObsPartial sh[OBS_THREADS];
    finish_block(jobs[blockIdx.x].partials, OBS_BLOCKS, out + blockIdx.x, sh);
}

// ---------------------------------------------------------------------------
// Tip radius (Sec. 3.3.2, Sec. 6.2.2): the paper fits the parabola
// y = y_tip - (x - x_tip)^2 / (2 rho) to the psi = 0 contour rotated so that
// the measured growth direction is vertical, up to one radius behind the tip
// (3D: rho_x in the plane of the growth axis and its in-plane normal, rho_z in
// the plane of the growth axis and z, 1/rho = (1/rho_x + 1/rho_z) / 2).
// Contour: 64 lines per transverse axis e, r(t) = (tip + s e) - t e_par with
// s = j h (j = -32..-1, 1..32) and t = m h / 4 (m <= 160); psi is interpolated
// multilinearly between cell centres and the first sample with psi >= 0 gives
// the crossing by linear interpolation.  Fit: c = sum t s^2 / sum s^4 over the
// crossings with t <= w, rho = 1 / (2c); w = 40 h, then the previous rho; four
// rounds.  One warp per line (its lanes take 32 samples at a time), then one
// thread per transverse axis fits in line order.  All FP64 operations are
// explicitly rounded (no contraction), so the crossings are reproducible.
constexpr int TIP_J = 32, TIP_M = 160, TIP_ROUNDS = 4;

template <typename T>
__device__ double tip_interp(const TipArgs& a, const T* __restrict__ psi, const double r[3], bool& inside) {
    const int n[3] = {a.nx, a.ny, a.dim == 3 ? a.nz : 1};
    int i0[3] = {0, 0, 0};
    double f[3] = {0.0, 0.0, 0.0};
    inside = true;
    for (int q = 0; q < a.dim; ++q) {
        const double u = __ddiv_rn(r[q], a.h);
        if (!(u >= 0.0) || u > (double)(n[q] - 1)) {
            inside = false;
            return 0.0;
        }
        int i = (int)floor(u);
        if (i > n[q] - 2) i = n[q] - 2;
        i0[q] = i;
        f[q] = __dsub_rn(u, (double)i);
    }
    auto P = [&](int di, int dj, int dk) -> double {
        return (double)psi[PF_CHK(((long long)(i0[2] + dk) * a.ny + (i0[1] + dj)) * a.nx + (i0[0] + di),
                                  (long long)a.nx * a.ny * (a.dim == 3 ? a.nz : 1))];
    };
    auto plane = [&](int dk) -> double {
        const double g0 = __dsub_rn(1.0, f[0]);
        const double lo = __dadd_rn(__dmul_rn(g0, P(0, 0, dk)), __dmul_rn(f[0], P(1, 0, dk)));
        const double hi = __dadd_rn(__dmul_rn(g0, P(0, 1, dk)), __dmul_rn(f[0], P(1, 1, dk)));
        return __dadd_rn(__dmul_rn(__dsub_rn(1.0, f[1]), lo), __dmul_rn(f[1], hi));
    };
    const double v0 = plane(0);
    if (a.dim == 2) return v0;
    return __dadd_rn(__dmul_rn(__dsub_rn(1.0, f[2]), v0), __dmul_rn(f[2], plane(1)));
}

// growth axis e_par and transverse axes e_x, e_z of the fit (explicitly rounded)
__device__ void tip_frame(const TipArgs& a, double frame[3][3]) {
    double ep[3] = {a.axis[0], a.axis[1], a.dim == 3 ? a.axis[2] : 0.0};
    const double na =
        __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ep[0], ep[0]), __dmul_rn(ep[1], ep[1])), __dmul_rn(ep[2], ep[2])));
    for (int q = 0; q < 3; ++q) ep[q] = __ddiv_rn(ep[q], na);
    double ex[3], ez[3] = {0.0, 0.0, 0.0};
    if (a.dim == 2) {
        ex[0] = ep[1];
        ex[1] = -ep[0];
        ex[2] = 0.0;
    } else {
        double ref[3] = {0.0, 0.0, 1.0};
        if (fabs(ep[2]) > 1.0 - 1e-6) {
            ref[0] = 1.0;
            ref[2] = 0.0;
        }
        const double pr =
            __dadd_rn(__dadd_rn(__dmul_rn(ref[0], ep[0]), __dmul_rn(ref[1], ep[1])), __dmul_rn(ref[2], ep[2]));
        for (int q = 0; q < 3; ++q) ez[q] = __dsub_rn(ref[q], __dmul_rn(pr, ep[q]));
        const double nz =
            __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ez[0], ez[0]), __dmul_rn(ez[1], ez[1])), __dmul_rn(ez[2], ez[2])));
        for (int q = 0; q < 3; ++q) ez[q] = __ddiv_rn(ez[q], nz);
        ex[0] = __dsub_rn(__dmul_rn(ez[1], ep[2]), __dmul_rn(ez[2], ep[1]));
        ex[1] = __dsub_rn(__dmul_rn(ez[2], ep[0]), __dmul_rn(ez[0], ep[2]));
        ex[2] = __dsub_rn(__dmul_rn(ez[0], ep[1]), __dmul_rn(ez[1], ep[0]));
    }
    for (int q = 0; q < 3; ++q) {
        frame[0][q] = ep[q];
        frame[1][q] = ex[q];
        frame[2][q] = ez[q];
    }
}

// One warp per contour line (64 per transverse axis); the lanes evaluate 32
// consecutive samples at once and the first sample that is outside the grid
// or has psi >= 0 ends the line, as in a sequential march.  t[line] = the
// crossing or NaN.
template <typename T> __global__ void __launch_bounds__(TIP_THREADS) k_tip_lines(TipArgs a, double* __restrict__ t) {
    __shared__ double frame[3][3];
    if (threadIdx.x == 0) tip_frame(a, frame);
    __syncthreads();
    const T* __restrict__ psi = static_cast<const T*>(a.psi);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (TIP_THREADS / 32) + (threadIdx.x >> 5);
    const int half = gw / (2 * TIP_J), l = gw % (2 * TIP_J);  // half 0: e_x lines, 1: e_z lines
    if (half >= (a.dim == 3 ? 2 : 1)) return;                 // whole warps only
    const double* e = frame[1 + half];
    const int j = l < TIP_J ? l - TIP_J : l - TIP_J + 1;
    const double s = __dmul_rn((double)j, a.h);
    const double dt = __dmul_rn(a.h, 0.25);
    double base[3];
    for (int q = 0; q < 3; ++q) base[q] = __dadd_rn(a.tip[q], __dmul_rn(s, e[q]));
    double tc = CUDART_NAN, carry = 0.0;
    for (int m0 = 0; m0 <= TIP_M; m0 += 32) {
        const int m = m0 + lane;
        double v = 0.0;
        bool inside = false;
        if (m <= TIP_M) {
            const double tm = __dmul_rn((double)m, dt);
            double r[3];
            for (int q = 0; q < 3; ++q) r[q] = __dsub_rn(base[q], __dmul_rn(tm, frame[0][q]));
            v = tip_interp<T>(a, psi, r, inside);
        }
        const bool ev = m <= TIP_M && (!inside || v >= 0.0);
        const unsigned b = __ballot_sync(FULL, ev);
        const double vup = __shfl_up_sync(FULL, v, 1);
        const double prev = lane == 0 ? carry : vup;  // psi at sample m - 1
        if (b) {
            const int f = __ffs(b) - 1;
            double tl = CUDART_NAN;
            if (lane == f && inside && v >= 0.0 && m >= 1)
                tl = __dadd_rn(__dmul_rn((double)(m - 1), dt), __dmul_rn(dt, __ddiv_rn(prev, __dsub_rn(prev, v))));
            tc = __shfl_sync(FULL, tl, f);
            break;
        }
        carry = __shfl_sync(FULL, v, 31);
    }
    if (lane == 0) t[half * 2 * TIP_J + l] = tc;
}

// Parabola fits of the crossings in line order (one thread per transverse
// axis), then rho (3D: 2 / (1/rho_x + 1/rho_z)).
__global__ void k_tip_fit(TipArgs a, const double* __restrict__ t, double* __restrict__ out) {
    const int half = threadIdx.x;
    const double dt = __dmul_rn(a.h, 0.25);
    if (half < (a.dim == 3 ? 2 : 1)) {
        double w = __dmul_rn((double)TIP_M, dt), rho = CUDART_NAN;
        int used = 0;
        for (int round = 0; round < TIP_ROUNDS; ++round) {
            double st = 0.0, s4 = 0.0;
            int n = 0;
            for (int k = 0; k < 2 * TIP_J; ++k) {
                const int j = k < TIP_J ? k - TIP_J : k - TIP_J + 1;
                const double s = __dmul_rn((double)j, a.h);
                const double tk = t[half * 2 * TIP_J + k];
                if (!(tk <= w)) continue;
                const double s2 = __dmul_rn(s, s);
                st = __dadd_rn(st, __dmul_rn(tk, s2));
                s4 = __dadd_rn(s4, __dmul_rn(s2, s2));
                ++n;
            }
            used = n;
            if (n == 0 || !(st > 0.0)) {
                rho = CUDART_NAN;
                break;
            }
            rho = __dmul_rn(0.5, __ddiv_rn(s4, st));
            w = rho;
        }
        out[1 + half] = rho;
        out[3 + half] = (double)used;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (a.dim == 2) {
            out[2] = CUDART_NAN;
            out[4] = 0.0;
            out[0] = out[1];
        } else {
            out[0] = __ddiv_rn(2.0, __dadd_rn(__ddiv_rn(1.0, out[1]), __ddiv_rn(1.0, out[2])));
        }
    }
}

template <typename T>
__global__ void k_init_seeds(int dim, int nx, int ny, int nz, double h, double U0, const SeedDev* __restrict__ seeds,
                             int n_seeds, T* __restrict__ psi, T* __restrict__ U, int16_t* __restrict__ grain) {
    const long long N = (long long)nx * ny * (dim == 3 ? nz : 1);
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const long long i = c % nx, j = (c / nx) % ny, k = c / ((long long)nx * ny);
        const double x = __dmul_rn((double)i, h), y = __dmul_rn((double)j, h);
        const double z = dim == 3 ? __dmul_rn((double)k, h) : 0.0;
        double best = -DBL_MAX;
        int bs = 0;
        bool any = false;
        for (int s = 0; s < n_seeds; ++s) {
            const double dx = __dsub_rn(x, seeds[s].x), dy = __dsub_rn(y, seeds[s].y);
            const double dz = dim == 3 ? __dsub_rn(z, seeds[s].z) : 0.0;
            const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            const double v = __dsub_rn(seeds[s].r, __dsqrt_rn(d2));
            if (!any || v > best) {
                best = v;
                bs = s;
                any = true;
            }
        }
        psi[c] = (T)best;
        U[c] = (T)U0;
        grain[c] = (int16_t)seeds[bs].grain;
    }
}

// advances the step clock of a group (one thread, after every step launch)
__global__ void k_tick(long long* clock) { *clock += 1; }

template <typename T> __global__ void k_fill(T* __restrict__ p, T v, long long n) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        p[c] = v;
}

// Compensated FP32 state (precision PF_F32C): split an FP64 field into hi =
// fl32(x) and lo = fl32(x - hi) (x - hi is exact in FP64), or join hi + lo
// back into FP64 (exact).
__global__ void k_split(const double* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo, long long n) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double v = x[c];
        const float h = __double2float_rn(v);
        hi[c] = h;
        lo[c] = __double2float_rn(v - (double)h);
    }
}
__global__ void k_join(const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ x, long long n) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        x[c] = (double)hi[c] + (double)lo[c];
}

// Frame shift by `rows` cells toward -y: dst(x, y, z) = src(x, y + rows, z)
// for y + rows < ny.  The vacated top rows, k rows beyond the last one, take
// (mode 0) the last row's value, (mode 1) the last row's value plus a k (psi:
// a = -h, a signed distance continued into the melt) or (mode 3) the value
// a + (last - a) exp(-b k) (U: the steady far field a + C exp(-Vp y / D) ahead
// of a front pulled at Vp, b = Vp h / D).  src and dst do not overlap.
template <typename T>
__global__ void k_shift_rows(const T* __restrict__ src, T* __restrict__ dst, int nx, int ny, int nz, int rows, int mode,
                             double a, double b) {
    const long long n = (long long)nx * ny * nz;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx);
        const long long yz = c / nx;
        const int y = (int)(yz % ny), z = (int)(yz / ny);
        const int ys = y + rows;
        const long long plane = (long long)z * ny;
        if (ys < ny) {
            dst[c] = src[(plane + ys) * nx + x];
        } else {
            const T top = src[(plane + ny - 1) * nx + x];
            // product and sum rounded separately (no contraction): top - k h exactly as written
            const double kk = (double)(ys - (ny - 1));
            dst[c] = mode == 0   ? top
                     : mode == 1 ? (T)__dadd_rn((double)top, __dmul_rn(a, kk))
                                 : (T)(a + ((double)top - a) * exp(-b * kk));
        }
    }
}

}  // namespace

// Fixed scratch for pf_observe_fields_noalloc: OBS_BLOCKS block partials and
// one result record (22 KB).  It lives in the module's global memory on every
// device that loads the library, for the life of the process.  Every call of
// that entry point overwrites all of it, so nothing needs clearing; calls whose
// kernels overlap on a device race on it.
static __device__ __align__(256) ObsPartial g_noalloc_scratch[OBS_BLOCKS + 1];

// Device address of the scratch on the current device, looked up on every
// call with cudaGetSymbolAddress (a host-side name of a __device__ array is
// not a device address).  Nothing is cached, so the address stays right after
// the device's context has been torn down and made again (cudaDeviceReset):
// the module is then loaded anew, possibly at another address.
cudaError_t noalloc_scratch(ObsPartial** partials, ObsPartial** result) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *partials = static_cast<ObsPartial*>(p);
    *result = *partials + OBS_BLOCKS;
    return cudaSuccess;
}

cudaError_t launch_observe_multi(const ObsJob* jobs, int n, ObsPartial* results, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_observe_multi<<<dim3(OBS_BLOCKS, n), OBS_THREADS, 0, st>>>(jobs);
    k_observe_finish_multi<<<n, OBS_THREADS, 0, st>>>(jobs, results);
    return cudaGetLastError();
}

cudaError_t launch_observe(const ObsArgs& a, ObsPartial* partials, ObsPartial* result, cudaStream_t st) {
    if (a.prec == 0)
        k_observe<float><<<OBS_BLOCKS, OBS_THREADS, 0, st>>>(a, partials);
    else
        k_observe<double><<<OBS_BLOCKS, OBS_THREADS, 0, st>>>(a, partials);
    k_observe_finish<<<1, OBS_THREADS, 0, st>>>(partials, OBS_BLOCKS, result);
    return cudaGetLastError();
}

PF_BOUNDS_READER(bounds_observe)

cudaError_t launch_tip_radius(const TipArgs& a, double* out, cudaStream_t st) {
    double* t = out + 8;  // 2 x 64 crossings after the five results
    const int blocks = (a.dim == 3 ? 2 : 1) * 2 * TIP_J / (TIP_THREADS / 32);
    if (a.prec == 0)
        k_tip_lines<float><<<blocks, TIP_THREADS, 0, st>>>(a, t);
    else
        k_tip_lines<double><<<blocks, TIP_THREADS, 0, st>>>(a, t);
    k_tip_fit<<<1, 32, 0, st>>>(a, t, out);
    return cudaGetLastError();
}

cudaError_t launch_tick(long long* clock, cudaStream_t st) {
    k_tick<<<1, 1, 0, st>>>(clock);
    return cudaGetLastError();
}

cudaError_t launch_init_seeds(int prec, int dim, int nx, int ny, int nz, double h, double U0, const SeedDev* seeds,
                              int n_seeds, void* psi, void* U, int16_t* grain, cudaStream_t st) {
    const int grid = 4 * 152, block = 256;
    if (prec == 0)
        k_init_seeds<float><<<grid, block, 0, st>>>(dim, nx, ny, nz, h, U0, seeds, n_seeds, static_cast<float*>(psi),
                                                    static_cast<float*>(U), grain);
    else
        k_init_seeds<double><<<grid, block, 0, st>>>(dim, nx, ny, nz, h, U0, seeds, n_seeds,
                                                     static_cast<double*>(psi), static_cast<double*>(U), grain);
    return cudaGetLastError();
}

cudaError_t launch_shift_rows(int kind, const void* src, void* dst, int nx, int ny, int nz, int rows, int mode,
                              double a, double b, cudaStream_t st) {
    const int grid = 4 * 152, block = 256;
    if (kind == 0)
        k_shift_rows<float><<<grid, block, 0, st>>>(static_cast<const float*>(src), static_cast<float*>(dst), nx, ny, nz,
                                                    rows, mode, a, b);
    else if (kind == 1)
        k_shift_rows<double><<<grid, block, 0, st>>>(static_cast<const double*>(src), static_cast<double*>(dst), nx, ny,
                                                     nz, rows, mode, a, b);
    else
        k_shift_rows<int16_t><<<grid, block, 0, st>>>(static_cast<const int16_t*>(src), static_cast<int16_t*>(dst), nx,
                                                      ny, nz, rows, 0, 0.0, 0.0);
    return cudaGetLastError();
}

cudaError_t launch_split(const double* x, float* hi, float* lo, long long n, cudaStream_t st) {
    const int block = 256;
    const int grid = 4 * 152;
    k_split<<<grid, block, 0, st>>>(x, hi, lo, n);
    return cudaGetLastError();
}

cudaError_t launch_join(const float* hi, const float* lo, double* x, long long n, cudaStream_t st) {
    const int block = 256;
    const int grid = 4 * 152;
    k_join<<<grid, block, 0, st>>>(hi, lo, x, n);
    return cudaGetLastError();
}

cudaError_t launch_fill(int prec, void* p, double v, long long n, cudaStream_t st) {
    const int grid = 4 * 152, block = 256;
    if (prec == 0)
        k_fill<float><<<grid, block, 0, st>>>(static_cast<float*>(p), (float)v, n);
    else
        k_fill<double><<<grid, block, 0, st>>>(static_cast<double*>(p), v, n);
    return cudaGetLastError();
}

}  // namespace pf
