// step2d.cu -- fused explicit time step of the quantitative alloy phase-field
// model in 2D for sm_103a (arXiv:2110.12448, Eqs. PF_a and PF_b).
//
// Warp-per-strip design.  Each warp owns a strip of 60 output columns and
// sweeps it row by row; lane t holds the two columns L = x0-2+2t, R = L+1
// (lanes 0 and 31 carry the halo).  Nothing is shared between warps: there is
// no shared memory and no block barrier.  Neighbour columns come over warp
// shuffles, rows live in a register ring, and every face flux is computed
// once and handed to the other cell that uses it (shuffle across columns,
// register carry across rows).  Global traffic per step: psi, U and the
// int16 grain read once, psi' and U' written once (float2 / int32 vectors).
//
// Iteration r of a sweep (rows are virtual: mirrored at the walls):
//   load psi(r+2), U(r+1), grain(r+1)            (prefetched one row ahead)
//   phase 1 at row r+1: d psi/dt of Eq. PF_a, psi' = psi + dt d psi/dt,
//     phi' and delta phi = phi' - phi (also on the ring columns x0-1, x0+60)
//   phase 2 at row r: U' of Eq. PF_b in conservative form
//
// Discretisations (h = lattice spacing):
//   L_{2,1} (Eq. 2D_L21) or L_{1,0} (Eq. 2D_L10);
//   G_{2,1} = 2/3 G_{1,0} + 1/3 G_{0,1} (App. A, Eqs. Grad_10, Grad_11) or G_{1,0};
//   O(eps4) terms: div(J - grad psi) over the four <10> faces, J from the face
//     gradient (two-point normal, four-point tangential difference) in the
//     crystal frame of the cell whose rate is computed; a_s^2 on the left-hand
//     side and in the G term from the centred gradient;
//   D = D~_{2,1}[1 - phi, U] (Eqs. divergence_10/_11, flux_10/_11), or the <10>
//     form with a two-point face mean for S_{1,0};
//   anti-trapping: D~_{2,1}[(1+(1-k)U) dphi/(sqrt2 dt), psi] (Eq. Anti_approx),
//     App. B's A_{2,1} (fluxes divided by the 21-point |grad psi| at the flux
//     point), or the <10> form normalised by the face gradient (S_{1,0});
//   U' = U + [dt (D D + A) + (1+(1-k)U) dphi] / (1+k-(1-k)phi'), D on phi^n,
//     U^n and the anti-trapping on psi^n: the solute integral is conserved
//     exactly with mirror walls.
// Walls: cell-centred mirrors.  Phase-1 results on ghost columns/rows are
// copied from their mirror cells, so the (not mirror-symmetric) anisotropic
// terms of a rotated crystal are never evaluated at a ghost position.
#include "pf_internal.cuh"

namespace pf {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARP_COLS = 64;  // columns held by a warp (60 outputs + 4 halo)

template <typename T> struct M;
template <> struct M<float> {
    // tanh x = 1 - 2 / (1 + e^{2x}) with the hardware exponential and
    // reciprocal: absolute error ~2e-7 over the whole range
    static __device__ __forceinline__ float tanh_(float x) {
        return 1.0f - __fdividef(2.0f, 1.0f + __expf(2.0f * x));
    }
    static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
};
template <> struct M<double> {
    static __device__ __forceinline__ double tanh_(double x) { return tanh(x); }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
};

template <typename T> __device__ __forceinline__ T shup(T v) { return __shfl_up_sync(FULL, v, 1); }
template <typename T> __device__ __forceinline__ T shdn(T v) { return __shfl_down_sync(FULL, v, 1); }

// A row as one lane sees it: columns L-2 .. L+3.
template <typename T> struct Row {
    T m2, m1, l, r, p1, p2;
    __device__ __forceinline__ T at(int o) const {
        return o == -2 ? m2 : o == -1 ? m1 : o == 0 ? l : o == 1 ? r : o == 2 ? p1 : p2;
    }
};

// Crystal frame of one grain (upper 2x2 of the crystal -> lab rotation).
template <typename T> struct Rot {
    T a, b, c, d;  // R00, R01, R10, R11
};

// Normal component of (J - g) for a lab-frame face gradient (gx, gy).
//   crystal components c = R^T g, r2 = |c|^2, s_p = c_p^2 / r2, q = sum s_p^2,
//   a_s = 1 - 3 eps + 4 eps q (= 1 + eps cos 4 theta, Eq. anis_function),
//   J'_p - c_p = c_p (a^2 - 1 - 16 eps a q + 16 eps a s_p)
// i.e. d(a_s^2 |g|^2 / 2)/dg - g, rotated back to the lab frame.
template <typename T>
__device__ __forceinline__ T aniso_qn(T gx, T gy, const Rot<T>& R, T eps, T hh, bool xface) {
    const T cx = R.a * gx + R.c * gy;
    const T cy = R.b * gx + R.d * gy;
    const T r2 = cx * cx + cy * cy;
    if (r2 * hh < Guard<T>::v) return T(0);
    const T inv = M<T>::rcp(r2);
    const T sx = cx * cx * inv, sy = cy * cy * inv;
    const T q = sx * sx + sy * sy;
    const T a = T(1) - T(3) * eps + T(4) * eps * q;
    const T c1 = T(16) * eps * a;
    const T c0 = a * a - T(1) - c1 * q;
    const T jx = cx * (c0 + c1 * sx), jy = cy * (c0 + c1 * sy);
    return xface ? (R.a * jx + R.b * jy) : (R.c * jx + R.d * jy);
}

template <typename T> __device__ __forceinline__ T aniso_a(T gx, T gy, const Rot<T>& R, T eps, T hh) {
    const T cx = R.a * gx + R.c * gy;
    const T cy = R.b * gx + R.d * gy;
    const T r2 = cx * cx + cy * cy;
    if (r2 * hh < Guard<T>::v) return T(1);
    const T inv = M<T>::rcp(r2);
    const T sx = cx * cx * inv, sy = cy * cy * inv;
    return T(1) - T(3) * eps + T(4) * eps * (sx * sx + sy * sy);
}

// App. B: |grad b| at a <10> face; B(p, q) = b at origin + p normal + q tangent.
template <typename T, typename F> __device__ __forceinline__ T appb_face(F B, T ih) {
    const T a1 = B(1, 1) - B(0, -1), a2 = B(0, 1) - B(1, -1);
    const T b1 = B(2, 1) - B(-1, -1), b2 = B(-1, 1) - B(2, -1);
    const T c1 = B(1, 2) - B(0, -2), c2 = B(0, 2) - B(1, -2);
    const T dn = (T(35.0 / 48.0) * (a1 - a2) - T(1.0 / 48.0) * (b1 - b2) - T(1.0 / 6.0) * (c1 - c2)) * ih;
    const T dt = (T(35.0 / 96.0) * (a1 + a2) - T(1.0 / 32.0) * (b1 + b2) - T(1.0 / 24.0) * (c1 + c2)) * ih;
    return M<T>::sqrt_(dn * dn + dt * dt);
}
// App. B: |grad b| at a corner; B(p, q) = b at origin + p x + q y.
template <typename T, typename F> __device__ __forceinline__ T appb_corner(F B, T ih) {
    const T a1 = B(1, 1) - B(0, 0), a2 = B(0, 1) - B(1, 0);
    const T b1 = B(2, 1) - B(-1, 0), b2 = B(-1, 1) - B(2, 0);
    const T c1 = B(1, 2) - B(0, -1), c2 = B(0, 2) - B(1, -1);
    const T dx = (T(5.0 / 8.0) * (a1 - a2) - T(1.0 / 48.0) * (b1 - b2) - T(1.0 / 16.0) * (c1 - c2)) * ih;
    const T dy = (T(5.0 / 8.0) * (a1 + a2) - T(1.0 / 16.0) * (b1 + b2) - T(1.0 / 48.0) * (c1 + c2)) * ih;
    return M<T>::sqrt_(dx * dx + dy * dy);
}

// f / m with the guard on |grad psi| of the standard anti-trapping forms
template <typename T> __device__ __forceinline__ T guarded_div(T f, T m, T hh) {
    return (m * m * hh < Guard<T>::v) ? T(0) : f * M<T>::rcp(m);
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using t = float2; };
template <> struct Vec2<double> { using t = double2; };

// Load the pair (c, c+1) of a row; c is even.  Vector load when both columns
// are inside and the row is 2-element aligned, mirrored scalar loads otherwise.
template <typename T>
__device__ __forceinline__ void load_pair(const T* __restrict__ row, int c, int nx, bool vec, T& a, T& b) {
    if (vec && c >= 0 && c + 1 < nx) {
        const typename Vec2<T>::t v = __ldg(reinterpret_cast<const typename Vec2<T>::t*>(row + c));
        a = v.x;
        b = v.y;
    } else {
        a = __ldg(row + mirror_idx(c, nx));
        b = __ldg(row + mirror_idx(c + 1, nx));
    }
}
__device__ __forceinline__ void load_grain_pair(const int16_t* __restrict__ row, int c, int nx, bool vec, int& a,
                                                int& b) {
    if (vec && c >= 0 && c + 1 < nx) {
        const int v = __ldg(reinterpret_cast<const int*>(row + c));
        a = (int)(int16_t)(v & 0xffff);
        b = (int)(int16_t)((unsigned)v >> 16);
    } else {
        a = __ldg(row + mirror_idx(c, nx));
        b = __ldg(row + mirror_idx(c + 1, nx));
    }
}
template <typename T>
__device__ __forceinline__ void store_pair(T* __restrict__ row, int c, bool vec, bool okL, bool okR, T a, T b) {
    if (vec && okL && okR) {
        typename Vec2<T>::t v;
        v.x = a;
        v.y = b;
        *reinterpret_cast<typename Vec2<T>::t*>(row + c) = v;
    } else {
        if (okL) row[c] = a;
        if (okR) row[c + 1] = b;
    }
}

// FP32 kernels are capped at 128 registers (4 blocks of 4 warps per SM): the
// sweep is latency-bound at 3 blocks.  FP64 kernels keep their registers.
#ifndef PF_STEP2D_MIN_BLOCKS_F32
#define PF_STEP2D_MIN_BLOCKS_F32 4
#endif

template <typename T, int S>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? PF_STEP2D_MIN_BLOCKS_F32 : 1) k_step2d(const WorkItem* __restrict__ work, int n_work,
                                                const InstRec* __restrict__ recs, int launch_parity) {
    constexpr bool ISO = (S == S21 || S == SBAR21);
    const int lane = threadIdx.x & 31;
    const int warps_per_block = blockDim.x >> 5;
    const int gw = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
    const int nw = gridDim.x * warps_per_block;
    const T SQ2 = T(1.41421356237309504880);
    const T ISQ2 = T(0.70710678118654752440);

    for (int w = gw; w < n_work; w += nw) {
        const WorkItem wi = work[w];
        const InstRec& rec = recs[wi.inst];
        const int nx = rec.nx, ny = rec.ny;
        const int par = rec.parity_offset ^ launch_parity;
        const T* __restrict__ psi = static_cast<const T*>(rec.psi[par]);
        const T* __restrict__ Uf = static_cast<const T*>(rec.U[par]);
        T* __restrict__ psi_o = static_cast<T*>(rec.psi[par ^ 1]);
        T* __restrict__ U_o = static_cast<T*>(rec.U[par ^ 1]);
        const int16_t* __restrict__ grain = rec.grain;
        const T* __restrict__ rot = static_cast<const T*>(rec.rot);
        const T ih = T(1.0 / rec.h), hh = T(rec.h * rec.h), dt = T(rec.dt);
        const T i4h = T(0.25 / rec.h);
        const T kk = T(rec.k), omk = T(1.0 - rec.k), eps = T(rec.eps4), lam = T(rec.lambda), Dc = T(rec.D);
        const T ih2 = T(1.0 / (rec.h * rec.h));
        const T i6h2 = T(1.0 / (6.0 * rec.h * rec.h));
        const T i4h2 = T(1.0 / (4.0 * rec.h * rec.h)), i8h2 = T(1.0 / (8.0 * rec.h * rec.h));
        const T isq2dt = T(1.0 / (1.41421356237309504880 * rec.dt));
        const bool vec = (nx & 1) == 0;

        const int x0 = wi.x0, y0 = wi.y0;
        const int y1 = min(y0 + wi.ext, ny);
        const int cL = x0 - 2 + 2 * lane;
        const bool realL = cL >= 0 && cL < nx, realR = cL + 1 >= 0 && cL + 1 < nx;
        const bool outL = lane >= 1 && lane <= 30 && realL;
        const bool outR = lane >= 1 && lane <= 30 && realR;
        // lanes holding the mirror images of ghost columns (phase-1 copies)
        const int mL = mirror_idx(cL, nx), mR = mirror_idx(cL + 1, nx);
        const int srcL = (mL - (x0 - 2)) >> 1, srcR = (mR - (x0 - 2)) >> 1;
        const bool hiL = ((mL - (x0 - 2)) & 1) != 0, hiR = ((mR - (x0 - 2)) & 1) != 0;

        auto fetch_row = [&](const T* f, int vr, T& a, T& b) {
            load_pair<T>(f + (size_t)mirror_idx(vr, ny) * nx, cL, nx, vec, a, b);
        };
        auto make_row = [&](T a, T b) {
            Row<T> row;
            row.l = a;
            row.r = b;
            row.m1 = shup(b);
            row.p1 = shdn(a);
            row.m2 = shup(a);
            row.p2 = shdn(b);
            return row;
        };
        auto rot_of = [&](int g) {
            const T* Rg = rot + 9 * g;
            Rot<T> R;
            R.a = __ldg(Rg + 0);
            R.b = __ldg(Rg + 1);
            R.c = __ldg(Rg + 3);
            R.d = __ldg(Rg + 4);
            return R;
        };
        auto phi_row = [&](const Row<T>& p) {
            Row<T> o;
            o.l = M<T>::tanh_(p.l * ISQ2);
            o.r = M<T>::tanh_(p.r * ISQ2);
            o.m1 = shup(o.r);
            o.p1 = shdn(o.l);
            o.m2 = o.p2 = T(0);
            return o;
        };
        // delta phi row from the own values: ghost columns take their mirror
        // cell's value, halo columns come from the neighbour lanes
        auto dphi_row = [&](T dL, T dR) {
            const T aL = __shfl_sync(FULL, dL, srcL), bL = __shfl_sync(FULL, dR, srcL);
            const T aR = __shfl_sync(FULL, dL, srcR), bR = __shfl_sync(FULL, dR, srcR);
            Row<T> o;
            o.l = realL ? dL : (hiL ? bL : aL);
            o.r = realR ? dR : (hiR ? bR : aR);
            o.m1 = shup(o.r);
            o.p1 = shdn(o.l);
            o.m2 = o.p2 = T(0);
            return o;
        };

        // anisotropy y-face carries (face between rows p-1 and p, own columns)
        T qyL_c = T(0), qyR_c = T(0);
        int gyL_c = -1, gyR_c = -1;
        int prow_c = -100;  // row p the carried faces belong to

        // phase 1 at real row p (psi rows Pm = p-1, P0 = p, Pp = p+1), grains
        // gL, gR: psi', phi' and delta phi for the own columns.
        auto phase1 = [&](int p, const Row<T>& Pm, const Row<T>& P0, const Row<T>& Pp, const Row<T>& ph0,
                          const Row<T>& u0, int gL, int gR, T& psinL, T& psinR, T& fL, T& fR, T& dL, T& dR) {
            const Rot<T> RL = rot_of(gL), RR = rot_of(gR);
            const int gM = shup(gR);  // grain of column L-1
            // x faces: (L|R) in L's frame, (R|R+1) in R's frame; (L-1|L) from lane-1
            const T gxi = (P0.r - P0.l) * ih, gyi = (Pp.r + Pp.l - Pm.r - Pm.l) * i4h;
            const T qx_lr_L = aniso_qn<T>(gxi, gyi, RL, eps, hh, true);
            const T qx_rp =
                aniso_qn<T>((P0.p1 - P0.r) * ih, (Pp.p1 + Pp.r - Pm.p1 - Pm.r) * i4h, RR, eps, hh, true);
            T qx_lr_R = qx_lr_L;
            if (gR != gL) qx_lr_R = aniso_qn<T>(gxi, gyi, RR, eps, hh, true);
            T qx_ml = shup(qx_rp);
            if (gM != gL || lane == 0)
                qx_ml = aniso_qn<T>((P0.l - P0.m1) * ih, (Pp.l + Pp.m1 - Pm.l - Pm.m1) * i4h, RL, eps, hh, true);
            // y faces: (p|p+1) computed here, (p-1|p) carried from row p-1
            const T qyL_p =
                aniso_qn<T>((Pp.r + P0.r - Pp.m1 - P0.m1) * i4h, (Pp.l - P0.l) * ih, RL, eps, hh, false);
            const T qyR_p =
                aniso_qn<T>((Pp.p1 + P0.p1 - Pp.l - P0.l) * i4h, (Pp.r - P0.r) * ih, RR, eps, hh, false);
            T qyL_m = qyL_c, qyR_m = qyR_c;
            if (prow_c != p || gyL_c != gL)
                qyL_m = aniso_qn<T>((P0.r + Pm.r - P0.m1 - Pm.m1) * i4h, (P0.l - Pm.l) * ih, RL, eps, hh, false);
            if (prow_c != p || gyR_c != gR)
                qyR_m = aniso_qn<T>((P0.p1 + Pm.p1 - P0.l - Pm.l) * i4h, (P0.r - Pm.r) * ih, RR, eps, hh, false);
            qyL_c = qyL_p;
            qyR_c = qyR_p;
            gyL_c = gL;
            gyR_c = gR;
            prow_c = p + 1;
            const T NL = (qx_lr_L - qx_ml + qyL_p - qyL_m) * ih;
            const T NR = (qx_rp - qx_lr_R + qyR_p - qyR_m) * ih;
            T LL, LR, GL, GR;
            if (ISO) {
                LL = (T(4) * (P0.m1 + P0.r + Pm.l + Pp.l) + (Pm.m1 + Pm.r + Pp.m1 + Pp.r) - T(20) * P0.l) * i6h2;
                LR = (T(4) * (P0.l + P0.p1 + Pm.r + Pp.r) + (Pm.l + Pm.p1 + Pp.l + Pp.p1) - T(20) * P0.r) * i6h2;
                const T exL = P0.r - P0.m1, eyL = Pp.l - Pm.l, dpL = Pp.r - Pm.m1, dmL = Pm.r - Pp.m1;
                const T exR = P0.p1 - P0.l, eyR = Pp.r - Pm.r, dpR = Pp.p1 - Pm.l, dmR = Pm.p1 - Pp.l;
                GL = T(2.0 / 3.0) * (exL * exL + eyL * eyL) * i4h2 + T(1.0 / 3.0) * (dpL * dpL + dmL * dmL) * i8h2;
                GR = T(2.0 / 3.0) * (exR * exR + eyR * eyR) * i4h2 + T(1.0 / 3.0) * (dpR * dpR + dmR * dmR) * i8h2;
            } else {
                LL = (P0.m1 + P0.r + Pm.l + Pp.l - T(4) * P0.l) * ih2;
                LR = (P0.l + P0.p1 + Pm.r + Pp.r - T(4) * P0.r) * ih2;
                const T exL = P0.r - P0.m1, eyL = Pp.l - Pm.l, exR = P0.p1 - P0.l, eyR = Pp.r - Pm.r;
                GL = (exL * exL + eyL * eyL) * i4h2;
                GR = (exR * exR + eyR * eyR) * i4h2;
            }
            const T acL = aniso_a<T>((P0.r - P0.m1) * T(0.5) * ih, (Pp.l - Pm.l) * T(0.5) * ih, RL, eps, hh);
            const T acR = aniso_a<T>((P0.p1 - P0.l) * T(0.5) * ih, (Pp.r - Pm.r) * T(0.5) * ih, RR, eps, hh);
            const T phL = ph0.l, phR = ph0.r, uL = u0.l, uR = u0.r;
            const T rL =
                (LL + NL + SQ2 * (phL - lam * (T(1) - phL * phL) * uL)) * M<T>::rcp(acL * acL) - SQ2 * phL * GL;
            const T rR =
                (LR + NR + SQ2 * (phR - lam * (T(1) - phR * phR) * uR)) * M<T>::rcp(acR * acR) - SQ2 * phR * GR;
            psinL = P0.l + dt * rL;
            psinR = P0.r + dt * rR;
            fL = M<T>::tanh_(psinL * ISQ2);
            fR = M<T>::tanh_(psinR * ISQ2);
            dL = fL - phL;
            dR = fR - phR;
        };

        // phase-2 carries: fluxes of row q-1 that row q uses, negated on use
        T cFYm_D[2] = {T(0), T(0)}, cFYm_A[2] = {T(0), T(0)};
        T cFDmm_D[2] = {T(0), T(0)}, cFDmm_A[2] = {T(0), T(0)};
        T cFDpm_D[2] = {T(0), T(0)}, cFDpm_A[2] = {T(0), T(0)};
        T cK_D[2] = {T(0), T(0)}, cK_A[2] = {T(0), T(0)};

        // Phase-2 fluxes at row q: alpha rows q (a*0), q+1 (a*1); U rows q, q+1;
        // psi rows q-2 .. q+2 (Pq[0..4]).  Writes the eight-flux sums of the own
        // columns (times 6 h^2 for the D~_{2,1} forms, times h^2 for S_{1,0})
        // and updates the carries.  need_x = false skips the x-face magnitudes
        // of S_{2,1}, which would read row q-2.
        auto fluxes = [&](const Row<T>& aD0, const Row<T>& aD1, const Row<T>& aA0, const Row<T>& aA1,
                          const Row<T>& bU0, const Row<T>& bU1, const Row<T>* Pq, bool need_x, T& sDL, T& sDR,
                          T& sAL, T& sAR) {
            const Row<T>& b0 = Pq[2];
            const Row<T>& b1 = Pq[3];
            if (S == S10) {
                T fxD[2], fyD[2], fxA[2], fyA[2];
                fxD[0] = T(0.5) * (aD0.l + aD0.r) * (bU0.r - bU0.l);
                fxD[1] = T(0.5) * (aD0.r + aD0.p1) * (bU0.p1 - bU0.r);
                fyD[0] = T(0.5) * (aD0.l + aD1.l) * (bU1.l - bU0.l);
                fyD[1] = T(0.5) * (aD0.r + aD1.r) * (bU1.r - bU0.r);
                {
                    const Row<T>& bm = Pq[1];
                    const T gxl = (b0.r - b0.l) * ih, gyl = (b1.r + b1.l - bm.r - bm.l) * i4h;
                    const T gxr = (b0.p1 - b0.r) * ih, gyr = (b1.p1 + b1.r - bm.p1 - bm.r) * i4h;
                    fxA[0] = guarded_div<T>(T(0.5) * (aA0.l + aA0.r) * (b0.r - b0.l),
                                            M<T>::sqrt_(gxl * gxl + gyl * gyl), hh);
                    fxA[1] = guarded_div<T>(T(0.5) * (aA0.r + aA0.p1) * (b0.p1 - b0.r),
                                            M<T>::sqrt_(gxr * gxr + gyr * gyr), hh);
                    const T yxl = (b1.r + b0.r - b1.m1 - b0.m1) * i4h, yyl = (b1.l - b0.l) * ih;
                    const T yxr = (b1.p1 + b0.p1 - b1.l - b0.l) * i4h, yyr = (b1.r - b0.r) * ih;
                    fyA[0] = guarded_div<T>(T(0.5) * (aA0.l + aA1.l) * (b1.l - b0.l),
                                            M<T>::sqrt_(yxl * yxl + yyl * yyl), hh);
                    fyA[1] = guarded_div<T>(T(0.5) * (aA0.r + aA1.r) * (b1.r - b0.r),
                                            M<T>::sqrt_(yxr * yxr + yyr * yyr), hh);
                }
                const T fxmD = shup(fxD[1]), fxmA = shup(fxA[1]);
                sDL = fxD[0] - fxmD + fyD[0] - cFYm_D[0];
                sDR = fxD[1] - fxD[0] + fyD[1] - cFYm_D[1];
                sAL = fxA[0] - fxmA + fyA[0] - cFYm_A[0];
                sAR = fxA[1] - fxA[0] + fyA[1] - cFYm_A[1];
                cFYm_D[0] = fyD[0];
                cFYm_D[1] = fyD[1];
                cFYm_A[0] = fyA[0];
                cFYm_A[1] = fyA[1];
                return;
            }
            // corner means: the (+1/2, +1/2) corner of columns L-1, L, R at row q
            const T KDm = T(0.25) * (aD0.m1 + aD0.l + aD1.m1 + aD1.l);
            const T KDl = T(0.25) * (aD0.l + aD0.r + aD1.l + aD1.r);
            const T KDr = T(0.25) * (aD0.r + aD0.p1 + aD1.r + aD1.p1);
            const T KAm = T(0.25) * (aA0.m1 + aA0.l + aA1.m1 + aA1.l);
            const T KAl = T(0.25) * (aA0.l + aA0.r + aA1.l + aA1.r);
            const T KAr = T(0.25) * (aA0.r + aA0.p1 + aA1.r + aA1.p1);
            // <10> faces x+, y+ (weight sum of Eq. flux_10) and <11> corners ++, -+
            const T FXpD_L = (aD0.l + aD0.r + KDl + cK_D[0]) * (bU0.r - bU0.l);
            const T FXpD_R = (aD0.r + aD0.p1 + KDr + cK_D[1]) * (bU0.p1 - bU0.r);
            const T FYpD_L = (aD0.l + aD1.l + KDl + KDm) * (bU1.l - bU0.l);
            const T FYpD_R = (aD0.r + aD1.r + KDr + KDl) * (bU1.r - bU0.r);
            const T FPPD_L = KDl * (bU1.r - bU0.l), FPPD_R = KDr * (bU1.p1 - bU0.r);
            const T FMPD_L = KDm * (bU1.m1 - bU0.l), FMPD_R = KDl * (bU1.l - bU0.r);
            T FXpA_L = (aA0.l + aA0.r + KAl + cK_A[0]) * (b0.r - b0.l);
            T FXpA_R = (aA0.r + aA0.p1 + KAr + cK_A[1]) * (b0.p1 - b0.r);
            T FYpA_L = (aA0.l + aA1.l + KAl + KAm) * (b1.l - b0.l);
            T FYpA_R = (aA0.r + aA1.r + KAr + KAl) * (b1.r - b0.r);
            T FPPA_L = KAl * (b1.r - b0.l), FPPA_R = KAr * (b1.p1 - b0.r);
            T FMPA_L = KAm * (b1.m1 - b0.l), FMPA_R = KAl * (b1.l - b0.r);
            if (S == S21) {
                // App. B: each anti-trapping flux divided by |grad psi| at its point;
                // ps(dx, dy) = psi at column L + dx, row q + dy
                auto ps = [&](int dx, int dy) -> T { return Pq[2 + dy].at(dx); };
                if (need_x) {
                    FXpA_L = guarded_div<T>(FXpA_L, appb_face<T>([&](int p, int t) { return ps(p, t); }, ih), hh);
                    FXpA_R =
                        guarded_div<T>(FXpA_R, appb_face<T>([&](int p, int t) { return ps(1 + p, t); }, ih), hh);
                }
                FYpA_L = guarded_div<T>(FYpA_L, appb_face<T>([&](int p, int t) { return ps(t, p); }, ih), hh);
                FYpA_R = guarded_div<T>(FYpA_R, appb_face<T>([&](int p, int t) { return ps(1 + t, p); }, ih), hh);
                FPPA_L = guarded_div<T>(FPPA_L, appb_corner<T>([&](int p, int t) { return ps(p, t); }, ih), hh);
                FPPA_R =
                    guarded_div<T>(FPPA_R, appb_corner<T>([&](int p, int t) { return ps(1 + p, t); }, ih), hh);
                FMPA_L =
                    guarded_div<T>(FMPA_L, appb_corner<T>([&](int p, int t) { return ps(p - 1, t); }, ih), hh);
                FMPA_R = guarded_div<T>(FMPA_R, appb_corner<T>([&](int p, int t) { return ps(p, t); }, ih), hh);
            }
            const T FXmD_L = shup(FXpD_R), FXmA_L = shup(FXpA_R);
            sDL = FXpD_L - FXmD_L + FYpD_L - cFYm_D[0] + FPPD_L + FMPD_L - cFDmm_D[0] - cFDpm_D[0];
            sDR = FXpD_R - FXpD_L + FYpD_R - cFYm_D[1] + FPPD_R + FMPD_R - cFDmm_D[1] - cFDpm_D[1];
            sAL = FXpA_L - FXmA_L + FYpA_L - cFYm_A[0] + FPPA_L + FMPA_L - cFDmm_A[0] - cFDpm_A[0];
            sAR = FXpA_R - FXpA_L + FYpA_R - cFYm_A[1] + FPPA_R + FMPA_R - cFDmm_A[1] - cFDpm_A[1];
            // carries for row q+1: its y- face is this y+ face, its (-1/2,-1/2)
            // corner is the (+1/2,+1/2) corner of the column to the left, its
            // (+1/2,-1/2) corner the (-1/2,+1/2) corner of the column to the right
            cFYm_D[0] = FYpD_L;
            cFYm_D[1] = FYpD_R;
            cFYm_A[0] = FYpA_L;
            cFYm_A[1] = FYpA_R;
            cFDmm_D[0] = shup(FPPD_R);
            cFDmm_D[1] = FPPD_L;
            cFDmm_A[0] = shup(FPPA_R);
            cFDmm_A[1] = FPPA_L;
            cFDpm_D[0] = FMPD_R;
            cFDpm_D[1] = shdn(FMPD_L);
            cFDpm_A[0] = FMPA_R;
            cFDpm_A[1] = shdn(FMPA_L);
            cK_D[0] = KDl;
            cK_D[1] = KDr;
            cK_A[0] = KAl;
            cK_A[1] = KAr;
        };
        auto alphaD = [&](const Row<T>& ph) {
            Row<T> a;
            a.m1 = T(1) - ph.m1;
            a.l = T(1) - ph.l;
            a.r = T(1) - ph.r;
            a.p1 = T(1) - ph.p1;
            a.m2 = a.p2 = T(0);
            return a;
        };
        auto alphaA = [&](const Row<T>& u, const Row<T>& d) {
            Row<T> a;
            a.m1 = (T(1) + omk * u.m1) * d.m1 * isq2dt;
            a.l = (T(1) + omk * u.l) * d.l * isq2dt;
            a.r = (T(1) + omk * u.r) * d.r * isq2dt;
            a.p1 = (T(1) + omk * u.p1) * d.p1 * isq2dt;
            a.m2 = a.p2 = T(0);
            return a;
        };

        // ---------------- prologue ----------------
        Row<T> P[5];   // psi rows r-2 .. r+2 (iteration r)
        Row<T> PH[2];  // phi rows r, r+1
        Row<T> UU[2];  // U rows r, r+1
        Row<T> DP[2];  // delta phi rows r, r+1
        T phinL, phinR;  // phi' at row r
        {
            // psi rows y0-3 .. y0+1 (row y0-3 is read only by S_{2,1}'s x-face
            // magnitudes, which the prologue skips)
            T a, b;
            for (int i = 1; i <= 4; ++i) {
                fetch_row(psi, y0 - 3 + i, a, b);
                P[i] = make_row(a, b);
            }
            P[0] = P[1];
            Row<T> phm = phi_row(P[2]), ph0 = phi_row(P[3]);
            fetch_row(Uf, y0 - 1, a, b);
            Row<T> um = make_row(a, b);
            fetch_row(Uf, y0, a, b);
            Row<T> u0 = make_row(a, b);
            // phase 1 at rows y0-1 and y0; the ghost row -1 copies row 0
            int gL, gR;
            T psL, psR, fL, fR, dLm = T(0), dRm = T(0), dL0, dR0;
            const bool ghost = (y0 - 1) < 0;
            if (!ghost) {
                load_grain_pair(grain + (size_t)(y0 - 1) * nx, cL, nx, vec, gL, gR);
                phase1(y0 - 1, P[1], P[2], P[3], phm, um, gL, gR, psL, psR, fL, fR, dLm, dRm);
            }
            load_grain_pair(grain + (size_t)y0 * nx, cL, nx, vec, gL, gR);
            phase1(y0, P[2], P[3], P[4], ph0, u0, gL, gR, psL, psR, fL, fR, dL0, dR0);
            if (ghost) {
                dLm = dL0;
                dRm = dR0;
            }
            phinL = fL;
            phinR = fR;
            if (y0 < y1) store_pair<T>(psi_o + (size_t)y0 * nx, cL, vec, outL, outR, psL, psR);
            const Row<T> dm = dphi_row(dLm, dRm), d0 = dphi_row(dL0, dR0);
            // phase-2 fluxes at row y0-1 (carries only); psi rows y0-3 .. y0+1
            T s0, s1, s2, s3;
            fluxes(alphaD(phm), alphaD(ph0), alphaA(um, dm), alphaA(u0, d0), um, u0, P, false, s0, s1, s2, s3);
            // ring state for iteration r = y0
            P[0] = P[1];
            P[1] = P[2];
            P[2] = P[3];
            P[3] = P[4];
            PH[0] = ph0;
            UU[0] = u0;
            DP[0] = d0;
        }

        // prefetch psi row y0+2 and U, grain row y0+1
        T nPa, nPb, nUa, nUb;
        int nGa = 0, nGb = 0;
        fetch_row(psi, y0 + 2, nPa, nPb);
        fetch_row(Uf, y0 + 1, nUa, nUb);
        if (y0 + 1 < ny) load_grain_pair(grain + (size_t)(y0 + 1) * nx, cL, nx, vec, nGa, nGb);

        // ---------------- sweep ----------------
        for (int r = y0; r < y1; ++r) {
            P[4] = make_row(nPa, nPb);
            UU[1] = make_row(nUa, nUb);
            PH[1] = phi_row(P[3]);
            const int gL = nGa, gR = nGb;
            fetch_row(psi, r + 3, nPa, nPb);
            fetch_row(Uf, r + 2, nUa, nUb);
            if (r + 2 < ny) load_grain_pair(grain + (size_t)(r + 2) * nx, cL, nx, vec, nGa, nGb);

            // phase 1 at row r+1
            T phnL = T(0), phnR = T(0);
            if (r + 1 < ny) {
                T psL, psR, dL, dR;
                phase1(r + 1, P[2], P[3], P[4], PH[1], UU[1], gL, gR, psL, psR, phnL, phnR, dL, dR);
                if (r + 1 < y1) store_pair<T>(psi_o + (size_t)(r + 1) * nx, cL, vec, outL, outR, psL, psR);
                DP[1] = dphi_row(dL, dR);
            } else {
                DP[1] = DP[0];  // ghost row ny mirrors row ny-1 = r
            }

            // phase 2 at row r
            {
                T sDL, sDR, sAL, sAR;
                fluxes(alphaD(PH[0]), alphaD(PH[1]), alphaA(UU[0], DP[0]), alphaA(UU[1], DP[1]), UU[0], UU[1], P,
                       true, sDL, sDR, sAL, sAR);
                const T cs = (S == S10) ? ih2 : i6h2;
                const T uL = UU[0].l, uR = UU[0].r;
                const T nL = uL + (dt * (Dc * sDL + sAL) * cs + (T(1) + omk * uL) * DP[0].l) *
                                      M<T>::rcp(T(1) + kk - omk * phinL);
                const T nR = uR + (dt * (Dc * sDR + sAR) * cs + (T(1) + omk * uR) * DP[0].r) *
                                      M<T>::rcp(T(1) + kk - omk * phinR);
                store_pair<T>(U_o + (size_t)r * nx, cL, vec, outL, outR, nL, nR);
            }
            phinL = phnL;
            phinR = phnR;
            P[0] = P[1];
            P[1] = P[2];
            P[2] = P[3];
            P[3] = P[4];
            PH[0] = PH[1];
            UU[0] = UU[1];
            DP[0] = DP[1];
        }
    }
}

constexpr int WARPS_PER_BLOCK = 4;

template <typename T, int S>
bool launch_one(int grid_warps, cudaStream_t st, const WorkItem* work, int n_work, const InstRec* recs, int lp) {
    const int blocks = (grid_warps + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    k_step2d<T, S><<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(work, n_work, recs, lp);
    return true;
}

template <typename T, int S> int occ_one() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2d<T, S>, 32 * WARPS_PER_BLOCK, 0) != cudaSuccess)
        return 0;
    return n * WARPS_PER_BLOCK;
}

}  // namespace

// The 2D kernel is warp-granular: `bx` must be 64 (columns a warp holds) and
// `grid` counts warps.
bool launch_step2d(int prec, int scheme, int bx, int grid, cudaStream_t st, const WorkItem* work, int n_work,
                   const InstRec* recs, int lp) {
    if (bx != WARP_COLS) return false;
    if (prec == 0) {
        switch (scheme) {
            case S10: return launch_one<float, S10>(grid, st, work, n_work, recs, lp);
            case S21: return launch_one<float, S21>(grid, st, work, n_work, recs, lp);
            case SBAR21: return launch_one<float, SBAR21>(grid, st, work, n_work, recs, lp);
        }
    } else {
        switch (scheme) {
            case S10: return launch_one<double, S10>(grid, st, work, n_work, recs, lp);
            case S21: return launch_one<double, S21>(grid, st, work, n_work, recs, lp);
            case SBAR21: return launch_one<double, SBAR21>(grid, st, work, n_work, recs, lp);
        }
    }
    return false;
}

// Warps of the fused kernel resident on one SM (0 if not compiled).
int occupancy_step2d(int prec, int scheme, int bx) {
    if (bx != WARP_COLS) return 0;
    if (prec == 0) {
        switch (scheme) {
            case S10: return occ_one<float, S10>();
            case S21: return occ_one<float, S21>();
            case SBAR21: return occ_one<float, SBAR21>();
        }
    } else {
        switch (scheme) {
            case S10: return occ_one<double, S10>();
            case S21: return occ_one<double, S21>();
            case SBAR21: return occ_one<double, SBAR21>();
        }
    }
    return 0;
}

}  // namespace pf
