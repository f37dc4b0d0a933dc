// step2d.cu -- fused explicit time step of the quantitative alloy phase-field
// model in 2D for sm_103a (arXiv:2110.12448, Eqs. PF_a and PF_b).
//
// One kernel advances psi and U together.  A block owns a strip of
// TX = BX - 4 columns and sweeps it row by row ("column-strip sweep"):
//
//   ring buffers in shared memory, indexed by virtual row (mirror ghosts):
//     psi  rows r-5 .. r+2 (8 slots)   phi = tanh(psi/sqrt2) alongside
//     U    rows r-3 .. r+1 (4 slots)   delta phi rows r-3 .. r+1 (4 slots)
//   iteration r:
//     load psi(r+2), U(r+1) for the BX columns x0-2 .. x0+TX+1
//     phase 1 at row r+1 on columns x0-1 .. x0+TX (ring-1 recompute):
//       d psi/dt of Eq. PF_a, psi', phi' and delta phi = phi' - phi
//     phase 2 at row r on columns x0 .. x0+TX-1:
//       U' of Eq. PF_b in conservative form
//
// Each HBM cell value is read once per step by the strip that owns it (plus
// 2 halo columns per 124 and 4 halo rows per sweep), and psi', U' are
// written once: 8 B/cell read + 8 B/cell written in FP32.
//
// No-flux walls are cell-centred mirrors.  A ring cell outside the domain
// takes phase-1 results of its mirror image (the thread computes the mirror
// cell), so the anisotropic terms, which are not mirror symmetric for a
// rotated crystal, are never evaluated at a ghost position.
//
// Discretisations (h = lattice spacing):
//   L_{2,1} (Eq. 2D_L21) or L_{1,0} (Eq. 2D_L10)
//   G_{2,1} = 2/3 G_{1,0} + 1/3 G_{0,1} (App. A) or G_{1,0}
//   O(eps4) terms: div(J - grad psi) on the four <10> faces, J from the face
//     gradient (two-point normal, four-point tangential difference) in the
//     cell's own crystal frame; a_s^2 on the left-hand side and in the G term
//     from the centred gradient
//   D = D~_{2,1}[1 - phi, U] (Eqs. divergence_10/_11, flux_10/_11) or the
//     <10> form with a two-point face mean (S_{1,0})
//   anti-trapping: D~_{2,1}[(1+(1-k)U) dphi/(sqrt2 dt), psi] (Eq.
//     Anti_approx), the App. B form A_{2,1} with the 21-point |grad psi|, or
//     the <10> form normalised by the face gradient (S_{1,0})
//   time levels: U' = U + [dt (D D + A) + (1+(1-k)U) dphi] / (1+k-(1-k)phi')
//     with D on phi^n, U^n and the anti-trapping on psi^n, which conserves
//     the solute integral exactly with mirror walls.
#include "pf_internal.cuh"

namespace pf {
namespace {

template <typename T> __device__ __forceinline__ T dtanh(T x);
template <> __device__ __forceinline__ float dtanh<float>(float x) { return tanhf(x); }
template <> __device__ __forceinline__ double dtanh<double>(double x) { return tanh(x); }
template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }

// Normal component (x face if xface, else y face) of (J - g) for the lab-frame
// face gradient (gx, gy) in a crystal frame with rotation R (crystal -> lab).
//   crystal components c = R^T g, r2 = |c|^2, s_p = c_p^2 / r2,
//   q = sum s_p^2, a_s = 1 - 3 eps + 4 eps q  (= 1 + eps cos 4 theta),
//   J'_p - c_p = c_p (a^2 - 1 - 16 eps a q + 16 eps a s_p),
// which is d(a_s^2 |g|^2 / 2)/dg minus g, rotated back by R.
template <typename T>
__device__ __forceinline__ T aniso_qn(T gx, T gy, T R00, T R01, T R10, T R11, T eps, T hh, bool xface) {
    const T cx = R00 * gx + R10 * gy;
    const T cy = R01 * gx + R11 * gy;
    const T r2 = cx * cx + cy * cy;
    if (r2 * hh < Guard<T>::v) return T(0);
    const T inv = T(1) / r2;
    const T sx = cx * cx * inv, sy = cy * cy * inv;
    const T q = sx * sx + sy * sy;
    const T a = T(1) - T(3) * eps + T(4) * eps * q;
    const T c1 = T(16) * eps * a;
    const T c0 = a * a - T(1) - c1 * q;
    const T jx = cx * (c0 + c1 * sx), jy = cy * (c0 + c1 * sy);
    return xface ? (R00 * jx + R01 * jy) : (R10 * jx + R11 * jy);
}

template <typename T>
__device__ __forceinline__ T aniso_a(T gx, T gy, T R00, T R01, T R10, T R11, T eps, T hh) {
    const T cx = R00 * gx + R10 * gy;
    const T cy = R01 * gx + R11 * gy;
    const T r2 = cx * cx + cy * cy;
    if (r2 * hh < Guard<T>::v) return T(1);
    const T inv = T(1) / r2;
    const T sx = cx * cx * inv, sy = cy * cy * inv;
    return T(1) - T(3) * eps + T(4) * eps * (sx * sx + sy * sy);
}

// App. B: |grad b| at a <10> face.  B(p, q) = b at origin + p (normal) + q
// (tangent); returns the magnitude of (d_n, d_t).
template <typename T, typename F>
__device__ __forceinline__ T appb_face(F B, T ih) {
    const T a1 = B(1, 1) - B(0, -1), a2 = B(0, 1) - B(1, -1);
    const T b1 = B(2, 1) - B(-1, -1), b2 = B(-1, 1) - B(2, -1);
    const T c1 = B(1, 2) - B(0, -2), c2 = B(0, 2) - B(1, -2);
    const T dn = (T(35.0 / 24.0) * (a1 - a2) * T(0.5) - T(1.0 / 8.0) * (b1 - b2) * T(1.0 / 6.0) -
                  T(1.0 / 3.0) * (c1 - c2) * T(0.5)) * ih;
    const T dt = (T(35.0 / 24.0) * (a1 + a2) * T(0.25) - T(1.0 / 8.0) * (b1 + b2) * T(0.25) -
                  T(1.0 / 3.0) * (c1 + c2) * T(0.125)) * ih;
    return dsqrt<T>(dn * dn + dt * dt);
}
// App. B: |grad b| at a corner; B(p, q) = b at origin + p x + q y.
template <typename T, typename F>
__device__ __forceinline__ T appb_corner(F B, T ih) {
    const T a1 = B(1, 1) - B(0, 0), a2 = B(0, 1) - B(1, 0);
    const T b1 = B(2, 1) - B(-1, 0), b2 = B(-1, 1) - B(2, 0);
    const T c1 = B(1, 2) - B(0, -1), c2 = B(0, 2) - B(1, -1);
    const T dx = (T(5.0 / 4.0) * (a1 - a2) * T(0.5) - T(1.0 / 8.0) * (b1 - b2) * T(1.0 / 6.0) -
                  T(1.0 / 8.0) * (c1 - c2) * T(0.5)) * ih;
    const T dy = (T(5.0 / 4.0) * (a1 + a2) * T(0.5) - T(1.0 / 8.0) * (b1 + b2) * T(0.5) -
                  T(1.0 / 8.0) * (c1 + c2) * T(1.0 / 6.0)) * ih;
    return dsqrt<T>(dx * dx + dy * dy);
}

// D~_{2,1}[a, b] * 6 h^2 on a 3x3 neighbourhood a[y][x], b[y][x] (centre [1][1]):
// four <10> fluxes with the alpha average of Eq. flux_10 and four <11> fluxes
// with the four-point mean C of Eq. flux_11, weights 2/3 and 1/3.
// <10>: D~_{1,0} = sum W db / (4 h^2), W = a0 + a1 + two corner means;
// weight 2/3 -> W db / (6 h^2).
template <typename T>
__device__ __forceinline__ T div21_x6h2(const T (&a)[3][3], const T (&b)[3][3]) {
    const T c = a[1][1];
    const T Cpp = T(0.25) * (c + a[1][2] + a[2][1] + a[2][2]);
    const T Cmp = T(0.25) * (c + a[1][0] + a[2][1] + a[2][0]);
    const T Cpm = T(0.25) * (c + a[1][2] + a[0][1] + a[0][2]);
    const T Cmm = T(0.25) * (c + a[1][0] + a[0][1] + a[0][0]);
    const T b0 = b[1][1];
    T s = (a[1][2] + c + Cpp + Cpm) * (b[1][2] - b0);
    s += (a[1][0] + c + Cmp + Cmm) * (b[1][0] - b0);
    s += (a[2][1] + c + Cpp + Cmp) * (b[2][1] - b0);
    s += (a[0][1] + c + Cpm + Cmm) * (b[0][1] - b0);
    // corners: D~_{0,1} = sum C db / (2 h^2); weight 1/3 -> C db / (6 h^2)
    s += Cpp * (b[2][2] - b0) + Cmp * (b[2][0] - b0) + Cpm * (b[0][2] - b0) + Cmm * (b[0][0] - b0);
    return s;
}

template <typename T, int S, int BX>
__global__ void __launch_bounds__(BX) k_step2d(const WorkItem* __restrict__ work, int n_work,
                                               const InstRec* __restrict__ recs, int launch_parity) {
    constexpr int TX = BX - 4;
    constexpr bool ISO = (S == S21 || S == SBAR21);
    __shared__ T s_psi[8][BX];
    __shared__ T s_phi[8][BX];
    __shared__ T s_U[4][BX];
    __shared__ T s_dphi[4][BX];
    const int t = threadIdx.x;
    const T SQ2 = T(1.41421356237309504880);
    const T ISQ2 = T(0.70710678118654752440);

    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const WorkItem wi = work[w];
        const InstRec& rec = recs[wi.inst];
        const int nx = rec.nx, ny = rec.ny;
        const int par = rec.parity_offset ^ launch_parity;
        const T* __restrict__ psi = static_cast<const T*>(rec.psi[par]);
        const T* __restrict__ U = static_cast<const T*>(rec.U[par]);
        T* __restrict__ psi_o = static_cast<T*>(rec.psi[par ^ 1]);
        T* __restrict__ U_o = static_cast<T*>(rec.U[par ^ 1]);
        const int16_t* __restrict__ grain = rec.grain;
        const T* __restrict__ rot = static_cast<const T*>(rec.rot);
        const T h = T(rec.h), ih = T(1.0 / rec.h), hh = T(rec.h * rec.h), dt = T(rec.dt);
        const T kk = T(rec.k), omk = T(1.0 - rec.k), eps = T(rec.eps4), lam = T(rec.lambda), Dc = T(rec.D);
        const T ih2 = T(1.0 / (rec.h * rec.h));
        const T i6h2 = T(1.0 / (6.0 * rec.h * rec.h));
        const T i4h2 = T(1.0 / (4.0 * rec.h * rec.h)), i8h2 = T(1.0 / (8.0 * rec.h * rec.h));
        const T isq2dt = T(1.0 / (1.41421356237309504880 * rec.dt));
        (void)h;

        const int x0 = wi.x0, y0 = wi.y0;
        const int y1 = min(y0 + wi.ext, ny);
        const int c = x0 - 2 + t;                 // virtual column of this thread
        const int cl = mirror_idx(c, nx);         // column loaded for it
        const bool do_p1 = (t >= 1) && (t <= BX - 2) && (c >= -1) && (c <= nx);
        const int mc = mirror_idx(c, nx);         // phase-1 cell column
        const int jc = mc - x0 + 2;               // its shared-memory column
        const bool do_p2 = (t >= 2) && (t <= BX - 3) && (c < nx);

        auto load_psi = [&](int vr) {
            const int rr = mirror_idx(vr, ny);
            const T v = psi[(size_t)rr * nx + cl];
            s_psi[vr & 7][t] = v;
            s_phi[vr & 7][t] = dtanh<T>(v * ISQ2);
        };
        auto load_U = [&](int vr) {
            const int rr = mirror_idx(vr, ny);
            s_U[vr & 3][t] = U[(size_t)rr * nx + cl];
        };

        // phase 1 at virtual row p: writes delta phi, returns phi' (and psi' via ref)
        auto phase1 = [&](int p, T& psin_out) -> T {
            const int mp = mirror_idx(p, ny);
            const int g = grain[(size_t)mp * nx + mc];
            const T* Rg = rot + 9 * g;
            const T R00 = Rg[0], R01 = Rg[1], R10 = Rg[3], R11 = Rg[4];
            const T* rowN = s_psi[(mp + 1) & 7];  // y + 1
            const T* row0 = s_psi[mp & 7];
            const T* rowS = s_psi[(mp - 1) & 7];  // y - 1
            const T pc = row0[jc], pe = row0[jc + 1], pw = row0[jc - 1];
            const T pn = rowN[jc], pne = rowN[jc + 1], pnw = rowN[jc - 1];
            const T ps = rowS[jc], pse = rowS[jc + 1], psw = rowS[jc - 1];
            const T ph = s_phi[mp & 7][jc];
            const T u = s_U[mp & 3][jc];
            T L, G;
            if (ISO) {
                L = (T(4) * (pe + pw + pn + ps) + (pne + pnw + pse + psw) - T(20) * pc) * i6h2;
                const T g10 = ((pe - pw) * (pe - pw) + (pn - ps) * (pn - ps)) * i4h2;
                const T g01 = ((pne - psw) * (pne - psw) + (pse - pnw) * (pse - pnw)) * i8h2;
                G = T(2.0 / 3.0) * g10 + T(1.0 / 3.0) * g01;
            } else {
                L = (pe + pw + pn + ps - T(4) * pc) * ih2;
                G = ((pe - pw) * (pe - pw) + (pn - ps) * (pn - ps)) * i4h2;
            }
            const T ac = aniso_a<T>((pe - pw) * T(0.5) * ih, (pn - ps) * T(0.5) * ih, R00, R01, R10, R11, eps, hh);
            const T i4h = T(0.25) * ih;
            // <10> faces: (J - g) normal components
            const T qxp = aniso_qn<T>((pe - pc) * ih, (pne + pn - pse - ps) * i4h, R00, R01, R10, R11, eps, hh, true);
            const T qxm = aniso_qn<T>((pc - pw) * ih, (pn + pnw - ps - psw) * i4h, R00, R01, R10, R11, eps, hh, true);
            const T qyp = aniso_qn<T>((pne + pe - pnw - pw) * i4h, (pn - pc) * ih, R00, R01, R10, R11, eps, hh, false);
            const T qym = aniso_qn<T>((pe + pse - pw - psw) * i4h, (pc - ps) * ih, R00, R01, R10, R11, eps, hh, false);
            const T N = (qxp - qxm + qyp - qym) * ih;
            const T rate = (L + N + SQ2 * (ph - lam * (T(1) - ph * ph) * u)) / (ac * ac) - SQ2 * ph * G;
            const T psin = pc + dt * rate;
            const T phin = dtanh<T>(psin * ISQ2);
            s_dphi[p & 3][t] = phin - ph;
            psin_out = psin;
            return phin;
        };

        // ---- prologue ----
        for (int vr = y0 - 2; vr <= y0 + 1; ++vr) load_psi(vr);
        load_U(y0 - 1);
        load_U(y0);
        __syncthreads();
        T phin_cur = T(0);
        {
            T dummy;
            if (do_p1) (void)phase1(y0 - 1, dummy);
            if (do_p1) {
                T psin;
                phin_cur = phase1(y0, psin);
                if (do_p2) psi_o[(size_t)y0 * nx + c] = psin;
            }
        }
        __syncthreads();

        // ---- sweep ----
        for (int r = y0; r < y1; ++r) {
            load_psi(r + 2);
            load_U(r + 1);
            __syncthreads();
            T phin_next = T(0);
            if (do_p1) {
                T psin;
                phin_next = phase1(r + 1, psin);
                if (do_p2 && r + 1 < y1) psi_o[(size_t)(r + 1) * nx + c] = psin;
            }
            __syncthreads();
            if (do_p2) {
                T aD[3][3], bU[3][3], aA[3][3], bP[3][3];
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        const T phv = s_phi[(r + dy) & 7][t + dx];
                        const T uv = s_U[(r + dy) & 3][t + dx];
                        aD[dy + 1][dx + 1] = T(1) - phv;
                        bU[dy + 1][dx + 1] = uv;
                        aA[dy + 1][dx + 1] = (T(1) + omk * uv) * s_dphi[(r + dy) & 3][t + dx] * isq2dt;
                        bP[dy + 1][dx + 1] = s_psi[(r + dy) & 7][t + dx];
                    }
                }
                T Dt, At;
                if (S == S10) {
                    const T ac = aD[1][1], bc = bU[1][1];
                    Dt = (T(0.5) * (aD[1][2] + ac) * (bU[1][2] - bc) + T(0.5) * (aD[1][0] + ac) * (bU[1][0] - bc) +
                          T(0.5) * (aD[2][1] + ac) * (bU[2][1] - bc) + T(0.5) * (aD[0][1] + ac) * (bU[0][1] - bc)) *
                         ih2;
                    // <10> anti-trapping normalised by the face gradient
                    const T i4h = T(0.25) * ih;
                    const T pc = bP[1][1];
                    T s = T(0);
                    {
                        const T gx = (bP[1][2] - pc) * ih, gy = (bP[2][2] + bP[2][1] - bP[0][2] - bP[0][1]) * i4h;
                        const T m2 = gx * gx + gy * gy;
                        if (!(m2 * hh < Guard<T>::v)) s += T(0.5) * (aA[1][2] + aA[1][1]) * gx / dsqrt<T>(m2);
                    }
                    {
                        const T gx = (pc - bP[1][0]) * ih, gy = (bP[2][1] + bP[2][0] - bP[0][1] - bP[0][0]) * i4h;
                        const T m2 = gx * gx + gy * gy;
                        if (!(m2 * hh < Guard<T>::v)) s -= T(0.5) * (aA[1][0] + aA[1][1]) * gx / dsqrt<T>(m2);
                    }
                    {
                        const T gx = (bP[2][2] + bP[1][2] - bP[2][0] - bP[1][0]) * i4h, gy = (bP[2][1] - pc) * ih;
                        const T m2 = gx * gx + gy * gy;
                        if (!(m2 * hh < Guard<T>::v)) s += T(0.5) * (aA[2][1] + aA[1][1]) * gy / dsqrt<T>(m2);
                    }
                    {
                        const T gx = (bP[1][2] + bP[0][2] - bP[1][0] - bP[0][0]) * i4h, gy = (pc - bP[0][1]) * ih;
                        const T m2 = gx * gx + gy * gy;
                        if (!(m2 * hh < Guard<T>::v)) s -= T(0.5) * (aA[0][1] + aA[1][1]) * gy / dsqrt<T>(m2);
                    }
                    At = s * ih;
                } else {
                    Dt = div21_x6h2<T>(aD, bU) * i6h2;
                    if (S == SBAR21) {
                        At = div21_x6h2<T>(aA, bP) * i6h2;
                    } else {
                        // S21: App. B standard anti-trapping with the 21-point |grad psi|
                        auto P = [&](int dx, int dy) -> T { return s_psi[(r + dy) & 7][t + dx]; };
                        const T a = aA[1][1];
                        const T Cpp = T(0.25) * (a + aA[1][2] + aA[2][1] + aA[2][2]);
                        const T Cmp = T(0.25) * (a + aA[1][0] + aA[2][1] + aA[2][0]);
                        const T Cpm = T(0.25) * (a + aA[1][2] + aA[0][1] + aA[0][2]);
                        const T Cmm = T(0.25) * (a + aA[1][0] + aA[0][1] + aA[0][0]);
                        const T b0 = bP[1][1];
                        const T mxp = appb_face<T>([&](int p, int q) { return P(p, q); }, ih);
                        const T mxm = appb_face<T>([&](int p, int q) { return P(p - 1, q); }, ih);
                        const T myp = appb_face<T>([&](int p, int q) { return P(q, p); }, ih);
                        const T mym = appb_face<T>([&](int p, int q) { return P(q, p - 1); }, ih);
                        const T mpp = appb_corner<T>([&](int p, int q) { return P(p, q); }, ih);
                        const T mmp = appb_corner<T>([&](int p, int q) { return P(p - 1, q); }, ih);
                        const T mpm = appb_corner<T>([&](int p, int q) { return P(p, q - 1); }, ih);
                        const T mmm = appb_corner<T>([&](int p, int q) { return P(p - 1, q - 1); }, ih);
                        T s = T(0);
                        auto acc = [&](T wgt, T db, T m) {
                            if (!(m * m * hh < Guard<T>::v)) s += wgt * db / m;
                        };
                        acc(aA[1][2] + a + Cpp + Cpm, bP[1][2] - b0, mxp);
                        acc(aA[1][0] + a + Cmp + Cmm, bP[1][0] - b0, mxm);
                        acc(aA[2][1] + a + Cpp + Cmp, bP[2][1] - b0, myp);
                        acc(aA[0][1] + a + Cpm + Cmm, bP[0][1] - b0, mym);
                        acc(Cpp, bP[2][2] - b0, mpp);
                        acc(Cmp, bP[2][0] - b0, mmp);
                        acc(Cpm, bP[0][2] - b0, mpm);
                        acc(Cmm, bP[0][0] - b0, mmm);
                        At = s * i6h2;
                    }
                }
                const T uc = bU[1][1];
                const T dph = s_dphi[r & 3][t];
                const T un = uc + (dt * (Dc * Dt + At) + (T(1) + omk * uc) * dph) / (T(1) + kk - omk * phin_cur);
                U_o[(size_t)r * nx + c] = un;
            }
            phin_cur = phin_next;
        }
        __syncthreads();
    }
}

template <typename T, int S, int BX>
bool launch_one(int grid, cudaStream_t st, const WorkItem* work, int n_work, const InstRec* recs, int lp) {
    k_step2d<T, S, BX><<<grid, BX, 0, st>>>(work, n_work, recs, lp);
    return true;
}

template <typename T, int S, int BX> int occ_one() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2d<T, S, BX>, BX, 0) != cudaSuccess) return 0;
    return n;
}

template <typename T, int S>
bool launch_bx(int bx, int grid, cudaStream_t st, const WorkItem* work, int n_work, const InstRec* recs, int lp) {
    switch (bx) {
        case 64: return launch_one<T, S, 64>(grid, st, work, n_work, recs, lp);
        case 128: return launch_one<T, S, 128>(grid, st, work, n_work, recs, lp);
        case 256: return launch_one<T, S, 256>(grid, st, work, n_work, recs, lp);
        default: return false;
    }
}
template <typename T, int S> int occ_bx(int bx) {
    switch (bx) {
        case 64: return occ_one<T, S, 64>();
        case 128: return occ_one<T, S, 128>();
        case 256: return occ_one<T, S, 256>();
        default: return 0;
    }
}

}  // namespace

bool launch_step2d(int prec, int scheme, int bx, int grid, cudaStream_t st, const WorkItem* work, int n_work,
                   const InstRec* recs, int lp) {
    if (prec == 0) {
        switch (scheme) {
            case S10: return launch_bx<float, S10>(bx, grid, st, work, n_work, recs, lp);
            case S21: return launch_bx<float, S21>(bx, grid, st, work, n_work, recs, lp);
            case SBAR21: return launch_bx<float, SBAR21>(bx, grid, st, work, n_work, recs, lp);
        }
    } else {
        switch (scheme) {
            case S10: return launch_bx<double, S10>(bx, grid, st, work, n_work, recs, lp);
            case S21: return launch_bx<double, S21>(bx, grid, st, work, n_work, recs, lp);
            case SBAR21: return launch_bx<double, SBAR21>(bx, grid, st, work, n_work, recs, lp);
        }
    }
    return false;
}

int occupancy_step2d(int prec, int scheme, int bx) {
    if (prec == 0) {
        switch (scheme) {
            case S10: return occ_bx<float, S10>(bx);
            case S21: return occ_bx<float, S21>(bx);
            case SBAR21: return occ_bx<float, SBAR21>(bx);
        }
    } else {
        switch (scheme) {
            case S10: return occ_bx<double, S10>(bx);
            case S21: return occ_bx<double, S21>(bx);
            case SBAR21: return occ_bx<double, SBAR21>(bx);
        }
    }
    return 0;
}

}  // namespace pf
