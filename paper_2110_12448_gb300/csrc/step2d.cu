// step2d.cu -- fused explicit time step of the quantitative alloy phase-field
// model in 2D for sm_103a (arXiv:2110.12448, Eqs. PF_a and PF_b).
//
// Warp-per-strip design.  Each warp owns a strip of 60 output columns and
// sweeps it row by row; lane t holds the two columns L = x0-2+2t, R = L+1
// (lanes 0 and 31 carry the halo).  Nothing is shared between warps: there is
// no shared memory and no block barrier.  Neighbour columns come over warp
// shuffles, rows live in a register ring, and every face flux is computed
// once and handed to the other cell that uses it (shuffle across columns,
// register carry across rows).  The two columns of a lane are processed as a
// packed pair (FP32: the sm_100 float2 FMA/ADD/MUL instructions, one issue
// slot for both columns).  Global traffic per step: psi, U and the int16
// grain read once, psi' and U' written once (float2 / int32 vectors).
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

// ---------------------------------------------------------------------------
// scalar helpers: FP32 uses the single-instruction approximate reciprocal and
// base-2 exponential; FP64 uses IEEE operations
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// x / y from the reciprocal estimate and one Newton correction of the
// quotient (Markstein): q = x r, then q + (x - q y) r with the residual in
// one FMA.  Within about an ulp of x / y for normal operands, with no
// slow-path test; the compensated state's divisions either feed a residual
// step that corrects the quotient to double-float precision or form small
// increments whose last-bit error is far below the state's lo half.
__device__ __forceinline__ float div_nr(float x, float y) {
    const float r = rcp_approx(y);
    const float q = x * r;
    return fmaf(fmaf(-q, y, x), r, q);
}
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <typename T> struct M;
#ifndef PF_PRECISE_F32
template <> struct M<float> {
    // tanh(x / sqrt2) = 1 - 2 / (1 + e^{sqrt2 x}) = 1 - 2 / (1 + 2^{sqrt2 log2(e) x});
    // absolute error ~2e-7 over the whole range
    static __device__ __forceinline__ float tanh_isq2(float x) {
        const float e = ex2_approx(x * 2.0402467570003297f);  // sqrt2 * log2(e)
        return fmaf(-2.0f, rcp_approx(1.0f + e), 1.0f);
    }
    static __device__ __forceinline__ float rcp(float x) { return rcp_approx(x); }
    // single-instruction approximate square root (0 at 0): the App. B and
    // <10> anti-trapping magnitudes, guarded where |grad psi| vanishes
    static __device__ __forceinline__ float sqrt_(float x) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
};
#else
// correctly rounded division and the library tanh (slower; for accuracy studies)
template <> struct M<float> {
    static __device__ __forceinline__ float tanh_isq2(float x) { return tanhf(x * 0.70710678118654752440f); }
    static __device__ __forceinline__ float rcp(float x) { return 1.0f / x; }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
};
#endif
template <> struct M<double> {
    static __device__ __forceinline__ double tanh_isq2(double x) { return tanh(x * 0.70710678118654752440); }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
};

// ---------------------------------------------------------------------------
// packed pair of the two columns of a lane
// ---------------------------------------------------------------------------
template <typename T> struct V;
template <> struct V<float> {
    float2 v;
    __device__ __forceinline__ float x() const { return v.x; }
    __device__ __forceinline__ float y() const { return v.y; }
};
template <> struct V<double> {
    double vx, vy;
    __device__ __forceinline__ double x() const { return vx; }
    __device__ __forceinline__ double y() const { return vy; }
};
__device__ __forceinline__ V<float> mk(float a, float b) {
    V<float> r;
    r.v = make_float2(a, b);
    return r;
}
__device__ __forceinline__ V<double> mk(double a, double b) {
    V<double> r;
    r.vx = a;
    r.vy = b;
    return r;
}
template <typename T> __device__ __forceinline__ V<T> bc(T a) { return mk(a, a); }
__device__ __forceinline__ V<float> operator+(V<float> a, V<float> b) {
    V<float> r;
    r.v = __fadd2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ V<float> operator-(V<float> a, V<float> b) {
    V<float> r;
    r.v = __ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v);  // exactly a - b
    return r;
}
__device__ __forceinline__ V<float> operator*(V<float> a, V<float> b) {
    V<float> r;
    r.v = __fmul2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ V<float> fma(V<float> a, V<float> b, V<float> c) {
    V<float> r;
    r.v = __ffma2_rn(a.v, b.v, c.v);
    return r;
}
__device__ __forceinline__ V<double> operator+(V<double> a, V<double> b) { return mk(a.vx + b.vx, a.vy + b.vy); }
__device__ __forceinline__ V<double> operator-(V<double> a, V<double> b) { return mk(a.vx - b.vx, a.vy - b.vy); }
__device__ __forceinline__ V<double> operator*(V<double> a, V<double> b) { return mk(a.vx * b.vx, a.vy * b.vy); }
__device__ __forceinline__ V<double> fma(V<double> a, V<double> b, V<double> c) {
    return mk(::fma(a.vx, b.vx, c.vx), ::fma(a.vy, b.vy, c.vy));
}
template <typename T> __device__ __forceinline__ V<T> rcp2(V<T> a) { return mk(M<T>::rcp(a.x()), M<T>::rcp(a.y())); }

template <typename T> __device__ __forceinline__ T shup(T v) { return __shfl_up_sync(FULL, v, 1); }
template <typename T> __device__ __forceinline__ T shdn(T v) { return __shfl_down_sync(FULL, v, 1); }

// A row as one lane sees it: columns L-2 .. L+3 (m2/p2 only for S_{2,1}'s psi).
template <typename T> struct Row {
    T m2, m1, l, r, p1, p2;
    __device__ __forceinline__ T at(int o) const {
        return o == -2 ? m2 : o == -1 ? m1 : o == 0 ? l : o == 1 ? r : o == 2 ? p1 : p2;
    }
    __device__ __forceinline__ V<T> W() const { return mk(m1, l); }  // west neighbours of (L, R)
    __device__ __forceinline__ V<T> C() const { return mk(l, r); }   // (L, R)
    __device__ __forceinline__ V<T> E() const { return mk(r, p1); }  // east neighbours
    __device__ __forceinline__ V<T> pat(int o) const { return mk(at(o), at(o + 1)); }
};

// Crystal frames of the two columns (upper 2x2 of crystal -> lab rotations).
template <typename T> struct Rot2 {
    V<T> a, b, c, d;  // (R00, R01, R10, R11) of column L in .x, of column R in .y
};

// Normal component of (J - g) for face gradients (gx, gy) of both columns.
//   crystal components c = R^T g, r2 = |c|^2, s_p = c_p^2 / r2, q = sum s_p^2,
//   a_s = 1 - 3 eps + 4 eps q (= 1 + eps cos 4 theta, Eq. anis_function),
//   J'_p - c_p = c_p (a^2 - 1 - 16 eps a q + 16 eps a s_p)
// i.e. d(a_s^2 |g|^2 / 2)/dg - g, rotated back to the lab frame; 0 below the
// |g|^2 h^2 guard.
template <typename T>
__device__ __forceinline__ V<T> aniso_qn2(V<T> gx, V<T> gy, const Rot2<T>& R, T eps, T hh, bool xface) {
    const V<T> cx = fma(R.a, gx, R.c * gy);
    const V<T> cy = fma(R.b, gx, R.d * gy);
    const V<T> r2 = fma(cx, cx, cy * cy);
    const V<T> inv = rcp2(r2);
    const V<T> sx = cx * cx * inv, sy = cy * cy * inv;
    const V<T> q = fma(sx, sx, sy * sy);
    const V<T> a = fma(bc<T>(T(4) * eps), q, bc<T>(T(1) - T(3) * eps));
    const V<T> c1 = bc<T>(T(16) * eps) * a;
    const V<T> c0 = fma(a, a, bc<T>(T(-1))) - c1 * q;
    const V<T> jx = cx * fma(c1, sx, c0), jy = cy * fma(c1, sy, c0);
    const V<T> o = xface ? fma(R.a, jx, R.b * jy) : fma(R.c, jx, R.d * jy);
    return mk(r2.x() * hh < Guard<T>::v ? T(0) : o.x(), r2.y() * hh < Guard<T>::v ? T(0) : o.y());
}
template <typename T> __device__ __forceinline__ V<T> aniso_a2(V<T> gx, V<T> gy, const Rot2<T>& R, T eps, T hh) {
    const V<T> cx = fma(R.a, gx, R.c * gy);
    const V<T> cy = fma(R.b, gx, R.d * gy);
    const V<T> r2 = fma(cx, cx, cy * cy);
    const V<T> inv = rcp2(r2);
    const V<T> sx = cx * cx * inv, sy = cy * cy * inv;
    const V<T> a = fma(bc<T>(T(4) * eps), fma(sx, sx, sy * sy), bc<T>(T(1) - T(3) * eps));
    return mk(r2.x() * hh < Guard<T>::v ? T(1) : a.x(), r2.y() * hh < Guard<T>::v ? T(1) : a.y());
}
// The same normal component of J - g without the cancellation in a^2 - 1
// (the compensated state): with s_x + s_y = 1 in 2D, a - 1 = eps (4q - 3) =
// eps (1 - 8 s_x s_y), a^2 - 1 = (a - 1)(a + 1), and s_x - q = s_y (s_x - s_y),
// s_y - q = -s_x (s_x - s_y), so
//   J'_x - c_x = c_x eps [b (2 + eps b) + 16 a s_y (s_x - s_y)],
//   J'_y - c_y = c_y eps [b (2 + eps b) - 16 a s_x (s_x - s_y)],  b = 1 - 8 s_x s_y,
// every term formed without subtracting nearly equal numbers.
template <typename T>
__device__ __forceinline__ V<T> aniso_qn2c(V<T> gx, V<T> gy, const Rot2<T>& R, T eps, T hh, bool xface) {
    const V<T> cx = fma(R.a, gx, R.c * gy);
    const V<T> cy = fma(R.b, gx, R.d * gy);
    const V<T> r2 = fma(cx, cx, cy * cy);
    const V<T> inv = rcp2(r2);
    const V<T> sx = cx * cx * inv, sy = cy * cy * inv;
    const V<T> dxy = (cx - cy) * (cx + cy) * inv;  // s_x - s_y
    const V<T> b = fma(bc<T>(T(-8)) * sx, sy, bc<T>(T(1)));
    const V<T> a = fma(bc<T>(eps), b, bc<T>(T(1)));
    const V<T> B = b * fma(bc<T>(eps), b, bc<T>(T(2)));
    const V<T> t = bc<T>(T(16)) * a * dxy;
    const V<T> jx = cx * bc<T>(eps) * fma(t, sy, B), jy = cy * bc<T>(eps) * fma(t * bc<T>(T(-1)), sx, B);
    const V<T> o = xface ? fma(R.a, jx, R.b * jy) : fma(R.c, jx, R.d * jy);
    return mk(r2.x() * hh < Guard<T>::v ? T(0) : o.x(), r2.y() * hh < Guard<T>::v ? T(0) : o.y());
}
template <typename T>
__device__ __forceinline__ T aniso_qn1c(T gx, T gy, T Ra, T Rb, T Rc, T Rd, T eps, T hh, bool xface) {
    const T cx = Ra * gx + Rc * gy;
    const T cy = Rb * gx + Rd * gy;
    const T r2 = cx * cx + cy * cy;
    if (r2 * hh < Guard<T>::v) return T(0);
    const T inv = M<T>::rcp(r2);
    const T sx = cx * cx * inv, sy = cy * cy * inv;
    const T dxy = (cx - cy) * (cx + cy) * inv;
    const T b = T(1) - T(8) * sx * sy;
    const T a = T(1) + eps * b;
    const T B = b * (T(2) + eps * b);
    const T t = T(16) * a * dxy;
    const T jx = cx * eps * (B + t * sy), jy = cy * eps * (B - t * sx);
    return xface ? (Ra * jx + Rb * jy) : (Rc * jx + Rd * jy);
}
// the anisotropic part 4 eps q of a_s = (1 - 3 eps) + 4 eps q (3 eps where
// the normal is undefined, so that a_s = 1): the compensated state forms
// a_s in double-float from it
template <typename T> __device__ __forceinline__ V<T> aniso_w2(V<T> gx, V<T> gy, const Rot2<T>& R, T eps, T hh) {
    const V<T> cx = fma(R.a, gx, R.c * gy);
    const V<T> cy = fma(R.b, gx, R.d * gy);
    const V<T> r2 = fma(cx, cx, cy * cy);
    const V<T> inv = rcp2(r2);
    const V<T> sx = cx * cx * inv, sy = cy * cy * inv;
    const V<T> w = bc<T>(T(4) * eps) * fma(sx, sx, sy * sy);
    return mk(r2.x() * hh < Guard<T>::v ? T(3) * eps : w.x(), r2.y() * hh < Guard<T>::v ? T(3) * eps : w.y());
}
// explicitly rounded scalar operations: the compiler contracts none of them,
// so every kernel that inlines the scalar face below computes the same bits
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// scalar version for the rare faces between two grains
template <typename T>
__device__ __forceinline__ T aniso_qn1(T gx, T gy, T Ra, T Rb, T Rc, T Rd, T eps, T hh, bool xface) {
    const T cx = Ra * gx + Rc * gy;
    const T cy = Rb * gx + Rd * gy;
    const T r2 = cx * cx + cy * cy;
    if (r2 * hh < Guard<T>::v) return T(0);
    const T inv = M<T>::rcp(r2);
    const T sx = cx * cx * inv, sy = cy * cy * inv;
    const T q = sx * sx + sy * sy;
    const T a = T(1) - T(3) * eps + T(4) * eps * q;
    const T c1 = T(16) * eps * a;
    const T c0 = a * a - T(1) - c1 * q;
    const T jx = cx * (c0 + c1 * sx), jy = cy * (c0 + c1 * sy);
    return xface ? (Ra * jx + Rb * jy) : (Rc * jx + Rd * jy);
}
// The same face with every operation explicitly rounded, for the T0 kernels:
// the fused T0 step and the two passes of the two-kernel form then compute
// the same bits (the contractible version above may be contracted
// differently in different kernels).
template <typename T>
__device__ __forceinline__ T aniso_qn1_rn(T gx, T gy, T Ra, T Rb, T Rc, T Rd, T eps, T hh, bool xface) {
    const T cx = rn_fma(Ra, gx, rn_mul(Rc, gy));
    const T cy = rn_fma(Rb, gx, rn_mul(Rd, gy));
    const T r2 = rn_fma(cx, cx, rn_mul(cy, cy));
    if (rn_mul(r2, hh) < Guard<T>::v) return T(0);
    const T inv = M<T>::rcp(r2);
    const T sx = rn_mul(rn_mul(cx, cx), inv), sy = rn_mul(rn_mul(cy, cy), inv);
    const T q = rn_fma(sx, sx, rn_mul(sy, sy));
    const T e4 = rn_mul(T(4), eps);
    const T a = rn_fma(e4, q, rn_fma(T(-3), eps, T(1)));
    const T c1 = rn_mul(rn_mul(T(16), eps), a);
    const T c0 = rn_add(rn_fma(a, a, T(-1)), -rn_mul(c1, q));
    const T jx = rn_mul(cx, rn_fma(c1, sx, c0)), jy = rn_mul(cy, rn_fma(c1, sy, c0));
    return xface ? rn_fma(Ra, jx, rn_mul(Rb, jy)) : rn_fma(Rc, jx, rn_mul(Rd, jy));
}

// App. B: |grad b| at a <10> face (pairs); B(p, q) = b at origin + p normal + q tangent.
template <typename T, typename F> __device__ __forceinline__ V<T> appb_face2(F B, T ih) {
    const V<T> a1 = B(1, 1) - B(0, -1), a2 = B(0, 1) - B(1, -1);
    const V<T> b1 = B(2, 1) - B(-1, -1), b2 = B(-1, 1) - B(2, -1);
    const V<T> c1 = B(1, 2) - B(0, -2), c2 = B(0, 2) - B(1, -2);
    const V<T> dn = (bc<T>(T(35.0 / 48.0)) * (a1 - a2) - bc<T>(T(1.0 / 48.0)) * (b1 - b2) -
                     bc<T>(T(1.0 / 6.0)) * (c1 - c2)) * bc<T>(ih);
    const V<T> dt = (bc<T>(T(35.0 / 96.0)) * (a1 + a2) - bc<T>(T(1.0 / 32.0)) * (b1 + b2) -
                     bc<T>(T(1.0 / 24.0)) * (c1 + c2)) * bc<T>(ih);
    const V<T> m2 = fma(dn, dn, dt * dt);
    return mk(M<T>::sqrt_(m2.x()), M<T>::sqrt_(m2.y()));
}
// App. B: |grad b| at a corner; B(p, q) = b at origin + p x + q y.
template <typename T, typename F> __device__ __forceinline__ V<T> appb_corner2(F B, T ih) {
    const V<T> a1 = B(1, 1) - B(0, 0), a2 = B(0, 1) - B(1, 0);
    const V<T> b1 = B(2, 1) - B(-1, 0), b2 = B(-1, 1) - B(2, 0);
    const V<T> c1 = B(1, 2) - B(0, -1), c2 = B(0, 2) - B(1, -1);
    const V<T> dx = (bc<T>(T(5.0 / 8.0)) * (a1 - a2) - bc<T>(T(1.0 / 48.0)) * (b1 - b2) -
                     bc<T>(T(1.0 / 16.0)) * (c1 - c2)) * bc<T>(ih);
    const V<T> dy = (bc<T>(T(5.0 / 8.0)) * (a1 + a2) - bc<T>(T(1.0 / 16.0)) * (b1 + b2) -
                     bc<T>(T(1.0 / 48.0)) * (c1 + c2)) * bc<T>(ih);
    const V<T> m2 = fma(dx, dx, dy * dy);
    return mk(M<T>::sqrt_(m2.x()), M<T>::sqrt_(m2.y()));
}
// App. B magnitude m at a flux point raised to at least half of the two-point
// slope |d| s (s = 1 / |e|): the quotient slope / m, the unit normal's
// component along e, then stays within [-2, 2]; it leaves that range only
// where grad psi has no direction (reading R-A21G)
template <typename T> __device__ __forceinline__ V<T> appb_floor2(V<T> m, V<T> d, T s) {
    return mk(fmax(m.x(), T(0.5) * s * fabs(d.x())), fmax(m.y(), T(0.5) * s * fabs(d.y())));
}
// f / m per column with the guard on |grad psi| of the standard anti-trapping forms
template <typename T> __device__ __forceinline__ V<T> guarded_div2(V<T> f, V<T> m, T hh) {
    const V<T> q = f * rcp2(m);
    return mk(m.x() * m.x() * hh < Guard<T>::v ? T(0) : q.x(), m.y() * m.y() * hh < Guard<T>::v ? T(0) : q.y());
}

// ---------------------------------------------------------------------------
// compensated state (precision PF_F32C): psi and U carried as FP32 pairs
// hi + lo (about 48 significant bits) while the rates use FP32 arithmetic.
// Three places decide the accuracy of a step beyond the rounding of the
// rates: the state update, phi, and delta phi.
// ---------------------------------------------------------------------------
// (hi, lo) + d: Knuth's two-sum of hi and d, the rounding error folded into
// lo, renormalised by Dekker's fast two-sum (the _rn intrinsics are never
// contracted into FMAs, which would break the error-free transformations)
__device__ __forceinline__ void cadd(float hi, float lo, float d, float& ho, float& lo_o) {
    const float s = __fadd_rn(hi, d);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(d, bb));
    const float l = __fadd_rn(lo, e);
    ho = __fadd_rn(s, l);
    lo_o = __fsub_rn(l, __fsub_rn(ho, s));
}
template <typename T> __device__ __forceinline__ void cadd2(V<T> hi, V<T> lo, V<T> d, V<T>& ho, V<T>& lo_o) {
    float a, b, c, e;
    cadd((float)hi.x(), (float)lo.x(), (float)d.x(), a, b);
    cadd((float)hi.y(), (float)lo.y(), (float)d.y(), c, e);
    ho = mk(T(a), T(c));
    lo_o = mk(T(b), T(e));
}
// phi = tanh((hi + lo) / sqrt2) with the library tanh (a few ulp); the
// argument is rounded once
__device__ __forceinline__ float phi_acc(float hi, float lo) {
    const float c = 0.70710678118654752440f;
    return tanhf(fmaf(hi, c, lo * c));
}
// phi(psi + d) - phi(psi) = T (1 - phi^2) / (1 + T phi) with T = tanh(d / sqrt2),
// the addition theorem of tanh: the increment keeps its relative accuracy,
// unlike the difference phi' - phi of two rounded values
__device__ __forceinline__ float dphi_acc(float phi, float d) {
    const float T = tanhf(d * 0.70710678118654752440f);
    return div_nr(T * fmaf(-phi, phi, 1.0f), fmaf(T, phi, 1.0f));
}

// ---------------------------------------------------------------------------
// double-float arithmetic on packed FP32 pairs (Dekker's double-length
// arithmetic, 1971: values h + l with |l| <= ulp(h) / 2; error-free two-sum
// and the FMA two-product).  The compensated state evaluates the psi rate this
// way: its terms are O(1) while the rate must be accurate to ~1e-8 absolute
// (a per-step perturbation of psi at the interface is amplified ~1e4-fold
// over 1e4 steps of the free dendrite), beyond FP32's 2^-24.
// ---------------------------------------------------------------------------
struct D2 {
    V<float> h, l;
};
__device__ __forceinline__ D2 d2(V<float> h, V<float> l) { return D2{h, l}; }
__device__ __forceinline__ D2 d2f(V<float> h) { return D2{h, bc<float>(0.0f)}; }
__device__ __forceinline__ D2 d2c(float h, float l) { return D2{bc<float>(h), bc<float>(l)}; }
__device__ __forceinline__ V<float> vneg(V<float> a) { return a * bc<float>(-1.0f); }
// s + e = a + b exactly (Knuth)
__device__ __forceinline__ D2 two_sum(V<float> a, V<float> b) {
    const V<float> s = a + b;
    const V<float> bb = s - a;
    return D2{s, (a - (s - bb)) + (b - bb)};
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ D2 fast_two_sum(V<float> a, V<float> b) {
    const V<float> s = a + b;
    return D2{s, b - (s - a)};
}
// p + e = a b exactly
__device__ __forceinline__ D2 two_prod(V<float> a, V<float> b) {
    const V<float> p = a * b;
    return D2{p, fma(a, b, vneg(p))};
}
__device__ __forceinline__ D2 dadd(D2 x, D2 y) {
    const D2 s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, s.l + (x.l + y.l));
}
__device__ __forceinline__ D2 dsub(D2 x, D2 y) { return dadd(x, D2{vneg(y.h), vneg(y.l)}); }
__device__ __forceinline__ D2 dmul(D2 x, D2 y) {
    const D2 p = two_prod(x.h, y.h);
    return fast_two_sum(p.h, fma(x.h, y.l, fma(x.l, y.h, p.l)));
}
__device__ __forceinline__ D2 dscale(D2 x, float c) { return D2{x.h * bc<float>(c), x.l * bc<float>(c)}; }  // c a power of 2
__device__ __forceinline__ D2 ddiv(D2 x, D2 y) {
    const V<float> q1 = mk(div_nr(x.h.x(), y.h.x()), div_nr(x.h.y(), y.h.y()));
    const D2 r = dsub(x, dmul(d2f(q1), y));
    const V<float> q2 = mk(div_nr(r.h.x(), y.h.x()), div_nr(r.h.y(), y.h.y()));
    return fast_two_sum(q1, q2);
}
// (hi_a + lo_a) - (hi_b + lo_b) with the hi difference exact
__device__ __forceinline__ D2 ddiff(V<float> ha, V<float> la, V<float> hb, V<float> lb) {
    const D2 s = two_sum(ha, vneg(hb));
    return D2{s.h, s.l + (la - lb)};
}
// e^x for x <= 0 (|x| < 80) in double-float, relative error ~1e-11: Cody-Waite
// reduction x = k ln2 + r, |r| <= ln2 / 2 (ln2 = L1 + L2 + L3, k L1 exact),
// e^r by its Taylor series (r, r^2/2, r^3/6 in double-float, r^4/24 ..
// r^9/9! in FP32, each below 1e-3 of the sum), then the exact scaling 2^k.
__device__ __forceinline__ D2 dexp_neg(D2 x) {
    const float L1 = 0.693115234375f, L2 = 3.194618329871446e-05f, L3 = 1.6465717678215697e-12f;
    const float kx = rintf(x.h.x() * 1.4426950216293335f), ky = rintf(x.h.y() * 1.4426950216293335f);
    const V<float> k = mk(kx, ky);
    const D2 r0 = two_sum(fma(vneg(k), bc<float>(L1), x.h), vneg(k * bc<float>(L2)));
    const D2 r = fast_two_sum(r0.h, r0.l + (x.l - k * bc<float>(L3)));
    const D2 r2 = dmul(r, r);
    const D2 r3 = dmul(r2, r);
    const V<float> rh = r.h;
    V<float> t = fma(rh, bc<float>(1.0f / 362880.0f), bc<float>(1.0f / 40320.0f));
    t = fma(rh, t, bc<float>(1.0f / 5040.0f));
    t = fma(rh, t, bc<float>(1.0f / 720.0f));
    t = fma(rh, t, bc<float>(1.0f / 120.0f));
    t = fma(rh, t, bc<float>(1.0f / 24.0f));
    t = t * (r2.h * r2.h);
    D2 e = dadd(dmul(r3, d2c(0.1666666716337204f, -4.967053879312289e-09f)), d2f(t));
    e = dadd(e, dscale(r2, 0.5f));
    e = dadd(e, r);
    e = dadd(e, d2c(1.0f, 0.0f));
    const V<float> p2 = mk(__int_as_float(((int)kx + 127) << 23), __int_as_float(((int)ky + 127) << 23));
    return D2{e.h * p2, e.l * p2};
}

// |psi| beyond which the FP64 library tanh of psi / sqrt2 returns exactly
// +-1 (from |psi / sqrt2| ~ 19 on).  FP64 rows beyond it take phi = sign(psi)
// without the tanh, which is expensive at GB300's FP64 rate (+31% for the FP64
// sweep); the FP32 exp2/reciprocal form costs less than the warp vote.
template <typename T> struct Bulk;
template <> struct Bulk<double> { static constexpr double psi = 32.0; };

template <typename T> struct ConstOf;
template <> struct ConstOf<float> {
    static __device__ __forceinline__ const float* get(const InstRec& r) { return r.cf; }
};
template <> struct ConstOf<double> {
    static __device__ __forceinline__ const double* get(const InstRec& r) { return r.cd; }
};

template <typename T> struct Vec2;
template <> struct Vec2<float> { using t = float2; };
template <> struct Vec2<double> { using t = double2; };

// Column index of a ghost column: periodic wrap or cell-centred mirror.
__device__ __forceinline__ int col_idx(int c, int nx, bool per) {
    return per ? ((c % nx) + nx) % nx : mirror_idx(c, nx);
}
// One periodic period applied to a strip column (c in [-2, nx + 62)): the
// wrapped pair stays contiguous, so it keeps the vector load; columns still
// outside [0, nx) (grids narrower than a strip) take the scalar path.
__device__ __forceinline__ int wrap_once(int c, int nx, bool per) {
    return !per ? c : (c < 0 ? c + nx : (c >= nx ? c - nx : c));
}

// Load the pair (c, c+1) of a row; c is even.  Vector load when both columns
// are inside and the row is 2-element aligned, wrapped or mirrored scalar
// loads otherwise.
template <typename T>
__device__ __forceinline__ void load_pair(const T* __restrict__ row, int c, int nx, bool vec, bool per, T& a, T& b) {
    c = wrap_once(c, nx, per);
    if (vec && c >= 0 && c + 1 < nx) {
        const typename Vec2<T>::t v = __ldg(reinterpret_cast<const typename Vec2<T>::t*>(row + PF_CHK(c, nx - 1)));
        a = v.x;
        b = v.y;
    } else {
        a = __ldg(row + PF_CHK(col_idx(c, nx, per), nx));
        b = __ldg(row + PF_CHK(col_idx(c + 1, nx, per), nx));
    }
}
__device__ __forceinline__ void load_grain_pair(const int16_t* __restrict__ row, int c, int nx, bool vec, bool per,
                                                int& a, int& b) {
    c = wrap_once(c, nx, per);
    if (vec && c >= 0 && c + 1 < nx) {
        const int v = __ldg(reinterpret_cast<const int*>(row + PF_CHK(c, nx - 1)));
        a = (int)(int16_t)(v & 0xffff);
        b = (int)(int16_t)((unsigned)v >> 16);
    } else {
        a = __ldg(row + PF_CHK(col_idx(c, nx, per), nx));
        b = __ldg(row + PF_CHK(col_idx(c + 1, nx, per), nx));
    }
}
template <typename T>
__device__ __forceinline__ void store_pair(T* __restrict__ row, int c, int nx, bool vec, bool okL, bool okR, V<T> v) {
    if (vec && okL && okR) {
        typename Vec2<T>::t o;
        o.x = v.x();
        o.y = v.y();
        *reinterpret_cast<typename Vec2<T>::t*>(row + PF_CHK(c, nx - 1)) = o;
    } else {
        if (okL) row[PF_CHK(c, nx)] = v.x();
        if (okR) row[PF_CHK(c + 1, nx)] = v.y();
    }
}

// Blocks of PF_STEP2D_WPB warps (each warp works alone); FP32 kernels ask for
// PF_STEP2D_MIN_BLOCKS_F32 resident blocks per SM, which caps their registers.
// One-warp blocks with a 128-register cap (16 resident warps per SM) measured
// ~20 % faster than four-warp blocks at the same occupancy.
#ifndef PF_STEP2D_WPB
#define PF_STEP2D_WPB 1
#endif
#ifndef PF_STEP2D_MIN_BLOCKS_F32
#define PF_STEP2D_MIN_BLOCKS_F32 16
#endif
// The compensated kernel holds the lo rows as well.  Capped at 168 registers
// (eleven blocks asked for, twelve resident warps per SM) it spills ~100 bytes
// of rarely used values and runs 13 % faster than uncapped at 246 registers
// (eight warps): its dependency chains need the extra warps more than the
// registers.
#ifndef PF_STEP2D_MIN_BLOCKS_F32C
#define PF_STEP2D_MIN_BLOCKS_F32C 11
#endif

// VAR 0: isothermal instances with mirror walls at the T1 time level (the
// flags below are compile-time false and their code disappears); VAR 1 (DS):
// instances with a frozen temperature and/or periodic x, T1 or T0 read from
// the record; VAR 2: isothermal instances with mirror walls at the T0 time
// level, T0 fixed at compile time.  CMP = true (T = float, VAR 0): the
// compensated state of precision PF_F32C, the lo halves of psi and U stored
// right after the hi halves of each time level.  MODE (T0 time level only,
// VAR 1 or 2): 0 the fused step; 1 the psi pass of the two-kernel form of
// Sec. 3.3.1, which stores psi' and d psi/dt (InstRec::rate); 2 its U pass,
// which reads d psi/dt back instead of recomputing phase 1 (U' needs only
// psi^n, U^n and d psi/dt^n at the T0 level).
template <typename T, int S, int VAR, bool CMP, int MODE = 0>
__global__ void __launch_bounds__(32 * PF_STEP2D_WPB,
                                  sizeof(T) == 4 ? (CMP ? PF_STEP2D_MIN_BLOCKS_F32C : PF_STEP2D_MIN_BLOCKS_F32) : 1)
    k_step2d(const WorkItem* __restrict__ work, int n_work, const InstRec* __restrict__ recs, int launch_parity,
             StepClock clk) {
    constexpr bool ISO = (S == S21 || S == SBAR21);
    constexpr bool DS = VAR == 1;   // frozen temperature / periodic x, T0 from the record
    constexpr bool T0I = VAR == 2;  // isothermal, mirror walls, T0
    const int lane = threadIdx.x & 31;
    const int warps_per_block = blockDim.x >> 5;
    const int gw = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
    const int nw = gridDim.x * warps_per_block;
    const T SQ2 = T(1.41421356237309504880);

    for (int w = gw; w < n_work; w += nw) {
        const WorkItem wi = work[w];
        const InstRec& rec = recs[wi.inst];
        const int nx = rec.nx, ny = rec.ny;
        const int par = rec.parity_offset ^ launch_parity;
        const T* __restrict__ psi = static_cast<const T*>(rec.psi[par]);
        const T* __restrict__ Uf = static_cast<const T*>(rec.U[par]);
        T* __restrict__ psi_o = static_cast<T*>(rec.psi[par ^ 1]);
        T* __restrict__ U_o = static_cast<T*>(rec.U[par ^ 1]);
        // compensated state: the lo half of a level follows its hi half
        const size_t NN = (size_t)nx * ny;
        const T* __restrict__ psiL = psi + NN;
        const T* __restrict__ UfL = Uf + NN;
        T* __restrict__ psi_oL = psi_o + NN;
        T* __restrict__ U_oL = U_o + NN;
        T* __restrict__ rate_b = static_cast<T*>(rec.rate);  // d psi/dt of the two-kernel form
        const int16_t* __restrict__ grain = rec.grain;
        const T* __restrict__ rot = static_cast<const T*>(rec.rot);
        const T* cst = ConstOf<T>::get(rec);
        const T ih = cst[C_IH], hh = cst[C_HH], dt = cst[C_DT];
        const T i4h = cst[C_I4H], ih_half = cst[C_IH_HALF];
        const T kk = cst[C_K], omk = cst[C_OMK], eps = cst[C_EPS], lam = cst[C_LAM], Dc = cst[C_D];
        const T ih2 = cst[C_IH2], i6h2 = cst[C_I6H2], g10c = cst[C_G10], g01c = cst[C_G01];
        const T isq2dt = cst[C_ISQ2DT];
        const bool vec = (nx & 1) == 0;
        const bool per = DS && rec.bcx != 0;
        // every cell in grain 0 (warp-uniform): one crystal frame, no grain
        // rows to read and no grain-boundary faces to recompute
        const bool one = rec.one_grain != 0;
        const bool t0 = T0I || (DS && rec.tlevel != 0);  // T0 time level
        // frozen temperature: zeta at row p = zeta_y0 + (p - y0) zA (Eqs. Thermal_F1/_F2);
        // the DS variant applies it branch-free (zA = zB = zC = 0 gives zeta = 0, F1 = 1)
        T zeta_y0 = T(0), zA = T(0);
        if (DS) {
            const long long n = clk.clock ? clk.base[wi.inst] + *clk.clock : clk.step;
            zeta_y0 = (T)((double)wi.y0 * rec.zA - rec.zB - (double)n * rec.zC);
            zA = (T)rec.zA;
        }

        const int x0 = wi.x0, y0 = wi.y0;
        const int y1 = min(y0 + wi.ext, ny);
        const int cL = x0 - 2 + 2 * lane;
        const bool realL = cL >= 0 && cL < nx, realR = cL + 1 >= 0 && cL + 1 < nx;
        const bool outL = lane >= 1 && lane <= 30 && realL;
        const bool outR = lane >= 1 && lane <= 30 && realR;
        // warp holds mirror ghost columns (periodic ghosts are real cells, computed in place)
        const bool edge = !per && ((x0 - 2 < 0) || (x0 + 62 > nx));
        // lanes holding the mirror images of ghost columns (phase-1 copies)
        const int mL = mirror_idx(cL, nx), mR = mirror_idx(cL + 1, nx);
        const int srcL = (mL - (x0 - 2)) >> 1, srcR = (mR - (x0 - 2)) >> 1;
        const bool hiL = ((mL - (x0 - 2)) & 1) != 0, hiR = ((mR - (x0 - 2)) & 1) != 0;

        auto fetch_row = [&](const T* f, int vr, T& a, T& b) {
            load_pair<T>(f + (size_t)PF_CHK(mirror_idx(vr, ny), ny) * nx, cL, nx, vec, per, a, b);
        };
        auto make_row = [&](T a, T b, bool wide) {
            Row<T> row;
            row.l = a;
            row.r = b;
            row.m1 = shup(b);
            row.p1 = shdn(a);
            if (wide) {
                row.m2 = shup(a);
                row.p2 = shdn(b);
            } else {
                row.m2 = row.p2 = T(0);
            }
            return row;
        };
        // phi of a row; FP64: where |psi| exceeds the saturation bound on the
        // whole row of the warp, phi = sign(psi) exactly (what tanh returns),
        // taken without the tanh and, since the row's neighbours are already in
        // place, without the shuffles
        auto phi_row = [&](const Row<T>& p) {
            Row<T> o;
            if constexpr (sizeof(T) == 8) {
                const T B = Bulk<T>::psi;
                if (__all_sync(FULL, fabs(p.l) > B && fabs(p.r) > B)) {
                    o.l = p.l > T(0) ? T(1) : T(-1);
                    o.r = p.r > T(0) ? T(1) : T(-1);
                    o.m1 = p.m1 > T(0) ? T(1) : T(-1);
                    o.p1 = p.p1 > T(0) ? T(1) : T(-1);
                    o.m2 = o.p2 = T(0);
                    return o;
                }
            }
            o.l = M<T>::tanh_isq2(p.l);
            o.r = M<T>::tanh_isq2(p.r);
            o.m1 = shup(o.r);
            o.p1 = shdn(o.l);
            o.m2 = o.p2 = T(0);
            return o;
        };
        // compensated state: phi of the own columns from hi + lo
        auto phi_row_c = [&](const Row<T>& p, V<T> lo) {
            Row<T> o;
            o.l = (T)phi_acc((float)p.l, (float)lo.x());
            o.r = (T)phi_acc((float)p.r, (float)lo.y());
            o.m1 = shup(o.r);
            o.p1 = shdn(o.l);
            o.m2 = o.p2 = T(0);
            return o;
        };
        // delta phi row: ghost columns take their mirror cell's value (only in
        // warps that hold ghost columns), halo columns come from the neighbours
        auto dphi_row = [&](V<T> d) {
            Row<T> o;
            o.l = d.x();
            o.r = d.y();
            if (edge) {
                // a far ghost column (beyond nx + 1) gets an out-of-range source lane,
                // which the shuffle reduces modulo 32; its value reaches no output
                const T aL = __shfl_sync(FULL, d.x(), srcL), bL = __shfl_sync(FULL, d.y(), srcL);
                const T aR = __shfl_sync(FULL, d.x(), srcR), bR = __shfl_sync(FULL, d.y(), srcR);
                o.l = realL ? o.l : (hiL ? bL : aL);
                o.r = realR ? o.r : (hiR ? bR : aR);
            }
            o.m1 = shup(o.r);
            o.p1 = shdn(o.l);
            o.m2 = o.p2 = T(0);
            return o;
        };

        // crystal frames of the own columns, reloaded when the grain changes
        Rot2<T> RR;
        int cgL = -1, cgR = -1;
        auto set_rot = [&](int gL, int gR) {
            if (gL != cgL || gR != cgR) {
                const T* A = rot + 9 * PF_CHK(gL, rec.n_grains);
                const T* B = rot + 9 * PF_CHK(gR, rec.n_grains);
                RR.a = mk(__ldg(A + 0), __ldg(B + 0));
                RR.b = mk(__ldg(A + 1), __ldg(B + 1));
                RR.c = mk(__ldg(A + 3), __ldg(B + 3));
                RR.d = mk(__ldg(A + 4), __ldg(B + 4));
                cgL = gL;
                cgR = gR;
            }
        };

        // anisotropy y-face carry (face between rows p-1 and p, own columns)
        V<T> qy_c = bc<T>(T(0));
        int gyL_c = -1, gyR_c = -1;
        int prow_c = -100;
        if (one) set_rot(0, 0);

        // phase 1 at real row p (psi rows Pm = p-1, P0 = p, Pp = p+1), grains
        // gL, gR: returns psi' and phi' of the own columns and delta phi.
        // double-float constants of the compensated state's psi rate
        auto dfc = [&](double x) -> D2 {
            const float h = (float)x;
            return d2c(h, (float)(x - (double)h));
        };
        D2 kL = d2c(0.f, 0.f), kG1 = kL, kG2 = kL, kS2 = kL, kDT = kL, kA0 = kL;
        if constexpr (CMP) {
            const double hd = rec.h;
            kL = dfc(ISO ? 1.0 / (6.0 * hd * hd) : 1.0 / (hd * hd));
            kG1 = dfc(ISO ? 2.0 / 3.0 / (4.0 * hd * hd) : 0.25 / (hd * hd));
            kG2 = dfc(ISO ? 1.0 / 3.0 / (8.0 * hd * hd) : 0.0);
            kS2 = dfc(1.41421356237309504880);
            kDT = dfc(rec.dt);
            kA0 = dfc(1.0 - 3.0 * rec.eps4);
        }

        auto phase1 = [&](int p, const Row<T>& Pm, const Row<T>& P0, const Row<T>& Pp, const Row<T>& ph0,
                          const Row<T>& u0, int gL, int gR, const Row<T>& Lm, const Row<T>& L0, const Row<T>& Lp,
                          V<T> ulo0, V<T>& psin, V<T>& psin_lo, V<T>& phin, V<T>& dph, V<T>& rate_o,
                          V<T>& phc) {
            if constexpr (MODE == 2) {
                // U pass of the two-kernel form: d psi/dt^n from the psi pass,
                // T0 increment dt (1 - phi^2)/sqrt2 d psi/dt, phi^n on the left
                T ra, rb;
                load_pair<T>(rate_b + (size_t)PF_CHK(p, ny) * nx, cL, nx, vec, per, ra, rb);
                const V<T> ph = ph0.C();
                rate_o = mk(ra, rb);
                dph = bc<T>(dt * T(0.70710678118654752440)) * (bc<T>(T(1)) - ph * ph) * rate_o;
                phin = ph;
                phc = ph;
                psin = psin_lo = bc<T>(T(0));
                return;
            }
            if (!one) set_rot(gL, gR);
            const int gM = one ? 0 : shup(gR);  // grain of column L-1
            const V<T> W0 = P0.W(), C0 = P0.C(), E0 = P0.E();
            const V<T> Wm = Pm.W(), Cm = Pm.C(), Em = Pm.E();
            const V<T> Wp = Pp.W(), Cp = Pp.C(), Ep = Pp.E();
            // x+ faces: (L|R) in L's frame, (R|R+1) in R's frame
            // face fluxes of J - g (the compensated state: the cancellation-free form)
            auto aq2 = [&](V<T> gx, V<T> gy, bool xf) -> V<T> {
                if constexpr (CMP) return aniso_qn2c<T>(gx, gy, RR, eps, hh, xf);
                return aniso_qn2<T>(gx, gy, RR, eps, hh, xf);
            };
            auto aq1 = [&](T gx, T gy, T Ra, T Rb, T Rc, T Rd) -> T {
                if constexpr (CMP) return aniso_qn1c<T>(gx, gy, Ra, Rb, Rc, Rd, eps, hh, true);
                if constexpr (VAR != 0) return aniso_qn1_rn<T>(gx, gy, Ra, Rb, Rc, Rd, eps, hh, true);
                return aniso_qn1<T>(gx, gy, Ra, Rb, Rc, Rd, eps, hh, true);
            };
            const V<T> gxX = (E0 - C0) * bc<T>(ih), gyX = ((Ep + Cp) - (Em + Cm)) * bc<T>(i4h);
            const V<T> Xp = aq2(gxX, gyX, true);
            // x- faces: from the left column; recomputed across grain boundaries.
            // Lane 0 receives its own value: its column L (x0-2) feeds no output.
            T xmL = shup(Xp.y()), xmR = Xp.x();
            if (!one) {
                if (gM != gL)
                    xmL = aq1((P0.l - P0.m1) * ih, ((Pp.l + Pp.m1) - (Pm.l + Pm.m1)) * i4h, RR.a.x(), RR.b.x(),
                              RR.c.x(), RR.d.x());
                if (gR != gL) xmR = aq1(gxX.x(), gyX.x(), RR.a.y(), RR.b.y(), RR.c.y(), RR.d.y());
            }
            // y+ faces; y- faces carried from row p-1 when valid
            const V<T> Yp = aq2(((Ep + E0) - (Wp + W0)) * bc<T>(i4h), (Cp - C0) * bc<T>(ih), false);
            V<T> Ym = qy_c;
            const bool okL = prow_c == p && (one || gyL_c == gL), okR = prow_c == p && (one || gyR_c == gR);
            if (!(okL && okR)) {
                const V<T> Yc = aq2(((E0 + Em) - (W0 + Wm)) * bc<T>(i4h), (C0 - Cm) * bc<T>(ih), false);
                Ym = mk(okL ? Ym.x() : Yc.x(), okR ? Ym.y() : Yc.y());
            }
            qy_c = Yp;
            gyL_c = gL;
            gyR_c = gR;
            prow_c = p + 1;
            const V<T> N = ((Xp - mk(xmL, xmR)) + (Yp - Ym)) * bc<T>(ih);
            // Laplacian, gradient square, centred-gradient anisotropy
            const V<T> ex = E0 - W0, ey = Cp - Cm;
            V<T> L, G;
            if (ISO) {
                L = fma(bc<T>(T(4)), (W0 + E0) + (Cm + Cp), ((Wm + Em) + (Wp + Ep)) - bc<T>(T(20)) * C0) *
                    bc<T>(i6h2);
                const V<T> dp = Ep - Wm, dm = Em - Wp;
                G = fma(bc<T>(g10c), fma(ex, ex, ey * ey), bc<T>(g01c) * fma(dp, dp, dm * dm));
            } else {
                L = ((W0 + E0) + (Cm + Cp) - bc<T>(T(4)) * C0) * bc<T>(ih2);
                G = bc<T>(T(0.25) * ih2) * fma(ex, ex, ey * ey);
            }
            const V<T> ac = aniso_a2<T>(ex * bc<T>(ih_half), ey * bc<T>(ih_half), RR, eps, hh);
            const V<T> ph = ph0.C();
            V<T> u = u0.C();  // F2 of Eq. PF_a
            T iF1 = T(1);     // 1 / F1
            if (DS) {
                const T z = zeta_y0 + T(p - y0) * zA;
                u = u + bc<T>(z);
                iF1 = M<T>::rcp(T(1) - omk * z);
            }
            if constexpr (CMP) {
                // The rate in double-float: psi differences to the centre exact
                // (hi differences by two-sum plus the lo differences); L and G
                // from them; phi and 1 - phi^2 from e = exp(-sqrt2 |psi|) as
                // sign (1 - e) / (1 + e) and 4 e / (1 + e)^2; a_s = (1 - 3 eps)
                // + 4 eps q with the FP32 anisotropic part; U with its lo
                // half; the O(eps4) face terms N in FP32.  psi' = (hi + lo) +
                // dt rate kept exactly; delta phi from the addition theorem.
                const V<T> cl = L0.C();
                auto dd = [&](V<T> hn, V<T> ln) { return ddiff(hn, ln, C0, cl); };
                const D2 dW = dd(W0, L0.W()), dE = dd(E0, L0.E()), dS = dd(Cm, Lm.C()), dN = dd(Cp, Lp.C());
                const D2 faces = dadd(dadd(dW, dE), dadd(dS, dN));
                const D2 gx = dsub(dE, dW), gy = dsub(dN, dS);
                D2 Ld, Gd;
                if (ISO) {
                    const D2 dWm = dd(Wm, Lm.W()), dEm = dd(Em, Lm.E()), dWp = dd(Wp, Lp.W()), dEp = dd(Ep, Lp.E());
                    Ld = dmul(dadd(dscale(faces, 4.0f), dadd(dadd(dWm, dEm), dadd(dWp, dEp))), kL);
                    const D2 gp = dsub(dEp, dWm), gm = dsub(dEm, dWp);
                    Gd = dadd(dmul(dadd(dmul(gx, gx), dmul(gy, gy)), kG1), dmul(dadd(dmul(gp, gp), dmul(gm, gm)), kG2));
                } else {
                    Ld = dmul(faces, kL);
                    Gd = dmul(dadd(dmul(gx, gx), dmul(gy, gy)), kG1);
                }
                // |psi| (clamped at 40: e < 1e-24 there) and its sign
                const bool nL = C0.x() < T(0), nR = C0.y() < T(0);
                const bool cLx = fabsf(C0.x()) > 40.0f, cRx = fabsf(C0.y()) > 40.0f;
                const D2 ap = d2(mk(cLx ? 40.0f : fabsf(C0.x()), cRx ? 40.0f : fabsf(C0.y())),
                                 mk(cLx ? 0.0f : (nL ? -cl.x() : cl.x()), cRx ? 0.0f : (nR ? -cl.y() : cl.y())));
                const D2 e = dexp_neg(dmul(ap, D2{vneg(kS2.h), vneg(kS2.l)}));
                const D2 one = d2c(1.0f, 0.0f);
                const D2 ep1 = dadd(one, e);
                const D2 pa = ddiv(dsub(one, e), ep1);
                const D2 phd = d2(mk(nL ? -pa.h.x() : pa.h.x(), nR ? -pa.h.y() : pa.h.y()),
                                  mk(nL ? -pa.l.x() : pa.l.x(), nR ? -pa.l.y() : pa.l.y()));
                const D2 omp = ddiv(dscale(e, 4.0f), dmul(ep1, ep1));  // 1 - phi^2
                const D2 cpl = dmul(dmul(omp, d2f(bc<T>(lam))), d2(u, ulo0));
                const D2 srcd = dmul(dsub(phd, cpl), kS2);
                const V<T> w = aniso_w2<T>(ex * bc<T>(ih_half), ey * bc<T>(ih_half), RR, eps, hh);
                const D2 ad = dadd(kA0, d2f(w));
                const D2 E = dadd(dadd(Ld, d2f(N)), srcd);
                const D2 rate = dsub(ddiv(E, dmul(ad, ad)), dmul(dmul(phd, kS2), Gd));
                const D2 d = dmul(rate, kDT);
                const D2 s1 = two_sum(C0, d.h);
                const D2 s2 = fast_two_sum(s1.h, s1.l + (cl + d.l));
                psin = s2.h;
                psin_lo = s2.l;
                const V<T> phh = phd.h;
                dph = mk((T)dphi_acc((float)phh.x(), (float)d.h.x()), (T)dphi_acc((float)phh.y(), (float)d.h.y()));
                phin = phh + dph;
                rate_o = rate.h;
                phc = phh;  // phi^n of the own columns, rounded once from double-float
                return;
            }
            const V<T> src = bc<T>(SQ2) * (ph - bc<T>(lam) * (bc<T>(T(1)) - ph * ph) * u);
            V<T> rate = (L + N + src) * rcp2(ac * ac) - bc<T>(SQ2) * ph * G;
            if (DS) rate = rate * bc<T>(iF1);
            rate_o = rate;
            phc = ph;
            psin = fma(bc<T>(dt), rate, C0);
            psin_lo = L0.C();
            if constexpr (T0I) {
                // T0: chain-rule increment dt (1 - phi^2)/sqrt2 dpsi/dt and phi^n on the
                // left-hand side; phi' is not needed
                dph = bc<T>(dt * T(0.70710678118654752440)) * (bc<T>(T(1)) - ph * ph) * rate;
                phin = ph;
                return;
            }
            if constexpr (sizeof(T) == 8) {
                const T B = Bulk<T>::psi;
                if (__all_sync(FULL, fabs(psin.x()) > B && fabs(psin.y()) > B))
                    phin = mk(psin.x() > T(0) ? T(1) : T(-1), psin.y() > T(0) ? T(1) : T(-1));
                else
                    phin = mk(M<T>::tanh_isq2(psin.x()), M<T>::tanh_isq2(psin.y()));
            } else {
                phin = mk(M<T>::tanh_isq2(psin.x()), M<T>::tanh_isq2(psin.y()));
            }
            dph = phin - ph;
            if (DS) {
                // T0: chain-rule increment dt (1 - phi^2)/sqrt2 dpsi/dt and phi^n on the left-hand side
                const V<T> d0 = bc<T>(dt * T(0.70710678118654752440)) * (bc<T>(T(1)) - ph * ph) * rate;
                dph = mk(t0 ? d0.x() : dph.x(), t0 ? d0.y() : dph.y());
                phin = mk(t0 ? ph.x() : phin.x(), t0 ? ph.y() : phin.y());
            }
        };

        // phase-2 carries: fluxes of row q-1 that row q uses (subtracted)
        V<T> cFYm_D = bc<T>(T(0)), cFYm_A = bc<T>(T(0));
        V<T> cFDmm_D = bc<T>(T(0)), cFDmm_A = bc<T>(T(0));
        V<T> cFDpm_D = bc<T>(T(0)), cFDpm_A = bc<T>(T(0));
        V<T> cK_D = bc<T>(T(0)), cK_A = bc<T>(T(0));

        // Phase-2 fluxes at row q: alpha rows q (a*0), q+1 (a*1); U rows q,
        // q+1; psi rows q-2 .. q+2 (Pq[0..4]).  Returns the eight-flux sums of
        // the own columns (x 6 h^2 for the D~_{2,1} forms, x h^2 for S_{1,0})
        // and updates the carries.  need_x = false skips S_{2,1}'s x-face
        // magnitudes, which would read row q-2.
        // skipA (warp-uniform): delta phi is exactly 0 on the rows q-1 .. q+1 of
        // the whole warp (bulk liquid or solid, where phi = +-1 exactly), so
        // every anti-trapping flux these rows form or carry is exactly 0: sA = 0
        // and the anti-trapping carries are 0, as the full evaluation gives.
        auto fluxes = [&](const Row<T>& aD0, const Row<T>& aD1, const Row<T>& aA0, const Row<T>& aA1,
                          const Row<T>& bU0, const Row<T>& bU1, const Row<T>& bL0, const Row<T>& bL1, const Row<T>* Pq,
                          bool need_x, bool skipA, V<T>& sD, V<T>& sA) {
            const Row<T>& b0 = Pq[2];
            const Row<T>& b1 = Pq[3];
            // differences of U; the compensated state adds those of the lo halves
            auto dU = [&](V<T> hi_diff, V<T> lo_diff) -> V<T> {
                if constexpr (CMP) return hi_diff + lo_diff;
                return hi_diff;
            };
            if (S == S10) {
                const V<T> half = bc<T>(T(0.5));
                const V<T> fxD = half * (aD0.C() + aD0.E()) * dU(bU0.E() - bU0.C(), bL0.E() - bL0.C());
                const V<T> fyD = half * (aD0.C() + aD1.C()) * dU(bU1.C() - bU0.C(), bL1.C() - bL0.C());
                sD = (fxD - mk(shup(fxD.y()), fxD.x())) + (fyD - cFYm_D);
                cFYm_D = fyD;
                if (skipA) {
                    sA = bc<T>(T(0));
                    cFYm_A = bc<T>(T(0));
                    return;
                }
                const Row<T>& bm = Pq[1];
                const V<T> dxp = b0.E() - b0.C(), dyp = b1.C() - b0.C();
                const V<T> gx = dxp * bc<T>(ih), gy = ((b1.E() + b1.C()) - (bm.E() + bm.C())) * bc<T>(i4h);
                const V<T> yx = ((b1.E() + b0.E()) - (b1.W() + b0.W())) * bc<T>(i4h), yy = dyp * bc<T>(ih);
                const V<T> mx = fma(gx, gx, gy * gy), my = fma(yx, yx, yy * yy);
                const V<T> fxA = guarded_div2<T>(half * (aA0.C() + aA0.E()) * dxp,
                                                 mk(M<T>::sqrt_(mx.x()), M<T>::sqrt_(mx.y())), hh);
                const V<T> fyA = guarded_div2<T>(half * (aA0.C() + aA1.C()) * dyp,
                                                 mk(M<T>::sqrt_(my.x()), M<T>::sqrt_(my.y())), hh);
                sA = (fxA - mk(shup(fxA.y()), fxA.x())) + (fyA - cFYm_A);
                cFYm_A = fyA;
                return;
            }
            const V<T> q4 = bc<T>(T(0.25));
            // corner means: the (+1/2, +1/2) corners of (L, R) and of (L-1, L)
            const V<T> KC_D = q4 * ((aD0.C() + aD0.E()) + (aD1.C() + aD1.E()));
            const V<T> KW_D = q4 * ((aD0.W() + aD0.C()) + (aD1.W() + aD1.C()));
            // <10> faces x+, y+ (weight sums of Eq. flux_10) and <11> corners ++, -+
            const V<T> u0c = bU0.C(), l0c = bL0.C();
            const V<T> FXpD = ((aD0.C() + aD0.E()) + (KC_D + cK_D)) * dU(bU0.E() - u0c, bL0.E() - l0c);
            const V<T> FYpD = ((aD0.C() + aD1.C()) + (KC_D + KW_D)) * dU(bU1.C() - u0c, bL1.C() - l0c);
            const V<T> FPPD = KC_D * dU(bU1.E() - u0c, bL1.E() - l0c), FMPD = KW_D * dU(bU1.W() - u0c, bL1.W() - l0c);
            sD = ((FXpD - mk(shup(FXpD.y()), FXpD.x())) + (FYpD - cFYm_D)) + ((FPPD + FMPD) - (cFDmm_D + cFDpm_D));
            // carries for row q+1: its y- face is this y+ face, its (-1/2,-1/2)
            // corner the (+1/2,+1/2) corner of the column to the left, its
            // (+1/2,-1/2) corner the (-1/2,+1/2) corner of the column to the right
            cFYm_D = FYpD;
            cFDmm_D = mk(shup(FPPD.y()), FPPD.x());
            cFDpm_D = mk(FMPD.y(), shdn(FMPD.x()));
            cK_D = KC_D;
            if (skipA) {
                sA = bc<T>(T(0));
                cFYm_A = cFDmm_A = cFDpm_A = cK_A = bc<T>(T(0));
                return;
            }
            const V<T> KC_A = q4 * ((aA0.C() + aA0.E()) + (aA1.C() + aA1.E()));
            const V<T> KW_A = q4 * ((aA0.W() + aA0.C()) + (aA1.W() + aA1.C()));
            const V<T> p0c = b0.C();
            V<T> FXpA = ((aA0.C() + aA0.E()) + (KC_A + cK_A)) * (b0.E() - p0c);
            V<T> FYpA = ((aA0.C() + aA1.C()) + (KC_A + KW_A)) * (b1.C() - p0c);
            V<T> FPPA = KC_A * (b1.E() - p0c), FMPA = KW_A * (b1.W() - p0c);
            if (S == S21) {
                // App. B: each anti-trapping flux divided by |grad psi| at its point;
                // ps(dx, dy) = psi at columns (L + dx, R + dx), row q + dy
                auto ps = [&](int dx, int dy) -> V<T> { return Pq[2 + dy].pat(dx); };
                const T ihd = ih * T(0.70710678118654752440);  // 1 / |e| of the <11> fluxes
                if (need_x)
                    FXpA = guarded_div2<T>(
                        FXpA, appb_floor2<T>(appb_face2<T>([&](int p, int t) { return ps(p, t); }, ih), b0.E() - p0c, ih),
                        hh);
                FYpA = guarded_div2<T>(
                    FYpA, appb_floor2<T>(appb_face2<T>([&](int p, int t) { return ps(t, p); }, ih), b1.C() - p0c, ih), hh);
                FPPA = guarded_div2<T>(
                    FPPA, appb_floor2<T>(appb_corner2<T>([&](int p, int t) { return ps(p, t); }, ih), b1.E() - p0c, ihd),
                    hh);
                FMPA = guarded_div2<T>(
                    FMPA,
                    appb_floor2<T>(appb_corner2<T>([&](int p, int t) { return ps(p - 1, t); }, ih), b1.W() - p0c, ihd),
                    hh);
            }
            sA = ((FXpA - mk(shup(FXpA.y()), FXpA.x())) + (FYpA - cFYm_A)) + ((FPPA + FMPA) - (cFDmm_A + cFDpm_A));
            cFYm_A = FYpA;
            cFDmm_A = mk(shup(FPPA.y()), FPPA.x());
            cFDpm_A = mk(FMPA.y(), shdn(FMPA.x()));
            cK_A = KC_A;
        };
        // delta phi row exactly 0 over the whole warp (see skipA)
        auto zero_row = [&](const Row<T>& d) -> bool {
            return __all_sync(FULL, d.l == T(0) && d.r == T(0));
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
        Row<T> P[5];      // psi rows r-2 .. r+2 (iteration r)
        Row<T> PH1, UU0, UU1, DP0;
        Row<T> AD0, AA0;  // alpha rows of row r
        Row<T> UL0, UL1;  // compensated state: lo halves of U rows r, r+1
        Row<T> LP[3];     // compensated state: lo halves of psi rows r .. r+2
        bool zA_prev = false, zA0 = false;  // delta phi rows r-1, r exactly 0 over the warp
        V<T> phin_cur;    // phi' at row r
        auto psi_store = [&](int row, V<T> hi, V<T> lo, V<T> rt) {
            if constexpr (MODE == 2) return;  // the U pass leaves psi' to the psi pass
            store_pair<T>(psi_o + (size_t)PF_CHK(row, ny) * nx, cL, nx, vec, outL, outR, hi);
            if constexpr (CMP) store_pair<T>(psi_oL + (size_t)PF_CHK(row, ny) * nx, cL, nx, vec, outL, outR, lo);
            if constexpr (MODE == 1) store_pair<T>(rate_b + (size_t)PF_CHK(row, ny) * nx, cL, nx, vec, outL, outR, rt);
        };
        {
            // psi rows y0-3 .. y0+1 (row y0-3 is read only by S_{2,1}'s x-face
            // magnitudes, which the prologue skips)
            T a, b;
            for (int i = 1; i <= 4; ++i) {
                fetch_row(psi, y0 - 3 + i, a, b);
                P[i] = make_row(a, b, S == S21);
            }
            P[0] = P[1];
            // compensated state: psi lo rows y0-2 .. y0+1, U lo rows y0-1, y0
            Row<T> lq[4];
            Row<T> ulm = make_row(T(0), T(0), false), ul0 = ulm;
            for (int i = 0; i < 4; ++i) lq[i] = ulm;
            if constexpr (CMP) {
                for (int i = 0; i < 4; ++i) {
                    fetch_row(psiL, y0 - 2 + i, a, b);
                    lq[i] = make_row(a, b, false);
                }
                fetch_row(UfL, y0 - 1, a, b);
                ulm = make_row(a, b, false);
                fetch_row(UfL, y0, a, b);
                ul0 = make_row(a, b, false);
            }
            const Row<T> phm = CMP ? phi_row_c(P[2], lq[1].C()) : phi_row(P[2]);
            const Row<T> ph0 = CMP ? phi_row_c(P[3], lq[2].C()) : phi_row(P[3]);
            fetch_row(Uf, y0 - 1, a, b);
            const Row<T> um = make_row(a, b, false);
            fetch_row(Uf, y0, a, b);
            const Row<T> u0 = make_row(a, b, false);
            // phase 1 at rows y0-1 and y0; the ghost row -1 copies row 0 (the
            // psi pass of the two-kernel form needs no row y0-1: no U fluxes)
            int gL, gR;
            V<T> psn, psnl, fn, dm = bc<T>(T(0)), d0, rt, phc_unused;
            const bool ghost = (y0 - 1) < 0;
            gL = gR = 0;
            if (!ghost && MODE != 1) {
                if (!one) load_grain_pair(grain + (size_t)PF_CHK((y0 - 1), ny) * nx, cL, nx, vec, per, gL, gR);
                phase1(y0 - 1, P[1], P[2], P[3], phm, um, gL, gR, lq[0], lq[1], lq[2], ulm.C(), psn, psnl, fn, dm, rt,
                       phc_unused);
            }
            if (!one) load_grain_pair(grain + (size_t)PF_CHK(y0, ny) * nx, cL, nx, vec, per, gL, gR);
            phase1(y0, P[2], P[3], P[4], ph0, u0, gL, gR, lq[1], lq[2], lq[3], ul0.C(), psn, psnl, fn, d0, rt,
                   phc_unused);
            if (ghost) dm = d0;
            phin_cur = fn;
            if (y0 < y1) psi_store(y0, psn, psnl, rt);
            const Row<T> dmr = dphi_row(dm), d0r = dphi_row(d0);
            // phase-2 fluxes at row y0-1 (carries only); psi rows y0-3 .. y0+1
            const Row<T> aDm = alphaD(phm), aAm = alphaA(um, dmr);
            AD0 = alphaD(ph0);
            AA0 = alphaA(u0, d0r);
            V<T> s0, s1;
            zA_prev = zero_row(dmr);
            zA0 = zero_row(d0r);
            if constexpr (MODE != 1) fluxes(aDm, AD0, aAm, AA0, um, u0, ulm, ul0, P, false, zA_prev && zA0, s0, s1);
            P[0] = P[1];
            P[1] = P[2];
            P[2] = P[3];
            P[3] = P[4];
            UU0 = u0;
            UL0 = ul0;
            LP[0] = lq[2];
            LP[1] = lq[3];
            DP0 = d0r;
        }

        // prefetch psi row y0+2 and U, grain row y0+1 (compensated state: the
        // lo halves of psi and U of row y0+1)
        T nPa, nPb, nUa, nUb, nPLa = T(0), nPLb = T(0), nULa = T(0), nULb = T(0);
        int nGa = 0, nGb = 0;
        fetch_row(psi, y0 + 2, nPa, nPb);
        fetch_row(Uf, y0 + 1, nUa, nUb);
        if constexpr (CMP) {
            fetch_row(psiL, y0 + 2, nPLa, nPLb);
            fetch_row(UfL, y0 + 1, nULa, nULb);
        }
        if (!one && y0 + 1 < ny) load_grain_pair(grain + (size_t)PF_CHK((y0 + 1), ny) * nx, cL, nx, vec, per, nGa, nGb);

        // ---------------- sweep ----------------
        for (int r = y0; r < y1; ++r) {
            P[4] = make_row(nPa, nPb, S == S21);
            UU1 = make_row(nUa, nUb, false);
            if constexpr (CMP) {
                LP[2] = make_row(nPLa, nPLb, false);
                UL1 = make_row(nULa, nULb, false);
            }
            // phi of row r+1 (the compensated state takes it from phase 1,
            // which forms it in double-float, below)
            if constexpr (!CMP) PH1 = phi_row(P[3]);
            const int gL = nGa, gR = nGb;
            fetch_row(psi, r + 3, nPa, nPb);
            fetch_row(Uf, r + 2, nUa, nUb);
            if constexpr (CMP) {
                fetch_row(psiL, r + 3, nPLa, nPLb);
                fetch_row(UfL, r + 2, nULa, nULb);
            }
            if (!one && r + 2 < ny) load_grain_pair(grain + (size_t)PF_CHK((r + 2), ny) * nx, cL, nx, vec, per, nGa, nGb);

            // phase 1 at row r+1 (the psi pass of the two-kernel form: only
            // rows it stores)
            V<T> phn = bc<T>(T(0));
            Row<T> DP1;
            if (r + 1 < ny && (MODE != 1 || r + 1 < y1)) {
                V<T> psn, psnl, d, rt, phc;
                phase1(r + 1, P[2], P[3], P[4], PH1, UU1, gL, gR, LP[0], LP[1], LP[2], UL1.C(), psn, psnl, phn, d,
                       rt, phc);
                if (r + 1 < y1) psi_store(r + 1, psn, psnl, rt);
                DP1 = dphi_row(d);
                if constexpr (CMP) {
                    PH1.l = phc.x();
                    PH1.r = phc.y();
                    PH1.m1 = shup(PH1.r);
                    PH1.p1 = shdn(PH1.l);
                    PH1.m2 = PH1.p2 = T(0);
                }
            } else {
                if constexpr (CMP) PH1 = phi_row_c(P[3], LP[1].C());
                DP1 = DP0;  // ghost row ny mirrors row ny-1 = r
            }
            if constexpr (MODE == 1) {
                P[0] = P[1];
                P[1] = P[2];
                P[2] = P[3];
                P[3] = P[4];
                UU0 = UU1;
                continue;
            }

            // phase 2 at row r
            const bool zA1 = zero_row(DP1);
            const bool skipA = zA_prev && zA0 && zA1;
            const Row<T> AD1 = alphaD(PH1), AA1 = alphaA(UU1, DP1);
            {
                V<T> sD, sA;
                fluxes(AD0, AD1, AA0, AA1, UU0, UU1, UL0, UL1, P, true, skipA, sD, sA);
                const T cs = (S == S10) ? ih2 : i6h2;
                const V<T> u = UU0.C();
                const V<T> num =
                    fma(bc<T>(dt * cs), fma(bc<T>(Dc), sD, sA), fma(bc<T>(omk), u, bc<T>(T(1))) * DP0.C());
                if constexpr (CMP) {
                    // U' = (hi + lo) + num / (1 + k - (1-k) phi'), kept exactly
                    const V<T> den = fma(bc<T>(-omk), phin_cur, bc<T>(T(1) + kk));
                    const V<T> inc = mk((T)div_nr((float)num.x(), (float)den.x()),
                                        (T)div_nr((float)num.y(), (float)den.y()));
                    V<T> uh, ul;
                    cadd2<T>(u, UL0.C(), inc, uh, ul);
                    store_pair<T>(U_o + (size_t)PF_CHK(r, ny) * nx, cL, nx, vec, outL, outR, uh);
                    store_pair<T>(U_oL + (size_t)PF_CHK(r, ny) * nx, cL, nx, vec, outL, outR, ul);
                } else {
                    const V<T> un = fma(num, rcp2(fma(bc<T>(-omk), phin_cur, bc<T>(T(1) + kk))), u);
                    store_pair<T>(U_o + (size_t)PF_CHK(r, ny) * nx, cL, nx, vec, outL, outR, un);
                }
            }
            phin_cur = phn;
            P[0] = P[1];
            P[1] = P[2];
            P[2] = P[3];
            P[3] = P[4];
            UU0 = UU1;
            if constexpr (CMP) {
                UL0 = UL1;
                LP[0] = LP[1];
                LP[1] = LP[2];
            }
            DP0 = DP1;
            AD0 = AD1;
            AA0 = AA1;
            zA_prev = zA0;
            zA0 = zA1;
        }
    }
}

constexpr int WARPS_PER_BLOCK = PF_STEP2D_WPB;

template <typename T, int S>
bool launch_one(int grid_warps, cudaStream_t st, const WorkItem* work, int n_work, const InstRec* recs, int lp,
                StepClock clk, int var, int mode) {
    const int blocks = (grid_warps + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    const int th = 32 * WARPS_PER_BLOCK;
    if (var < 0 || var > 2) return false;
    if (mode != 0 && var == 0) return false;  // the two-kernel form runs at the T0 level (variant 1 or 2)
    if (mode == 1) {
        if (var == 2) k_step2d<T, S, 2, false, 1><<<blocks, th, 0, st>>>(work, n_work, recs, lp, clk);
        else k_step2d<T, S, 1, false, 1><<<blocks, th, 0, st>>>(work, n_work, recs, lp, clk);
    } else if (mode == 2) {
        if (var == 2) k_step2d<T, S, 2, false, 2><<<blocks, th, 0, st>>>(work, n_work, recs, lp, clk);
        else k_step2d<T, S, 1, false, 2><<<blocks, th, 0, st>>>(work, n_work, recs, lp, clk);
    } else if (var == 2) {
        k_step2d<T, S, 2, false><<<blocks, th, 0, st>>>(work, n_work, recs, lp, clk);
    } else if (var == 1) {
        k_step2d<T, S, 1, false><<<blocks, th, 0, st>>>(work, n_work, recs, lp, clk);
    } else {
        k_step2d<T, S, 0, false><<<blocks, th, 0, st>>>(work, n_work, recs, lp, clk);
    }
    return true;
}
// compensated state (isothermal, mirror walls, T1 only)
template <int S>
bool launch_cmp(int grid_warps, cudaStream_t st, const WorkItem* work, int n_work, const InstRec* recs, int lp,
                StepClock clk, int var) {
    if (var != 0) return false;
    const int blocks = (grid_warps + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    k_step2d<float, S, 0, true><<<blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(work, n_work, recs, lp, clk);
    return true;
}

template <typename T, int S> int occ_one(int var, int mode) {
    int n = 0;
    if (var < 0 || var > 2 || (mode != 0 && var == 0)) return 0;
    const int th = 32 * WARPS_PER_BLOCK;
    cudaError_t e;
    if (mode == 1)
        e = var == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2d<T, S, 2, false, 1>, th, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2d<T, S, 1, false, 1>, th, 0);
    else if (mode == 2)
        e = var == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2d<T, S, 2, false, 2>, th, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2d<T, S, 1, false, 2>, th, 0);
    else if (var == 2)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2d<T, S, 2, false>, th, 0);
    else if (var == 1)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2d<T, S, 1, false>, th, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2d<T, S, 0, false>, th, 0);
    return e == cudaSuccess ? n * WARPS_PER_BLOCK : 0;
}
template <int S> int occ_cmp(int var) {
    if (var != 0) return 0;
    int n = 0;
    const cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2d<float, S, 0, true>, 32 * WARPS_PER_BLOCK, 0);
    return e == cudaSuccess ? n * WARPS_PER_BLOCK : 0;
}

}  // namespace

PF_BOUNDS_READER(bounds_step2d)

// The 2D kernel is warp-granular: `bx` must be 64 (columns a warp holds) and
// `grid` counts warps.
bool launch_step2d(int prec, int scheme, int bx, int grid, cudaStream_t st, const WorkItem* work, int n_work,
                   const InstRec* recs, int lp, StepClock clk, int var, int mode) {
    if (bx != WARP_COLS) return false;
    if (prec == 0) {
        switch (scheme) {
            case S10: return launch_one<float, S10>(grid, st, work, n_work, recs, lp, clk, var, mode);
            case S21: return launch_one<float, S21>(grid, st, work, n_work, recs, lp, clk, var, mode);
            case SBAR21: return launch_one<float, SBAR21>(grid, st, work, n_work, recs, lp, clk, var, mode);
        }
    } else if (prec == 2) {
        if (mode != 0) return false;
        switch (scheme) {
            case S10: return launch_cmp<S10>(grid, st, work, n_work, recs, lp, clk, var);
            case S21: return launch_cmp<S21>(grid, st, work, n_work, recs, lp, clk, var);
            case SBAR21: return launch_cmp<SBAR21>(grid, st, work, n_work, recs, lp, clk, var);
        }
    } else {
        switch (scheme) {
            case S10: return launch_one<double, S10>(grid, st, work, n_work, recs, lp, clk, var, mode);
            case S21: return launch_one<double, S21>(grid, st, work, n_work, recs, lp, clk, var, mode);
            case SBAR21: return launch_one<double, SBAR21>(grid, st, work, n_work, recs, lp, clk, var, mode);
        }
    }
    return false;
}

// Warps of the fused kernel (mode 0) or of a pass of the two-kernel form
// resident on one SM (0 if not compiled).
int occupancy_step2d(int prec, int scheme, int bx, int var, int mode) {
    if (bx != WARP_COLS) return 0;
    if (prec == 0) {
        switch (scheme) {
            case S10: return occ_one<float, S10>(var, mode);
            case S21: return occ_one<float, S21>(var, mode);
            case SBAR21: return occ_one<float, SBAR21>(var, mode);
        }
    } else if (prec == 2) {
        if (mode != 0) return 0;
        switch (scheme) {
            case S10: return occ_cmp<S10>(var);
            case S21: return occ_cmp<S21>(var);
            case SBAR21: return occ_cmp<SBAR21>(var);
        }
    } else {
        switch (scheme) {
            case S10: return occ_one<double, S10>(var, mode);
            case S21: return occ_one<double, S21>(var, mode);
            case SBAR21: return occ_one<double, SBAR21>(var, mode);
        }
    }
    return 0;
}

}  // namespace pf
