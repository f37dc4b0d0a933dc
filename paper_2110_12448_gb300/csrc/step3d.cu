// step3d.cu -- fused explicit time step of the quantitative alloy phase-field
// model in 3D for sm_103a (arXiv:2110.12448, Sec. 5-6, Eqs. PF_a and PF_b).
//
// 2.5D blocking: a block owns a TX x TY column of cells and sweeps it along z
// with shared-memory plane rings (psi with a 2-cell halo in x and y, phi, U and
// delta phi on the 1-cell ring).  Global loads are issued one plane ahead into
// registers, and each thread keeps the crystal frame of its phase-1 cell in
// registers until the cell's grain changes.  Iteration z:
//   store psi plane z+2 (and phi on the ring region), U plane z+1 into the
//     rings; fetch psi plane z+3, U and grain plane z+2
//   phase 1 at plane z+1 on the (TX+2) x (TY+2) ring region: d psi/dt, psi',
//     phi', delta phi; ring cells outside the domain take their mirror cell's
//     values (the thread computes the mirror cell)
//   phase 2 at plane z on the TX x TY outputs: U'
// Each cell of psi and U is read from HBM once per step by the column that
// owns it (halo reads hit L2) and psi', U' are written once.
//
// Schemes: S-bar_{1,2,0}: L_{1,2,0} = 1/3 L_{1,0,0} + 2/3 L_{0,1,0} (Eqs.
// 3D_L100, 3D_L110), G_{1,2,0} (Eqs. Grad_100, Grad_110), D~_{1,2,0} (Eqs.
// divergence_100, divergence_110 with the alpha averages of Sec. 5.2) for D
// and the approximated anti-trapping (Eq. Anti_approx).  S_{1,0,0}: the <100>
// shell with a two-point face mean for D and the standard anti-trapping
// normalised by the face gradient.  Anisotropy: div(J - grad psi) over the
// six <100> faces in the cell's crystal frame (cubic a_s of Eq.
// anis_function), a_s^2 from the centred gradient.
#include "pf_internal.cuh"

namespace pf {
namespace {

template <typename T> struct M3;
template <> struct M3<float> {
    static __device__ __forceinline__ float tanh_(float x) {
        return 1.0f - __fdividef(2.0f, 1.0f + __expf(2.0f * x));
    }
    static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
    // single-instruction approximate square root (0 at 0) for the <100>
    // anti-trapping magnitude; the flux is guarded where |grad psi| vanishes
    static __device__ __forceinline__ float sqrt_(float x) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
};
template <> struct M3<double> {
    // tanh is exactly +-1 beyond |x| = 22.6 (|psi| = 32); the FP64 library
    // tanh is expensive at GB300's FP64 rate, and most cells are that far
    static __device__ __forceinline__ double tanh_(double x) { return fabs(x) > 22.6 ? copysign(1.0, x) : tanh(x); }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
};

// Component `ax` of (J - g) for a lab-frame face gradient g, crystal frame R
// (row-major crystal -> lab).  a_s = 1 - 3 eps + 4 eps sum n'^4, J = d(a_s^2
// |g|^2 / 2)/dg; see the 2D kernel for the algebra.
template <typename T>
__device__ __forceinline__ T aniso_q3(const T g[3], const T R[9], T eps, T hh, int ax) {
    T c[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) c[p] = R[p] * g[0] + R[3 + p] * g[1] + R[6 + p] * g[2];
    const T r2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    // evaluated unconditionally and selected at the end (no divergent branch)
    const bool guard = r2 * hh < Guard<T>::v;
    const T inv = M3<T>::rcp(guard ? T(1) : r2);
    T s[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) s[p] = c[p] * c[p] * inv;
    const T q = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
    const T a = T(1) - T(3) * eps + T(4) * eps * q;
    const T c1 = T(16) * eps * a;
    const T c0 = a * a - T(1) - c1 * q;
    T out = T(0);
#pragma unroll
    for (int p = 0; p < 3; ++p) out += R[3 * ax + p] * (c[p] * (c0 + c1 * s[p]));
    return guard ? T(0) : out;
}
template <typename T> __device__ __forceinline__ T aniso_a3(const T g[3], const T R[9], T eps, T hh) {
    T c[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) c[p] = R[p] * g[0] + R[3 + p] * g[1] + R[6 + p] * g[2];
    const T r2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    const bool guard = r2 * hh < Guard<T>::v;
    const T inv = M3<T>::rcp(guard ? T(1) : r2);
    T q = T(0);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const T s = c[p] * c[p] * inv;
        q += s * s;
    }
    return guard ? T(1) : T(1) - T(3) * eps + T(4) * eps * q;
}

// The D~ fluxes of the D term (alpha = 1 - phi, beta = U) and of the
// approximated anti-trapping term (alpha from delta phi, beta = psi) share
// their stencils and weights, so S-bar_{1,2,0} evaluates them as one pair
// (D, A): packed FP32x2 arithmetic in FP32, two scalars in FP64.
template <typename T> struct P2;
template <> struct P2<float> {
    float2 v;
    __device__ __forceinline__ float d() const { return v.x; }
    __device__ __forceinline__ float a() const { return v.y; }
};
template <> struct P2<double> {
    double x, y;
    __device__ __forceinline__ double d() const { return x; }
    __device__ __forceinline__ double a() const { return y; }
};
__device__ __forceinline__ P2<float> p2(float d, float a) {
    P2<float> r;
    r.v = make_float2(d, a);
    return r;
}
__device__ __forceinline__ P2<double> p2(double d, double a) {
    P2<double> r;
    r.x = d;
    r.y = a;
    return r;
}
__device__ __forceinline__ P2<float> operator+(P2<float> a, P2<float> b) {
    P2<float> r;
    r.v = __fadd2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ P2<float> operator-(P2<float> a, P2<float> b) {
    P2<float> r;
    r.v = __ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v);  // exactly a - b
    return r;
}
__device__ __forceinline__ P2<float> operator*(P2<float> a, P2<float> b) {
    P2<float> r;
    r.v = __fmul2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ P2<double> operator+(P2<double> a, P2<double> b) { return p2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ P2<double> operator-(P2<double> a, P2<double> b) { return p2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ P2<double> operator*(P2<double> a, P2<double> b) { return p2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ P2<float> fma2(P2<float> a, P2<float> b, P2<float> c) {
    P2<float> r;
    r.v = __ffma2_rn(a.v, b.v, c.v);
    return r;
}
__device__ __forceinline__ P2<double> fma2(P2<double> a, P2<double> b, P2<double> c) {
    return p2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
template <typename T> __device__ __forceinline__ P2<T> bc2(T c) { return p2(c, c); }

// Component `ax` of (J - g) for the two opposite faces of a cell along ax
// (lab-frame face gradients g[p] = (g_p of the + face, g_p of the - face)),
// both in the cell's crystal frame R: aniso_q3 on a packed pair.
template <typename T>
__device__ __forceinline__ P2<T> aniso_q3p(const P2<T> g[3], const T R[9], T eps, T hh, int ax) {
    P2<T> c[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) c[p] = fma2(bc2<T>(R[p]), g[0], fma2(bc2<T>(R[3 + p]), g[1], bc2<T>(R[6 + p]) * g[2]));
    const P2<T> r2 = fma2(c[0], c[0], fma2(c[1], c[1], c[2] * c[2]));
    const bool zd = r2.d() * hh < Guard<T>::v, za = r2.a() * hh < Guard<T>::v;
    const P2<T> inv = p2(M3<T>::rcp(r2.d()), M3<T>::rcp(r2.a()));
    P2<T> sp[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) sp[p] = c[p] * c[p] * inv;
    const P2<T> q = fma2(sp[0], sp[0], fma2(sp[1], sp[1], sp[2] * sp[2]));
    const P2<T> a = fma2(bc2<T>(T(4) * eps), q, bc2<T>(T(1) - T(3) * eps));
    const P2<T> c1 = bc2<T>(T(16) * eps) * a;
    const P2<T> c0 = fma2(a, a, bc2<T>(T(-1))) - c1 * q;
    P2<T> out = bc2<T>(T(0));
#pragma unroll
    for (int p = 0; p < 3; ++p) out = fma2(bc2<T>(R[3 * ax + p]), c[p] * fma2(c1, sp[p], c0), out);
    return p2(zd ? T(0) : out.d(), za ? T(0) : out.a());
}

// shared-memory element of a (D, anti-trapping) pair: one 8- or 16-byte load
template <typename T> struct Pair3;
template <> struct Pair3<float> {
    using t = float2;
    static __device__ __forceinline__ P2<float> get(float2 v) {
        P2<float> r;
        r.v = v;
        return r;
    }
    static __device__ __forceinline__ float2 put(float d, float a) { return make_float2(d, a); }
};
template <> struct Pair3<double> {
    using t = double2;
    static __device__ __forceinline__ P2<double> get(double2 v) { return p2(v.x, v.y); }
    static __device__ __forceinline__ double2 put(double d, double a) { return make_double2(d, a); }
};

template <typename T> struct ConstOf3;
template <> struct ConstOf3<float> {
    static __device__ __forceinline__ const float* get(const InstRec& r) { return r.cf; }
};
template <> struct ConstOf3<double> {
    static __device__ __forceinline__ const double* get(const InstRec& r) { return r.cd; }
};

template <typename T, int S, int TX, int TY> struct Tile3 {
    static constexpr int AX = TX + 2, AY = TY + 2;  // ring-1 region = threads
    static constexpr int PX = TX + 4, PY = TY + 4;  // psi region (halo 2)
    static constexpr int NT = AX * AY;
    // owned phase-2 fluxes per field: in-plane (+x, +y faces [, +x+y, +x-y
    // edges]) and toward the next plane (+z face [, +x+z, -x+z, +y+z, -y+z])
    static constexpr int NFI = (S == SBAR120) ? 4 : 2;
    static constexpr int NFZ = (S == SBAR120) ? 5 : 1;
    static constexpr size_t smem =
        sizeof(T) * (8 * PX * PY + 8 * NT + 4 * NT + 4 * NT + 2 * 4 * NT + 2 * NFI * NT + 2 * 2 * NFZ * NT);
};

// Resident blocks per SM asked of the FP32 kernels on the 30 x 6 tile: two
// for S-bar_{1,2,0} (128 registers), three for S_{1,0,0} (80 registers, 20 B
// spilled).  Independent blocks keep their barrier phases apart, which pays
// for the tile's larger ring recompute; three S_{1,0,0} blocks run 7 % faster
// than two, while S-bar_{1,2,0} spills too much at 80 registers.
template <typename T, int S, int TX, int TY>
__global__ void __launch_bounds__((TX + 2) * (TY + 2), (sizeof(T) == 4 && TY == 6) ? (S == S100 ? 3 : 2) : 1) k_step3d(const WorkItem* __restrict__ work, int n_work,
                                                              const InstRec* __restrict__ recs, int launch_parity,
                                                              StepClock clk) {
    using TL = Tile3<T, S, TX, TY>;
    constexpr int AX = TL::AX, AY = TL::AY, PX = TL::PX, PY = TL::PY, NT = TL::NT;
    constexpr int NFI = TL::NFI, NFZ = TL::NFZ;
    constexpr bool ISO = (S == SBAR120);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s_psi = reinterpret_cast<T*>(smem_raw);  // [8][PY][PX]
    T* s_phi = s_psi + 8 * PX * PY;             // [8][AY][AX]
    T* s_U = s_phi + 8 * NT;                    // [4][AY][AX]
    T* s_dphi = s_U + 4 * NT;                   // [4][AY][AX]
    // (D, anti-trapping) pairs, interleaved so that a packed pair is one load:
    using T2 = typename Pair3<T>::t;
    T2* s_al = reinterpret_cast<T2*>(s_dphi + 4 * NT);  // [4][AY][AX] alphas: 1 - phi and the anti-trapping alpha
    T2* s_fi = s_al + 4 * NT;                            // [NFI][NT] owned in-plane fluxes
    T2* s_fz = s_fi + NFI * NT;                          // [2 buffers][NFZ][NT] owned fluxes to the next plane
    const int tid = threadIdx.x;
    const int tx = tid % AX, ty = tid / AX;
    const T SQ2 = T(1.41421356237309504880);
    const T ISQ2 = T(0.70710678118654752440);

    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const WorkItem wi = work[w];
        const InstRec& rec = recs[wi.inst];
        const int nx = rec.nx, ny = rec.ny, nz = rec.nz;
        const long long sxy = (long long)nx * ny;
        const int par = rec.parity_offset ^ launch_parity;
        const T* __restrict__ psi = static_cast<const T*>(rec.psi[par]);
        const T* __restrict__ Uf = static_cast<const T*>(rec.U[par]);
        T* __restrict__ psi_o = static_cast<T*>(rec.psi[par ^ 1]);
        T* __restrict__ U_o = static_cast<T*>(rec.U[par ^ 1]);
        const int16_t* __restrict__ grain = rec.grain;
        const T* __restrict__ rot = static_cast<const T*>(rec.rot);
        const T* cst = ConstOf3<T>::get(rec);
        const T ih = cst[C_IH], hh = cst[C_HH], dt = cst[C_DT];
        const T i4h = cst[C_I4H];
        const T kk = cst[C_K], omk = cst[C_OMK], eps = cst[C_EPS], lam = cst[C_LAM], Dc = cst[C_D];
        const T ih2 = cst[C_IH2];
        const T isq2dt = cst[C_ISQ2DT];
        const int x0 = wi.x0, y0 = wi.y0, z0 = wi.z0;
        const bool t0 = rec.tlevel != 0;  // T0 time level
        const int z1 = min(z0 + wi.ext, nz);

        // this thread's ring-region cell and the cell it computes in phase 1
        const int vx = x0 - 1 + tx, vy = y0 - 1 + ty;
        // x walls: mirror, or periodic (rec.bcx); y and z walls: mirror
        const bool per = rec.bcx != 0;
        auto xidx = [&](int c) -> int { return per ? ((c % nx) + nx) % nx : mirror_idx(c, nx); };
        const int mx = xidx(vx), my = mirror_idx(vy, ny);
        const bool do_p1 = vx >= -1 && vx <= nx && vy >= -1 && vy <= ny;
        const bool do_p2 = tx >= 1 && tx <= AX - 2 && ty >= 1 && ty <= AY - 2 && vx < nx && vy < ny;
        // psi-region index of the phase-1 cell: a mirror ghost evaluates its mirror
        // cell; a periodic ghost evaluates in place (its tile neighbourhood is
        // the wrapped cell's)
        const int jx = per ? vx - x0 + 2 : mx - x0 + 2, jy = my - y0 + 2;
        // frozen temperature along +y (Eqs. Thermal_F1/_F2): zeta of the phase-1
        // cell at this launch's step; F2 = U + zeta, the rate divided by F1
        T zc = T(0), iF1 = T(1);
        if (rec.thermal) {
            const long long n = clk.clock ? clk.base[wi.inst] + *clk.clock : clk.step;
            zc = (T)((double)my * rec.zA - rec.zB - (double)n * rec.zC);
            iF1 = T(1) / (T(1) - omk * zc);
        }

        // shared-memory elements of the block (the checked build bounds every
        // ring access by the whole allocation: the unconditional owned-flux
        // loads read one ring cell past an array on purpose)
        constexpr long long SM_ELEMS = (long long)(TL::smem / sizeof(T));
        const long long NN = sxy * nz;  // cells of the instance
        auto PS = [&](int z, int y, int x) -> T& { return s_psi[PF_CHK(((z & 7) * PY + y) * PX + x, 8 * PX * PY)]; };
        auto RG = [&](T* base, int slots, int z, int y, int x) -> T& {
            return s_psi[PF_CHK((base - s_psi) + (((z & (slots - 1)) * AY + y) * AX + x), SM_ELEMS)];
        };
        // pair arrays, indexed in pairs; the checked build bounds a pair by the
        // whole allocation (two elements)
        constexpr long long SM_PAIRS = SM_ELEMS / 2;
        auto PR = [&](T2* base, long long i) -> T2& {
            return reinterpret_cast<T2*>(s_psi)[PF_CHK((base - reinterpret_cast<T2*>(s_psi)) + i, SM_PAIRS)];
        };
        auto AL = [&](int z, int y, int x) -> T2& { return PR(s_al, ((z & 3) * AY + y) * AX + x); };

        // plane loads, split into a global fetch into registers (issued one
        // plane ahead) and a store into the shared-memory rings
        constexpr int NPL = (PX * PY + NT - 1) / NT;  // psi cells per thread and plane
        T pv[NPL];
        T uv = T(0);
        auto fetch_psi = [&](int vz) {
            const long long rz = mirror_idx(vz, nz);
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
                const int i = tid + k * NT;
                if (i < PX * PY) {
                    const int px = i % PX, py = i / PX;
                    const int gx = xidx(x0 - 2 + px), gy = mirror_idx(y0 - 2 + py, ny);
                    pv[k] = __ldg(psi + PF_CHK(rz * sxy + (long long)gy * nx + gx, NN));
                }
            }
        };
        auto put_psi = [&](int vz) {
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
                const int i = tid + k * NT;
                if (i < PX * PY) {
                    const int px = i % PX, py = i / PX;
                    PS(vz, py, px) = pv[k];
                    if (px >= 1 && px <= PX - 2 && py >= 1 && py <= PY - 2)
                        RG(s_phi, 8, vz, py - 1, px - 1) = M3<T>::tanh_(pv[k] * ISQ2);
                }
            }
        };
        auto load_psi_plane = [&](int vz) {
            fetch_psi(vz);
            put_psi(vz);
        };
        auto fetch_U = [&](int vz) { uv = __ldg(Uf + PF_CHK(mirror_idx(vz, nz) * sxy + (long long)my * nx + mx, NN)); };
        auto put_U = [&](int vz) { RG(s_U, 4, vz, ty, tx) = uv; };
        auto load_U_plane = [&](int vz) {
            fetch_U(vz);
            put_U(vz);
        };
        auto grain_at = [&](int p) -> int { return grain[PF_CHK(mirror_idx(p, nz) * sxy + (long long)my * nx + mx, NN)]; };
        // crystal frame of the phase-1 cell, reloaded only when its grain changes
        T R[9];
        int gR = -1;

        // anisotropy: the +z face of the cell's previous plane is its -z face
        T qz_c = T(0);
        int gz_c = -1, pz_c = -100;

        // phase 1 at real plane p for the cell (mx, my, p); returns phi',
        // writes delta phi and the alphas of the U equation for this slot
        auto phase1 = [&](int p, int g, T& psin) -> T {
            if (g != gR) {
#pragma unroll
                for (int q = 0; q < 9; ++q) R[q] = __ldg(rot + 9 * PF_CHK(g, rec.n_grains) + q);
                gR = g;
            }
            // element offsets of the cell in its three psi planes, formed once:
            // the neighbour offsets then fold into the loads' immediates
            const int pb[3] = {(((p - 1) & 7) * PY + jy) * PX + jx, ((p & 7) * PY + jy) * PX + jx,
                               (((p + 1) & 7) * PY + jy) * PX + jx};
            auto P = [&](int dx, int dy, int dz) -> T { return s_psi[PF_CHK(pb[dz + 1] + dy * PX + dx, 8 * PX * PY)]; };
            const T pc = P(0, 0, 0);
            const T s100 = P(1, 0, 0) + P(-1, 0, 0) + P(0, 1, 0) + P(0, -1, 0) + P(0, 0, 1) + P(0, 0, -1);
            T L, G;
            {
                const T ex = P(1, 0, 0) - P(-1, 0, 0), ey = P(0, 1, 0) - P(0, -1, 0), ez = P(0, 0, 1) - P(0, 0, -1);
                const T g100 = (ex * ex + ey * ey + ez * ez) * T(0.25) * ih2;
                if (ISO) {
                    T s110 = T(0);
#pragma unroll
                    for (int a = -1; a <= 1; a += 2)
#pragma unroll
                        for (int b = -1; b <= 1; b += 2) s110 += P(a, b, 0) + P(a, 0, b) + P(0, a, b);
                    L = (T(1.0 / 3.0) * (s100 - T(6) * pc) + T(2.0 / 3.0) * T(0.25) * (s110 - T(12) * pc)) * ih2;
                    const T d1 = P(1, 1, 0) - P(-1, -1, 0), d2 = P(1, -1, 0) - P(-1, 1, 0);
                    const T d3 = P(1, 0, 1) - P(-1, 0, -1), d4 = P(-1, 0, 1) - P(1, 0, -1);
                    const T d5 = P(0, 1, 1) - P(0, -1, -1), d6 = P(0, -1, 1) - P(0, 1, -1);
                    const T g010 = (d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6) * T(1.0 / 16.0) * ih2;
                    G = T(1.0 / 3.0) * g100 + T(2.0 / 3.0) * g010;
                } else {
                    L = (s100 - T(6) * pc) * ih2;
                    G = g100;
                }
            }
            // <100> faces; the -z face comes from the plane below when valid
            auto face = [&](int ax, int sg) -> T {
                const int e[3] = {ax == 0 ? sg : 0, ax == 1 ? sg : 0, ax == 2 ? sg : 0};
                T gf[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (q == ax) {
                        gf[q] = (P(e[0], e[1], e[2]) - pc) * ih * T(sg);
                    } else {
                        const int t[3] = {q == 0, q == 1, q == 2};
                        gf[q] = (P(e[0] + t[0], e[1] + t[1], e[2] + t[2]) + P(t[0], t[1], t[2]) -
                                 P(e[0] - t[0], e[1] - t[1], e[2] - t[2]) - P(-t[0], -t[1], -t[2])) *
                                i4h;
                    }
                }
                return aniso_q3<T>(gf, R, eps, hh, ax);
            };
            // the two faces along x (and along y) as one packed pair (+ face, - face)
            auto face_pair = [&](int ax) -> P2<T> {
                P2<T> gf[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int e[3] = {ax == 0, ax == 1, ax == 2};
                    if (q == ax) {
                        gf[q] = p2((P(e[0], e[1], e[2]) - pc) * ih, (pc - P(-e[0], -e[1], -e[2])) * ih);
                    } else {
                        const int t[3] = {q == 0, q == 1, q == 2};
                        const P2<T> up = p2(P(e[0] + t[0], e[1] + t[1], e[2] + t[2]), P(-e[0] + t[0], -e[1] + t[1], -e[2] + t[2]));
                        const P2<T> dn = p2(P(e[0] - t[0], e[1] - t[1], e[2] - t[2]), P(-e[0] - t[0], -e[1] - t[1], -e[2] - t[2]));
                        gf[q] = ((up + bc2<T>(P(t[0], t[1], t[2]))) - (dn + bc2<T>(P(-t[0], -t[1], -t[2])))) * bc2<T>(i4h);
                    }
                }
                return aniso_q3p<T>(gf, R, eps, hh, ax);
            };
            const T qzp = face(2, 1);
            const T qzm = (pz_c == p && gz_c == g) ? qz_c : face(2, -1);
            qz_c = qzp;
            gz_c = g;
            pz_c = p + 1;
            const P2<T> fx = face_pair(0), fy = face_pair(1);
            const T N = (((fx.d() - fx.a()) + (fy.d() - fy.a())) + (qzp - qzm)) * ih;
            T gc[3] = {(P(1, 0, 0) - P(-1, 0, 0)) * T(0.5) * ih, (P(0, 1, 0) - P(0, -1, 0)) * T(0.5) * ih,
                       (P(0, 0, 1) - P(0, 0, -1)) * T(0.5) * ih};
            const T ac = aniso_a3<T>(gc, R, eps, hh);
            const T ph = RG(s_phi, 8, p, jy - 1, jx - 1);
            const T u = RG(s_U, 4, p, jy - 1, jx - 1);
            const T rate =
                ((L + N + SQ2 * (ph - lam * (T(1) - ph * ph) * (u + zc))) * M3<T>::rcp(ac * ac) - SQ2 * ph * G) * iF1;
            psin = pc + dt * rate;
            const T phn = M3<T>::tanh_(psin * ISQ2);
            // T1: delta phi = phi' - phi; T0: chain-rule increment, phi^n on the left-hand side
            const T dph = t0 ? dt * (T(1) - ph * ph) * ISQ2 * rate : phn - ph;
            RG(s_dphi, 4, p, ty, tx) = dph;
            AL(p, ty, tx) = Pair3<T>::put(T(1) - ph, (T(1) + omk * u) * dph * isq2dt);
            return t0 ? ph : phn;
        };
        // ghost plane vz takes the slot values of plane mz
        auto copy_plane = [&](int vz, int mz) {
            RG(s_dphi, 4, vz, ty, tx) = RG(s_dphi, 4, mz, ty, tx);
            AL(vz, ty, tx) = AL(mz, ty, tx);
        };

        // Owned phase-2 fluxes of this ring cell: in-plane at plane r (into
        // s_fi) and toward plane r+1 (into s_fz[buf]).  A flux is stored times
        // 6 h^2 for D~_{1,2,0} (faces weight 2, edges weight 1) and times h^2
        // for S_{1,0,0}; fluxes whose stencil leaves the ring region are set to
        // zero (no output cell uses them).
        auto owned_fluxes = [&](int r, int buf) {
            // ring-region offsets of the cell in planes r-1 .. r+1 and its
            // psi-region offsets, formed once (neighbour offsets fold into
            // the loads' immediates)
            const int rb[3] = {(((r - 1) & 3) * AY + ty) * AX + tx, ((r & 3) * AY + ty) * AX + tx,
                               (((r + 1) & 3) * AY + ty) * AX + tx};
            const int qb[3] = {(((r - 1) & 7) * PY + ty + 1) * PX + tx + 1, ((r & 7) * PY + ty + 1) * PX + tx + 1,
                               (((r + 1) & 7) * PY + ty + 1) * PX + tx + 1};
            auto ALr = [&](int dx, int dy, int dz) -> T2& { return PR(s_al, rb[dz + 1] + dy * AX + dx); };
            auto aD = [&](int dx, int dy, int dz) -> T { return ALr(dx, dy, dz).x; };
            auto aA = [&](int dx, int dy, int dz) -> T { return ALr(dx, dy, dz).y; };
            auto bU = [&](int dx, int dy, int dz) -> T {
                return s_psi[PF_CHK((s_U - s_psi) + rb[dz + 1] + dy * AX + dx, SM_ELEMS)];
            };
            auto bP = [&](int dx, int dy, int dz) -> T {
                return s_psi[PF_CHK(qb[dz + 1] + dy * PX + dx, 8 * PX * PY)];
            };
            const T u0 = bU(0, 0, 0), p0 = bP(0, 0, 0);
            // (D, A) pairs of alpha (one load) and beta
            auto A2 = [&](int dx, int dy, int dz) -> P2<T> { return Pair3<T>::get(ALr(dx, dy, dz)); };
            auto B2 = [&](int dx, int dy, int dz) -> P2<T> { return p2(bU(dx, dy, dz), bP(dx, dy, dz)); };
            const P2<T> b00 = p2(u0, p0);
            // <100> face toward e (S_{1,0,0}): returns the (D, A) flux
            auto face = [&](const int e[3], T& fD, T& fA) {
                {
                    fD = T(0.5) * (aD(0, 0, 0) + aD(e[0], e[1], e[2])) * (bU(e[0], e[1], e[2]) - u0);
                    T gf[3];
                    int ax = e[0] != 0 ? 0 : (e[1] != 0 ? 1 : 2);
                    const int sg = e[ax];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        if (q == ax) {
                            gf[q] = (bP(e[0], e[1], e[2]) - p0) * ih * T(sg);
                        } else {
                            const int t[3] = {q == 0, q == 1, q == 2};
                            gf[q] = (bP(e[0] + t[0], e[1] + t[1], e[2] + t[2]) + bP(t[0], t[1], t[2]) -
                                     bP(e[0] - t[0], e[1] - t[1], e[2] - t[2]) - bP(-t[0], -t[1], -t[2])) *
                                    i4h;
                        }
                    }
                    const T m2 = gf[0] * gf[0] + gf[1] * gf[1] + gf[2] * gf[2];
                    fA = (m2 * hh < Guard<T>::v) ? T(0)
                                                  : T(0.5) * (aA(0, 0, 0) + aA(e[0], e[1], e[2])) *
                                                        (bP(e[0], e[1], e[2]) - p0) * M3<T>::rcp(M3<T>::sqrt_(m2));
                }
            };
            // Every owned flux is evaluated unconditionally, so that the
            // compiler can share the neighbourhood loads between fluxes.  A
            // flux whose stencil leaves the ring region reads the adjacent
            // ring slot or array, always inside the block's shared memory; no
            // output cell reads such a flux (each flux that flux_sum reads
            // has its whole stencil inside the ring), so it is stored as it
            // comes out.
            T oD[NFI + NFZ], oA[NFI + NFZ];
            if constexpr (ISO) {
                // D~_{1,2,0} fluxes from shared sums of the 27 (D, A) alpha
                // pairs around the cell: a face toward e weighs 1/2 the mean
                // pair (0, e) and 1/8 the eight tangential neighbours of the
                // pair; an edge toward e1 + e2 weighs 3/16 the four cells of
                // its square and 1/32 the eight cells beside it along the
                // third axis.  Column sums along z, y and x (Kz, Jy, Ix) give
                // the tangential terms of all nine fluxes.
                auto Kz = [&](int dx, int dy) { return A2(dx, dy, -1) + A2(dx, dy, 1); };
                auto Jy = [&](int dx, int dz) { return A2(dx, -1, dz) + A2(dx, 1, dz); };
                auto Ix = [&](int dy, int dz) { return A2(-1, dy, dz) + A2(1, dy, dz); };
                const P2<T> a0 = A2(0, 0, 0);
                const P2<T> nX = a0 + A2(1, 0, 0), nY = a0 + A2(0, 1, 0), nZ = a0 + A2(0, 0, 1);
                const P2<T> k00 = Kz(0, 0), k10 = Kz(1, 0), k01 = Kz(0, 1);
                const P2<T> j00 = Jy(0, 0), j10 = Jy(1, 0), j01 = Jy(0, 1);
                const P2<T> i00 = Ix(0, 0), i10 = Ix(1, 0), i01 = Ix(0, 1);
                const P2<T> kx = k00 + k10, jx = j00 + j10, iy = i00 + i10, jz = j00 + j01;
                const P2<T> hf = bc2<T>(T(0.5)), ef = bc2<T>(T(1.0 / 8.0));
                const P2<T> he = bc2<T>(T(3.0 / 16.0)), ee = bc2<T>(T(1.0 / 32.0));
                auto put = [&](int q, P2<T> n, P2<T> m, P2<T> h, P2<T> e, int dx, int dy, int dz) {
                    const P2<T> f = fma2(h, n, e * m) * (B2(dx, dy, dz) - b00);
                    oD[q] = f.d();
                    oA[q] = f.a();
                };
                // in-plane: +x face, +y face, +x+y and +x-y edges
                put(0, nX, jx + kx, hf, ef, 1, 0, 0);
                put(1, nY, iy + (k00 + k01), hf, ef, 0, 1, 0);
                put(2, nX + (A2(0, 1, 0) + A2(1, 1, 0)), kx + (k01 + Kz(1, 1)), he, ee, 1, 1, 0);
                put(3, nX + (A2(0, -1, 0) + A2(1, -1, 0)), kx + (Kz(0, -1) + Kz(1, -1)), he, ee, 1, -1, 0);
                // toward plane r+1: +z face, +x+z, -x+z, +y+z, -y+z edges
                put(NFI, nZ, (i00 + i01) + jz, hf, ef, 0, 0, 1);
                put(NFI + 1, nX + (A2(0, 0, 1) + A2(1, 0, 1)), jx + (j01 + Jy(1, 1)), he, ee, 1, 0, 1);
                put(NFI + 2, nZ + (A2(-1, 0, 0) + A2(-1, 0, 1)), (j00 + Jy(-1, 0)) + (j01 + Jy(-1, 1)), he, ee, -1, 0,
                    1);
                put(NFI + 3, nY + (A2(0, 0, 1) + A2(0, 1, 1)), iy + (i01 + Ix(1, 1)), he, ee, 0, 1, 1);
                put(NFI + 4, nZ + (A2(0, -1, 0) + A2(0, -1, 1)), (i00 + Ix(-1, 0)) + (i01 + Ix(-1, 1)), he, ee, 0, -1,
                    1);
            } else {
                {
                    const int e[3] = {1, 0, 0};
                    face(e, oD[0], oA[0]);
                }
                {
                    const int e[3] = {0, 1, 0};
                    face(e, oD[1], oA[1]);
                }
                const int e[3] = {0, 0, 1};
                face(e, oD[NFI], oA[NFI]);
            }
#pragma unroll
            for (int q = 0; q < NFI; ++q) PR(s_fi, (long long)q * NT + tid) = Pair3<T>::put(oD[q], oA[q]);
#pragma unroll
            for (int q = 0; q < NFZ; ++q)
                PR(s_fz, (long long)(buf * NFZ + q) * NT + tid) = Pair3<T>::put(oD[NFI + q], oA[NFI + q]);
        };
        // eight/eighteen-flux sums of an output cell at plane r: own fluxes
        // plus the negated owned fluxes of the neighbours that share them
        auto flux_sum = [&](int bufz_cur, int bufz_prev, T& sD, T& sA) {
            auto FI2 = [&](int k, int dx, int dy) -> P2<T> {
                return Pair3<T>::get(s_fi[PF_CHK(k * NT + tid + dy * AX + dx, NFI * NT)]);
            };
            auto FZ2 = [&](int b, int k, int dx, int dy) -> P2<T> {
                return Pair3<T>::get(s_fz[PF_CHK((b * NFZ + k) * NT + tid + dy * AX + dx, 2 * NFZ * NT)]);
            };
            P2<T> a = (FI2(0, 0, 0) - FI2(0, -1, 0)) + (FI2(1, 0, 0) - FI2(1, 0, -1));
            a = a + (FZ2(bufz_cur, 0, 0, 0) - FZ2(bufz_prev, 0, 0, 0));
            if (ISO) {
                // in-plane edges: own +x+y, +x-y; received -x-y from (-1,-1), -x+y from (-1,+1)
                a = a + ((FI2(2, 0, 0) - FI2(2, -1, -1)) + (FI2(3, 0, 0) - FI2(3, -1, 1)));
                // edges to the next plane (own) and from the previous plane (received):
                // +x-z = -(-x+z of (+1,0)), -x-z = -(+x+z of (-1,0)),
                // +y-z = -(-y+z of (0,+1)), -y-z = -(+y+z of (0,-1))
                a = a + ((((FZ2(bufz_cur, 1, 0, 0) + FZ2(bufz_cur, 2, 0, 0)) + FZ2(bufz_cur, 3, 0, 0)) +
                          FZ2(bufz_cur, 4, 0, 0)) -
                         (((FZ2(bufz_prev, 2, 1, 0) + FZ2(bufz_prev, 1, -1, 0)) + FZ2(bufz_prev, 4, 0, 1)) +
                          FZ2(bufz_prev, 3, 0, -1)));
            }
            sD = a.d();
            sA = a.a();
        };

        // ---- prologue ----
        for (int vz = z0 - 2; vz <= z0 + 1; ++vz) load_psi_plane(vz);
        load_U_plane(z0 - 1);
        load_U_plane(z0);
        __syncthreads();
        T phin_cur = T(0);
        if (do_p1) {
            T psn;
            if (z0 - 1 >= 0) {
                T d;
                (void)phase1(z0 - 1, grain_at(z0 - 1), d);
            }
            phin_cur = phase1(z0, grain_at(z0), psn);
            if (do_p2 && z0 < z1) psi_o[PF_CHK(z0 * sxy + (long long)vy * nx + vx, NN)] = psn;
            if (z0 - 1 < 0) copy_plane(z0 - 1, z0);
        }
        __syncthreads();
        // fluxes from plane z0-1 to z0 (buffer of plane z0-1)
        owned_fluxes(z0 - 1, (z0 - 1) & 1);
        __syncthreads();

        // prefetch psi plane z0+2, U and grain plane z0+1
        fetch_psi(z0 + 2);
        fetch_U(z0 + 1);
        int gv = do_p1 ? grain_at(z0 + 1) : 0;
        for (int r = z0; r < z1; ++r) {
            put_psi(r + 2);
            put_U(r + 1);
            const int g1 = gv;
            if (r + 1 < z1) {
                fetch_psi(r + 3);
                fetch_U(r + 2);
                if (do_p1) gv = grain_at(r + 2);
            }
            __syncthreads();
            T phin_next = T(0);
            if (do_p1) {
                if (r + 1 < nz) {
                    T psn;
                    phin_next = phase1(r + 1, g1, psn);
                    if (do_p2 && r + 1 < z1) psi_o[PF_CHK((r + 1) * sxy + (long long)vy * nx + vx, NN)] = psn;
                } else {
                    copy_plane(r + 1, r);
                }
            }
            __syncthreads();
            owned_fluxes(r, r & 1);
            __syncthreads();
            if (do_p2) {
                T sD, sA;
                flux_sum(r & 1, (r - 1) & 1, sD, sA);
                const T cs = ISO ? T(1.0 / 6.0) * ih2 : ih2;
                const T u0 = RG(s_U, 4, r, ty, tx);
                const T dph = RG(s_dphi, 4, r, ty, tx);
                const T un = u0 + (dt * (Dc * sD + sA) * cs + (T(1) + omk * u0) * dph) *
                                      M3<T>::rcp(T(1) + kk - omk * phin_cur);
                U_o[PF_CHK(r * sxy + (long long)vy * nx + vx, NN)] = un;
            }
            phin_cur = phin_next;
        }
        __syncthreads();
    }
}

template <typename T, int S, int TX, int TY>
bool launch_t(int grid, cudaStream_t st, const WorkItem* work, int n_work, const InstRec* recs, int lp,
              StepClock clk) {
    using TL = Tile3<T, S, TX, TY>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_step3d<T, S, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TL::smem) !=
            cudaSuccess) {
            cudaGetLastError();  // a tile that does not fit is an answer, not an error for later calls
            return false;
        }
        attr = true;
    }
    k_step3d<T, S, TX, TY><<<grid, TL::NT, TL::smem, st>>>(work, n_work, recs, lp, clk);
    return true;
}
template <typename T, int S, int TX, int TY> int occ_t() {
    using TL = Tile3<T, S, TX, TY>;
    // a tile whose shared memory exceeds the per-block limit (FP64 with the
    // 30 x 14 tile) is not available: 0, with the runtime's error cleared
    if (cudaFuncSetAttribute(k_step3d<T, S, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TL::smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step3d<T, S, TX, TY>, TL::NT, TL::smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// Compiled tiles (block_x, block_y) = (TX + 4, TY + 4): (34, 18) and (34, 10).
template <typename T, int S>
bool launch_s(int bx, int by, int grid, cudaStream_t st, const WorkItem* work, int n_work, const InstRec* recs, int lp,
              StepClock clk) {
    if (bx == 34 && by == 18) return launch_t<T, S, 30, 14>(grid, st, work, n_work, recs, lp, clk);
    if (bx == 34 && by == 10) return launch_t<T, S, 30, 6>(grid, st, work, n_work, recs, lp, clk);
    return false;
}
template <typename T, int S> int occ_s(int bx, int by) {
    if (bx == 34 && by == 18) return occ_t<T, S, 30, 14>();
    if (bx == 34 && by == 10) return occ_t<T, S, 30, 6>();
    return 0;
}

}  // namespace

PF_BOUNDS_READER(bounds_step3d)

bool launch_step3d(int prec, int scheme, int bx, int by, int grid, cudaStream_t st, const WorkItem* work, int n_work,
                   const InstRec* recs, int lp, StepClock clk) {
    if (prec == 0) {
        if (scheme == S100) return launch_s<float, S100>(bx, by, grid, st, work, n_work, recs, lp, clk);
        if (scheme == SBAR120) return launch_s<float, SBAR120>(bx, by, grid, st, work, n_work, recs, lp, clk);
    } else {
        if (scheme == S100) return launch_s<double, S100>(bx, by, grid, st, work, n_work, recs, lp, clk);
        if (scheme == SBAR120) return launch_s<double, SBAR120>(bx, by, grid, st, work, n_work, recs, lp, clk);
    }
    return false;
}

int occupancy_step3d(int prec, int scheme, int bx, int by) {
    if (prec == 0) {
        if (scheme == S100) return occ_s<float, S100>(bx, by);
        if (scheme == SBAR120) return occ_s<float, SBAR120>(bx, by);
    } else {
        if (scheme == S100) return occ_s<double, S100>(bx, by);
        if (scheme == SBAR120) return occ_s<double, SBAR120>(bx, by);
    }
    return 0;
}

}  // namespace pf
