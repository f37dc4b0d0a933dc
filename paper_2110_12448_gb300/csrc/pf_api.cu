// pf_api.cu -- the C-ABI of include/pf.h: parameter validation, layout of
// the caller's device buffer, work lists, launches, observation and the
// batching groups (one persistent launch per class, CUDA-graph replay).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pf.h"
#include "pf_internal.cuh"

using namespace pf;

namespace {

thread_local std::string g_last_cuda;

int cuda_fail(cudaError_t e, const char* what) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    g_last_cuda = buf;
    return PF_ERR_CUDA;
}
// Host-side fault injection (pf_debug_inject_launch_failure): the number of
// steps that may still launch before an injected launch failure (-1: off).
std::atomic<long long> g_inject{-1};

// True if launching the next k steps runs into the armed failure (which is
// then consumed and reported like a CUDA error); else the k steps are counted.
bool inject_hits(long long k) {
    long long v = g_inject.load();
    if (v < 0) return false;
    if (v < k) {
        g_inject.store(-1);
        g_last_cuda = "injected launch failure (pf_debug_inject_launch_failure)";
        return true;
    }
    g_inject.store(v - k);
    return false;
}

#define CK(call)                                       \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool valid_params(const pf_params* p) {
    if (!p) return false;
    if (p->dim != 2 && p->dim != 3) return false;
    if (p->nx < 4 || p->ny < 4 || (p->dim == 3 && p->nz < 4)) return false;
    if (p->nx > (1 << 20) || p->ny > (1 << 20) || (p->dim == 3 && p->nz > (1 << 14))) return false;
    if (p->dim == 2 && !(p->scheme == PF_S10 || p->scheme == PF_S21 || p->scheme == PF_SBAR21)) return false;
    if (p->dim == 3 && !(p->scheme == PF_S100 || p->scheme == PF_SBAR120)) return false;
    if (p->precision != PF_F32 && p->precision != PF_F64 && p->precision != PF_F32C) return false;
    // the compensated FP32 state: 2D isothermal runs with mirror walls and the T1 time level
    if (p->precision == PF_F32C && (p->dim != 2 || p->thermal != PF_ISOTHERMAL || p->bc_x != PF_BC_MIRROR ||
                                    p->time_level != PF_T1))
        return false;
    if (!(p->h > 0) || !(p->dt > 0) || !std::isfinite(p->h) || !std::isfinite(p->dt)) return false;
    if (!(p->k > 0 && p->k < 1)) return false;
    if (!(p->eps4 >= 0 && p->eps4 < 0.25)) return false;
    if (!(p->D > 0) || !(p->lambda >= 0) || !std::isfinite(p->U0)) return false;
    if (p->max_grains < 1 || p->max_grains > 32767 || p->max_seeds < 0 || p->max_seeds > (1 << 20)) return false;
    if (p->bc_x != PF_BC_MIRROR && p->bc_x != PF_BC_PERIODIC) return false;
    if (p->thermal != PF_ISOTHERMAL && p->thermal != PF_FROZEN_GRADIENT) return false;
    if (p->time_level != PF_T1 && p->time_level != PF_T0) return false;
    if (p->kernels != PF_FUSED && p->kernels != PF_TWO_KERNELS) return false;
    // the two-kernel form: 2D, T0 time level, plain FP32 or FP64 fields
    if (p->kernels == PF_TWO_KERNELS &&
        (p->dim != 2 || p->time_level != PF_T0 || (p->precision != PF_F32 && p->precision != PF_F64)))
        return false;
    double F1min = 1.0;
    if (p->thermal == PF_FROZEN_GRADIENT) {
        if (!(p->lT > 0) || !std::isfinite(p->lT) || !(p->Vp >= 0) || !std::isfinite(p->Vp) ||
            !std::isfinite(p->yT))
            return false;
        // F1 = 1 - (1-k) zeta is smallest at the top row at t = 0 (the isotherm only moves up)
        F1min = 1.0 - (1.0 - p->k) * (((p->ny - 1) * p->h - p->yT) / p->lT);
        if (!(F1min >= 0.05)) return false;
        F1min = std::min(F1min, 1.0);
    }
    // explicit Euler bound: dt <= 2 h^2 / (Lambda max(D, 1 / F1min))
    const bool iso = p->scheme == PF_S21 || p->scheme == PF_SBAR21 || p->scheme == PF_SBAR120;
    const double lam = iso ? 16.0 / 3.0 : (p->dim == 2 ? 8.0 : 12.0);
    const double bound = 2.0 * p->h * p->h / (lam * std::max(p->D, 1.0 / F1min));
    if (p->dt > bound) return false;
    return true;
}

struct Layout {
    size_t psi0, psi1, U0, U1, grain, rot, seeds, partials, result, work, rec, rate, total;
    size_t N;
    int esz, max_seeds, max_work;
};

long long cells(const pf_params* p) { return (long long)p->nx * p->ny * (p->dim == 3 ? p->nz : 1); }

int cdiv(int a, int b) { return (a + b - 1) / b; }

// precision code of the step kernels: 0 float, 1 double, 2 compensated float pairs
int kprec(const pf_params& p) { return p.precision == PF_F64 ? 1 : (p.precision == PF_F32C ? 2 : 0); }

// capacity of the work list: the smallest tile any compiled shape produces
int max_work_items(const pf_params* p) {
    if (p->dim == 2) return cdiv(p->nx, 60) * cdiv(p->ny, 8);
    return cdiv(p->nx, 12) * cdiv(p->ny, 4) * cdiv(p->nz, 4);
}

Layout layout(const pf_params* p) {
    Layout L{};
    L.N = (size_t)cells(p);
    // bytes per cell of one field and level: FP32C holds hi and lo halves
    L.esz = p->precision == PF_F32 ? 4 : 8;
    L.max_seeds = p->max_seeds > 0 ? p->max_seeds : 64;
    L.max_work = max_work_items(p);
    size_t o = 0;
    auto take = [&](size_t n) {
        size_t r = o;
        o = align256(o + n);
        return r;
    };
    L.psi0 = take(L.N * L.esz);
    L.psi1 = take(L.N * L.esz);
    L.U0 = take(L.N * L.esz);
    L.U1 = take(L.N * L.esz);
    L.grain = take(L.N * sizeof(int16_t));
    L.rot = take((size_t)p->max_grains * 9 * L.esz);
    L.seeds = take((size_t)L.max_seeds * sizeof(SeedDev));
    L.partials = take((size_t)OBS_BLOCKS * sizeof(ObsPartial));
    L.result = take(sizeof(ObsPartial));
    L.work = take((size_t)L.max_work * sizeof(WorkItem));
    L.rec = take(sizeof(InstRec));
    L.rate = p->kernels == PF_TWO_KERNELS ? take(L.N * L.esz) : 0;  // d psi/dt between the two kernels
    L.total = o;
    return L;
}

int g_num_sms = 0;
int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 152;
    }
    return g_num_sms;
}

}  // namespace

struct pf_sim {
    pf_params p;
    Layout L;
    char* base;
    cudaStream_t st;
    void* psi[2];
    void* U[2];
    int16_t* grain;
    void* rot;
    SeedDev* seeds;
    ObsPartial* partials;
    ObsPartial* result;
    WorkItem* work;
    InstRec* rec;
    void* rate;  // d psi/dt of the two-kernel form (nullptr when fused)
    int n_grains;
    int gmax;         // largest grain index in the map (0: every cell in grain 0)
    int64_t rec_gen;  // advanced by every change the instance record carries
    std::vector<double> rot_h, centres_h;
    int64_t step;
    int bx, by, sweep, n_work, grid;
    bool work_dirty;
    std::vector<WorkItem> work_h;
    std::vector<int> have_prev;       // per grain + 2 (index 0: pulling axis, 1: global)
    std::vector<double> prev;         // t, x, y, z per slot
    pf_group* group;
};

namespace {

void default_tile(pf_sim* s) {
    if (s->p.dim == 2) {
        s->bx = 64;  // one warp per 60-column strip
        s->by = 1;
        s->sweep = 32;
    } else {
        // (TX + 4, TY + 4): 30 x 6 output columns
        s->bx = 34;
        s->by = 10;
        s->sweep = 32;
    }
}

void build_work(const pf_sim* s, int inst, std::vector<WorkItem>& out) {
    const pf_params& p = s->p;
    if (p.dim == 2) {
        const int TX = s->bx - 4;
        for (int y0 = 0; y0 < p.ny; y0 += s->sweep)
            for (int x0 = 0; x0 < p.nx; x0 += TX) out.push_back(WorkItem{inst, x0, y0, 0, s->sweep, 0, 0, 0});
    } else {
        const int TX = s->bx - 4, TY = s->by - 4;
        for (int z0 = 0; z0 < p.nz; z0 += s->sweep)
            for (int y0 = 0; y0 < p.ny; y0 += TY)
                for (int x0 = 0; x0 < p.nx; x0 += TX) out.push_back(WorkItem{inst, x0, y0, z0, s->sweep, 0, 0, 0});
    }
}

// the 2D kernel variant: 1 frozen temperature and/or periodic x (either time
// level), 2 isothermal with mirror walls at the T0 level, 0 otherwise
int ds_of(const pf_params& p) {
    if (p.thermal == PF_FROZEN_GRADIENT || p.bc_x == PF_BC_PERIODIC) return 1;
    return p.time_level == PF_T0 ? 2 : 0;
}

// resident units of the step's kernel; for the two-kernel form those of the
// pass with fewer, so that one persistent grid serves both passes
int occupancy_of(const pf_params& p, int bx, int by) {
    const int prec = kprec(p);
    if (p.dim == 3) return occupancy_step3d(prec, p.scheme, bx, by);
    if (p.kernels == PF_TWO_KERNELS)
        return std::min(occupancy_step2d(prec, p.scheme, bx, ds_of(p), 1), occupancy_step2d(prec, p.scheme, bx, ds_of(p), 2));
    return occupancy_step2d(prec, p.scheme, bx, ds_of(p));
}

int occupancy(const pf_sim* s) { return occupancy_of(s->p, s->bx, s->by); }

InstRec make_rec(const pf_sim* s, int parity_offset) {
    InstRec r{};
    r.psi[0] = s->psi[0];
    r.psi[1] = s->psi[1];
    r.U[0] = s->U[0];
    r.U[1] = s->U[1];
    r.grain = s->grain;
    r.rot = s->rot;
    r.rate = s->rate;
    r.nx = s->p.nx;
    r.ny = s->p.ny;
    r.nz = s->p.dim == 3 ? s->p.nz : 1;
    r.parity_offset = parity_offset;
    r.thermal = s->p.thermal == PF_FROZEN_GRADIENT ? 1 : 0;
    r.bcx = s->p.bc_x == PF_BC_PERIODIC ? 1 : 0;
    r.tlevel = s->p.time_level == PF_T0 ? 1 : 0;
    r.n_grains = s->n_grains;
    r.one_grain = s->gmax == 0 ? 1 : 0;
    if (r.thermal) {
        r.zA = s->p.h / s->p.lT;
        r.zB = s->p.yT / s->p.lT;
        r.zC = s->p.Vp * s->p.dt / s->p.lT;
    }
    r.h = s->p.h;
    r.dt = s->p.dt;
    r.k = s->p.k;
    r.eps4 = s->p.eps4;
    r.lambda = s->p.lambda;
    r.D = s->p.D;
    const double h = s->p.h;
    double c[NC];
    c[C_IH] = 1.0 / h;
    c[C_I4H] = 0.25 / h;
    c[C_IH_HALF] = 0.5 / h;
    c[C_HH] = h * h;
    c[C_IH2] = 1.0 / (h * h);
    c[C_I6H2] = 1.0 / (6.0 * h * h);
    c[C_G10] = 2.0 / 3.0 / (4.0 * h * h);
    c[C_G01] = 1.0 / 3.0 / (8.0 * h * h);
    c[C_DT] = s->p.dt;
    c[C_K] = s->p.k;
    c[C_OMK] = 1.0 - s->p.k;
    c[C_EPS] = s->p.eps4;
    c[C_LAM] = s->p.lambda;
    c[C_D] = s->p.D;
    c[C_ISQ2DT] = 1.0 / (1.41421356237309504880 * s->p.dt);
    c[C_I4H2] = 1.0 / (4.0 * h * h);
    for (int i = 0; i < NC; ++i) {
        r.cd[i] = c[i];
        r.cf[i] = (float)c[i];
    }
    return r;
}

int upload_work(pf_sim* s) {
    s->work_h.clear();
    build_work(s, 0, s->work_h);
    if ((int)s->work_h.size() > s->L.max_work) return PF_ERR_INVALID;
    s->n_work = (int)s->work_h.size();
    CK(cudaMemcpyAsync(s->work, s->work_h.data(), s->work_h.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s->st));
    InstRec r = make_rec(s, 0);
    CK(cudaMemcpyAsync(s->rec, &r, sizeof(r), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    const int occ = occupancy(s);
    if (occ <= 0) return PF_ERR_INVALID;
    s->grid = std::min(s->n_work, occ * num_sms());
    s->work_dirty = false;
    return PF_OK;
}

int upload_rot(pf_sim* s) {
    const int n = s->n_grains;
    if (s->p.precision == PF_F64) {
        CK(cudaMemcpyAsync(s->rot, s->rot_h.data(), (size_t)n * 9 * sizeof(double), cudaMemcpyHostToDevice, s->st));
        CK(cudaStreamSynchronize(s->st));
    } else {
        std::vector<float> f(s->rot_h.begin(), s->rot_h.end());
        CK(cudaMemcpyAsync(s->rot, f.data(), (size_t)n * 9 * sizeof(float), cudaMemcpyHostToDevice, s->st));
        CK(cudaStreamSynchronize(s->st));
    }
    return PF_OK;
}

// One step of a handle from step `step` (its parity selects the time level).
bool launch_sim_step(const pf_sim* s, int64_t step) {
    const int prec = kprec(s->p);
    const int lp = (int)(step & 1);
    const StepClock clk{nullptr, nullptr, (long long)step};
    if (s->p.dim == 2 && s->p.kernels == PF_TWO_KERNELS)
        return launch_step2d(prec, s->p.scheme, s->bx, s->grid, s->st, s->work, s->n_work, s->rec, lp, clk,
                             ds_of(s->p), 1) &&
               launch_step2d(prec, s->p.scheme, s->bx, s->grid, s->st, s->work, s->n_work, s->rec, lp, clk,
                             ds_of(s->p), 2);
    if (s->p.dim == 2)
        return launch_step2d(prec, s->p.scheme, s->bx, s->grid, s->st, s->work, s->n_work, s->rec, lp, clk,
                             ds_of(s->p));
    return launch_step3d(prec, s->p.scheme, s->bx, s->by, s->grid, s->st, s->work, s->n_work, s->rec, lp,
                         StepClock{nullptr, nullptr, (long long)step});
}

// Compensated FP32 state (PF_F32C): the 8 bytes per cell of a level hold the
// hi half (N floats) followed by the lo half.  Between steps the other level
// is free, so FP64 copies of the current fields are formed there (join) and
// FP64 fields from the host are split from there into the current level.
float* lo_of(const pf_sim* s, void* hi) { return static_cast<float*>(hi) + s->L.N; }

cudaError_t join_current(const pf_sim* s, bool psi, bool U) {
    const int cur = (int)(s->step & 1), oth = cur ^ 1;
    cudaError_t e = cudaSuccess;
    if (psi)
        e = launch_join(static_cast<const float*>(s->psi[cur]), lo_of(s, s->psi[cur]), static_cast<double*>(s->psi[oth]),
                        (long long)s->L.N, s->st);
    if (e == cudaSuccess && U)
        e = launch_join(static_cast<const float*>(s->U[cur]), lo_of(s, s->U[cur]), static_cast<double*>(s->U[oth]),
                        (long long)s->L.N, s->st);
    return e;
}

cudaError_t split_into_current(const pf_sim* s, bool psi, bool U) {
    const int cur = (int)(s->step & 1), oth = cur ^ 1;
    cudaError_t e = cudaSuccess;
    if (psi)
        e = launch_split(static_cast<const double*>(s->psi[oth]), static_cast<float*>(s->psi[cur]), lo_of(s, s->psi[cur]),
                         (long long)s->L.N, s->st);
    if (e == cudaSuccess && U)
        e = launch_split(static_cast<const double*>(s->U[oth]), static_cast<float*>(s->U[cur]), lo_of(s, s->U[cur]),
                         (long long)s->L.N, s->st);
    return e;
}

}  // namespace

extern "C" {

size_t pf_required_bytes(const pf_params* p) {
    if (!valid_params(p)) return 0;
    return layout(p).total;
}

int pf_create(const pf_params* p, void* dev_mem, size_t bytes, void* stream, pf_sim** out) {
    if (!out) return PF_ERR_INVALID;
    *out = nullptr;
    if (!valid_params(p) || !dev_mem) return PF_ERR_INVALID;
    if (((uintptr_t)dev_mem & 255) != 0) return PF_ERR_INVALID;
    Layout L = layout(p);
    if (bytes < L.total) return PF_ERR_BUDGET;
    pf_sim* s = new (std::nothrow) pf_sim();
    if (!s) return PF_ERR_INVALID;
    s->p = *p;
    if (s->p.dim == 2) s->p.nz = 1;
    s->L = L;
    s->base = static_cast<char*>(dev_mem);
    s->st = static_cast<cudaStream_t>(stream);
    s->psi[0] = s->base + L.psi0;
    s->psi[1] = s->base + L.psi1;
    s->U[0] = s->base + L.U0;
    s->U[1] = s->base + L.U1;
    s->grain = reinterpret_cast<int16_t*>(s->base + L.grain);
    s->rot = s->base + L.rot;
    s->seeds = reinterpret_cast<SeedDev*>(s->base + L.seeds);
    s->partials = reinterpret_cast<ObsPartial*>(s->base + L.partials);
    s->result = reinterpret_cast<ObsPartial*>(s->base + L.result);
    s->work = reinterpret_cast<WorkItem*>(s->base + L.work);
    s->rec = reinterpret_cast<InstRec*>(s->base + L.rec);
    s->rate = p->kernels == PF_TWO_KERNELS ? s->base + L.rate : nullptr;
    s->n_grains = 1;
    s->gmax = 0;  // the grain map starts zero-filled
    s->rec_gen = 0;
    s->rot_h.assign(9, 0.0);
    s->rot_h[0] = s->rot_h[4] = s->rot_h[8] = 1.0;
    s->centres_h.assign(3, 0.0);
    s->centres_h[0] = (p->nx - 1) * 0.5 * p->h;
    s->centres_h[1] = (p->ny - 1) * 0.5 * p->h;
    s->centres_h[2] = p->dim == 3 ? (p->nz - 1) * 0.5 * p->h : 0.0;
    s->step = 0;
    s->group = nullptr;
    s->have_prev.assign(3, 0);
    s->prev.assign(12, 0.0);
    default_tile(s);
    int rc;
    if ((rc = upload_rot(s)) != PF_OK) { delete s; return rc; }
    cudaError_t e;
    if ((e = cudaMemsetAsync(s->grain, 0, L.N * sizeof(int16_t), s->st)) != cudaSuccess) { delete s; return cuda_fail(e, "memset grain"); }
    const int prec = p->precision == PF_F64 ? 1 : 0;
    if ((e = launch_fill(prec, s->psi[0], -1e3, (long long)L.N, s->st)) != cudaSuccess) { delete s; return cuda_fail(e, "fill psi"); }
    if (p->precision == PF_F32C) {
        // U0 = hi + lo exactly; psi = -1e3 is a float
        const float u_hi = (float)p->U0;
        const double u_lo = p->U0 - (double)u_hi;
        if ((e = launch_fill(0, lo_of(s, s->psi[0]), 0.0, (long long)L.N, s->st)) != cudaSuccess ||
            (e = launch_fill(0, s->U[0], (double)u_hi, (long long)L.N, s->st)) != cudaSuccess ||
            (e = launch_fill(0, lo_of(s, s->U[0]), u_lo, (long long)L.N, s->st)) != cudaSuccess) {
            delete s;
            return cuda_fail(e, "fill compensated fields");
        }
    } else if ((e = launch_fill(prec, s->U[0], p->U0, (long long)L.N, s->st)) != cudaSuccess) {
        delete s;
        return cuda_fail(e, "fill U");
    }
    if ((rc = upload_work(s)) != PF_OK) { delete s; return rc; }
    *out = s;
    return PF_OK;
}

int pf_set_grains(pf_sim* s, int n_grains, const double* rot9, const double* centres3) {
    if (!s || !rot9 || n_grains < 1 || n_grains > s->p.max_grains) return PF_ERR_INVALID;
    for (int i = 0; i < 9 * n_grains; ++i)
        if (!std::isfinite(rot9[i])) return PF_ERR_INVALID;
    s->n_grains = n_grains;
    s->rot_h.assign(rot9, rot9 + 9 * n_grains);
    s->centres_h.assign(3 * n_grains, 0.0);
    for (int g = 0; g < n_grains; ++g) {
        if (centres3) {
            for (int a = 0; a < 3; ++a) s->centres_h[3 * g + a] = centres3[3 * g + a];
        } else {
            s->centres_h[3 * g + 0] = (s->p.nx - 1) * 0.5 * s->p.h;
            s->centres_h[3 * g + 1] = (s->p.ny - 1) * 0.5 * s->p.h;
            s->centres_h[3 * g + 2] = s->p.dim == 3 ? (s->p.nz - 1) * 0.5 * s->p.h : 0.0;
        }
    }
    s->have_prev.assign(n_grains + 2, 0);
    s->prev.assign(4 * (n_grains + 2), 0.0);
    s->work_dirty = true;  // the instance record carries the grain count
    ++s->rec_gen;
    return upload_rot(s);
}

int pf_init_seeds(pf_sim* s, int n_seeds, const pf_seed* seeds) {
    if (!s || !seeds || n_seeds < 1 || n_seeds > s->L.max_seeds) return PF_ERR_INVALID;
    std::vector<SeedDev> h(n_seeds);
    for (int i = 0; i < n_seeds; ++i) {
        if (seeds[i].grain < 0 || seeds[i].grain >= s->n_grains) return PF_ERR_INVALID;
        if (!std::isfinite(seeds[i].x) || !std::isfinite(seeds[i].y) || !std::isfinite(seeds[i].z) ||
            !std::isfinite(seeds[i].r))
            return PF_ERR_INVALID;
        h[i] = SeedDev{seeds[i].x, seeds[i].y, s->p.dim == 3 ? seeds[i].z : 0.0, seeds[i].r, seeds[i].grain, 0};
    }
    // every cell takes the grain of its nearest seed
    int gmax = 0;
    for (int i = 0; i < n_seeds; ++i) gmax = std::max(gmax, (int)seeds[i].grain);
    CK(cudaMemcpyAsync(s->seeds, h.data(), n_seeds * sizeof(SeedDev), cudaMemcpyHostToDevice, s->st));
    const int cur = (int)(s->step & 1);
    if (s->p.precision == PF_F32C) {
        // FP64 seed fields in the free level, split into the current one
        CK(launch_init_seeds(1, s->p.dim, s->p.nx, s->p.ny, s->p.nz, s->p.h, s->p.U0, s->seeds, n_seeds,
                             s->psi[cur ^ 1], s->U[cur ^ 1], s->grain, s->st));
        CK(split_into_current(s, true, true));
    } else {
        CK(launch_init_seeds(s->p.precision == PF_F64 ? 1 : 0, s->p.dim, s->p.nx, s->p.ny, s->p.nz, s->p.h, s->p.U0,
                             s->seeds, n_seeds, s->psi[cur], s->U[cur], s->grain, s->st));
    }
    CK(cudaStreamSynchronize(s->st));
    s->gmax = gmax;
    s->work_dirty = true;
    ++s->rec_gen;
    return PF_OK;
}

int pf_set_grain_index(pf_sim* s, const int16_t* g) {
    if (!s || !g) return PF_ERR_INVALID;
    int gmax = 0;
    for (size_t c = 0; c < s->L.N; ++c) {
        if (g[c] < 0 || g[c] >= s->n_grains) return PF_ERR_INVALID;
        gmax = std::max(gmax, (int)g[c]);
    }
    CK(cudaMemcpyAsync(s->grain, g, s->L.N * sizeof(int16_t), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    s->gmax = gmax;  // the instance record says whether every cell is in grain 0
    s->work_dirty = true;
    ++s->rec_gen;
    return PF_OK;
}

int pf_get_grain_index(pf_sim* s, int16_t* g) {
    if (!s || !g) return PF_ERR_INVALID;
    CK(cudaMemcpyAsync(g, s->grain, s->L.N * sizeof(int16_t), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return PF_OK;
}

int pf_step(pf_sim* s, int64_t n) {
    if (!s || n < 0) return PF_ERR_INVALID;
    if (s->group) return PF_ERR_STATE;
    if (s->work_dirty) {
        int rc = upload_work(s);
        if (rc != PF_OK) return rc;
    }
    for (int64_t i = 0; i < n; ++i) {
        // on a failure the handle stays consistent: it has advanced by the i steps launched
        if (inject_hits(1)) {
            s->step += i;
            return PF_ERR_CUDA;
        }
        if (!launch_sim_step(s, s->step + i)) {
            s->step += i;
            return PF_ERR_INVALID;
        }
    }
    if (n > 0) CK(cudaGetLastError());
    s->step += n;
    return PF_OK;
}

}  // extern "C"

namespace {

// Arguments of the observe reductions of grain g (-2: pulling axis, -1: all
// cells, else one grain) of a handle; the compensated state is observed
// through FP64 copies of hi + lo.
int observe_args(pf_sim* s, int grain, ObsArgs& a) {
    const int dim = s->p.dim;
    const int gg = grain < 0 ? 0 : grain;
    const double* R = &s->rot_h[9 * gg];
    // growth axis: crystal axis (+- column of R) with the largest y component,
    // or +y itself (grain -2: the pulling axis of directional solidification)
    double d[3] = {0, 0, 0}, best = -INFINITY;
    if (grain == -2) {
        d[1] = 1.0;
    } else {
        for (int ax = 0; ax < dim; ++ax)
            for (int sg = 1; sg >= -1; sg -= 2) {
                const double yc = sg * R[3 + ax];
                if (yc > best) {
                    best = yc;
                    for (int q = 0; q < 3; ++q) d[q] = q < dim ? sg * R[q * 3 + ax] : 0.0;
                }
            }
    }
    int ea = 0;
    for (int ax = 1; ax < dim; ++ax)
        if (std::fabs(d[ax]) > std::fabs(d[ea])) ea = ax;
    const int es = d[ea] >= 0 ? 1 : -1;
    a = ObsArgs{};
    const int cur = (int)(s->step & 1);
    a.psi = s->psi[cur];
    a.U = s->U[cur];
    a.grain = s->grain;
    a.prec = s->p.precision == PF_F64 ? 1 : 0;
    if (s->p.precision == PF_F32C) {
        // the reductions read FP64 copies of hi + lo
        CK(join_current(s, true, true));
        a.psi = s->psi[cur ^ 1];
        a.U = s->U[cur ^ 1];
        a.prec = 1;
    }
    a.dim = dim;
    a.nx = s->p.nx;
    a.ny = s->p.ny;
    a.nz = dim == 3 ? s->p.nz : 1;
    a.grain_filter = grain < 0 ? -1 : grain;
    a.h = s->p.h;
    a.k = s->p.k;
    for (int q = 0; q < 3; ++q) {
        a.cg[q] = s->centres_h[3 * gg + q];
        a.d[q] = d[q];
    }
    a.ea = ea;
    a.es = es;
    return PF_OK;
}

// Fill *out from the reduced record r and advance the tip history of the slot.
int observe_finish(pf_sim* s, int grain, const ObsArgs& a, const ObsPartial& r, pf_obs* out) {
    const int dim = s->p.dim;
    std::memset(out, 0, sizeof(*out));
    out->step = s->step;
    out->t = (double)s->step * s->p.dt;
    const double hd = dim == 3 ? s->p.h * s->p.h * s->p.h : s->p.h * s->p.h;
    out->solute = r.solute * hd;
    out->solid_fraction = r.solid / (double)s->L.N;
    out->nonfinite = (int32_t)r.nonfinite;
    out->found = r.tip_index >= 0 ? 1 : 0;
    out->tip_index = r.tip_index;
    out->tip_score = r.tip_index >= 0 ? r.score : -INFINITY;
    const int slot = grain + 2;
    if (r.tip_index >= 0) {
        for (int q = 0; q < 3; ++q) out->tip[q] = r.tip[q];
        const double rx = r.tip[0] - a.cg[0], ry = r.tip[1] - a.cg[1], rz = dim == 3 ? r.tip[2] - a.cg[2] : 0.0;
        out->angle_xy_deg = std::atan2(-rx, ry) * (180.0 / 3.14159265358979323846);
        out->angle_out_deg = std::atan2(rz, std::sqrt(rx * rx + ry * ry)) * (180.0 / 3.14159265358979323846);
        if (s->have_prev[slot] && out->t > s->prev[4 * slot]) {
            double dd = 0.0;
            for (int q = 0; q < 3; ++q) dd += (r.tip[q] - s->prev[4 * slot + 1 + q]) * (r.tip[q] - s->prev[4 * slot + 1 + q]);
            out->v_tip = std::sqrt(dd) / (out->t - s->prev[4 * slot]);
        }
        s->have_prev[slot] = 1;
        s->prev[4 * slot] = out->t;
        for (int q = 0; q < 3; ++q) s->prev[4 * slot + 1 + q] = r.tip[q];
    } else {
        out->tip[0] = out->tip[1] = out->tip[2] = NAN;
        out->angle_xy_deg = out->angle_out_deg = NAN;
    }
    return r.nonfinite > 0 ? PF_ERR_NONFINITE : PF_OK;
}

}  // namespace

extern "C" {

int pf_observe(pf_sim* s, int grain, pf_obs* out) {
    if (!s || !out || grain < -2 || grain >= s->n_grains) return PF_ERR_INVALID;
    ObsArgs a;
    int rc = observe_args(s, grain, a);
    if (rc != PF_OK) return rc;
    CK(launch_observe(a, s->partials, s->result, s->st));
    ObsPartial r;
    CK(cudaMemcpyAsync(&r, s->result, sizeof(r), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return observe_finish(s, grain, a, r, out);
}

int pf_get_fields(pf_sim* s, void* psi_host, void* U_host) {
    if (!s || (!psi_host && !U_host)) return PF_ERR_INVALID;
    int cur = (int)(s->step & 1);
    const size_t b = s->L.N * s->L.esz;
    if (s->p.precision == PF_F32C) {  // FP64 host arrays: hi + lo joined in the free level
        CK(join_current(s, psi_host != nullptr, U_host != nullptr));
        cur ^= 1;
    }
    if (psi_host) CK(cudaMemcpyAsync(psi_host, s->psi[cur], b, cudaMemcpyDeviceToHost, s->st));
    if (U_host) CK(cudaMemcpyAsync(U_host, s->U[cur], b, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return PF_OK;
}

int pf_tip_radius(pf_sim* s, int grain, const double tip[3], double v_tip, pf_tip* out) {
    if (!s || !out || !tip || grain < -1 || grain >= s->n_grains) return PF_ERR_INVALID;
    const int dim = s->p.dim;
    for (int q = 0; q < dim; ++q)
        if (!std::isfinite(tip[q])) return PF_ERR_INVALID;
    const int gg = grain < 0 ? 0 : grain;
    TipArgs a{};
    const int cur = (int)(s->step & 1);
    a.psi = s->psi[cur];
    a.prec = s->p.precision == PF_F64 ? 1 : 0;
    if (s->p.precision == PF_F32C) {
        CK(join_current(s, true, false));
        a.psi = s->psi[cur ^ 1];
        a.prec = 1;
    }
    a.dim = dim;
    a.nx = s->p.nx;
    a.ny = s->p.ny;
    a.nz = dim == 3 ? s->p.nz : 1;
    a.h = s->p.h;
    double na = 0.0;
    for (int q = 0; q < 3; ++q) {
        a.tip[q] = q < dim ? tip[q] : 0.0;
        a.axis[q] = q < dim ? tip[q] - s->centres_h[3 * gg + q] : 0.0;
        na += a.axis[q] * a.axis[q];
    }
    if (!(na > 0.0)) return PF_ERR_INVALID;
    // the observe scratch holds the five results
    double* dres = reinterpret_cast<double*>(s->partials);
    CK(launch_tip_radius(a, dres, s->st));
    double r[5];
    CK(cudaMemcpyAsync(r, dres, sizeof(r), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    std::memset(out, 0, sizeof(*out));
    out->rho = r[0];
    out->rho_x = r[1];
    out->rho_z = r[2];
    out->n_x = (int32_t)r[3];
    out->n_z = (int32_t)r[4];
    const double nrm = std::sqrt(na);
    for (int q = 0; q < 3; ++q) out->axis[q] = a.axis[q] / nrm;
    const double a1 = 5.0 * std::sqrt(2.0) / 8.0, omega = -s->p.U0, k = s->p.k;
    out->d0_star = (1.0 - (1.0 - k) * omega) / k * a1 / s->p.lambda;
    out->sigma_star = (v_tip > 0.0 && std::isfinite(r[0])) ? 2.0 * s->p.D * out->d0_star / (r[0] * r[0] * v_tip) : NAN;
    return PF_OK;
}

int pf_set_fields(pf_sim* s, const void* psi_host, const void* U_host) {
    if (!s || (!psi_host && !U_host)) return PF_ERR_INVALID;
    const bool cmp = s->p.precision == PF_F32C;  // FP64 host arrays, split from the free level
    const int cur = (int)(s->step & 1), dst = cmp ? cur ^ 1 : cur;
    const size_t b = s->L.N * s->L.esz;
    if (psi_host) CK(cudaMemcpyAsync(s->psi[dst], psi_host, b, cudaMemcpyHostToDevice, s->st));
    if (U_host) CK(cudaMemcpyAsync(s->U[dst], U_host, b, cudaMemcpyHostToDevice, s->st));
    if (cmp) CK(split_into_current(s, psi_host != nullptr, U_host != nullptr));
    CK(cudaStreamSynchronize(s->st));
    return PF_OK;
}

int pf_set_fields_async(pf_sim* s, const void* psi_host, const void* U_host) {
    if (!s || (!psi_host && !U_host)) return PF_ERR_INVALID;
    const bool cmp = s->p.precision == PF_F32C;
    const int cur = (int)(s->step & 1), dst = cmp ? cur ^ 1 : cur;
    const size_t b = s->L.N * s->L.esz;
    if (psi_host) CK(cudaMemcpyAsync(s->psi[dst], psi_host, b, cudaMemcpyHostToDevice, s->st));
    if (U_host) CK(cudaMemcpyAsync(s->U[dst], U_host, b, cudaMemcpyHostToDevice, s->st));
    if (cmp) CK(split_into_current(s, psi_host != nullptr, U_host != nullptr));
    return PF_OK;
}

int pf_get_fields_async(pf_sim* s, void* psi_host, void* U_host) {
    if (!s || (!psi_host && !U_host)) return PF_ERR_INVALID;
    int cur = (int)(s->step & 1);
    const size_t b = s->L.N * s->L.esz;
    if (s->p.precision == PF_F32C) {
        CK(join_current(s, psi_host != nullptr, U_host != nullptr));
        cur ^= 1;
    }
    if (psi_host) CK(cudaMemcpyAsync(psi_host, s->psi[cur], b, cudaMemcpyDeviceToHost, s->st));
    if (U_host) CK(cudaMemcpyAsync(U_host, s->U[cur], b, cudaMemcpyDeviceToHost, s->st));
    return PF_OK;
}

int pf_synchronize(pf_sim* s) {
    if (!s) return PF_ERR_INVALID;
    CK(cudaStreamSynchronize(s->st));
    return PF_OK;
}

int pf_get_step(pf_sim* s, int64_t* step) {
    if (!s || !step) return PF_ERR_INVALID;
    *step = s->step;
    return PF_OK;
}

int pf_set_step(pf_sim* s, int64_t step) {
    if (!s || step < 0) return PF_ERR_INVALID;
    if (s->group) return PF_ERR_STATE;
    if ((step & 1) != (s->step & 1)) {
        // keep the current fields where the new counter expects them
        const int from = (int)(s->step & 1), to = from ^ 1;
        const size_t b = s->L.N * s->L.esz;
        CK(cudaMemcpyAsync(s->psi[to], s->psi[from], b, cudaMemcpyDeviceToDevice, s->st));
        CK(cudaMemcpyAsync(s->U[to], s->U[from], b, cudaMemcpyDeviceToDevice, s->st));
        CK(cudaStreamSynchronize(s->st));
    }
    s->step = step;
    std::fill(s->have_prev.begin(), s->have_prev.end(), 0);
    return PF_OK;
}

int pf_shift_frame(pf_sim* s, int rows) {
    if (!s || rows <= 0 || rows >= s->p.ny || s->p.precision == PF_F32C) return PF_ERR_INVALID;
    if (s->group) return PF_ERR_STATE;
    if (s->p.thermal == PF_FROZEN_GRADIENT) {
        // the moved frame must pass the creation checks (F1 = 1 - (1-k) zeta >= 0.05 over the grid,
        // explicit step stable at 1 / F1min) at the current step; zeta only falls later
        pf_params q = s->p;
        q.yT = s->p.yT - rows * s->p.h + s->p.Vp * s->p.dt * (double)s->step;
        if (!valid_params(&q)) return PF_ERR_INVALID;
    }
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.dim == 3 ? s->p.nz : 1;
    const int cur = (int)(s->step & 1), oth = cur ^ 1;
    const int kind = s->p.precision == PF_F64 ? 1 : 0;
    const size_t b = s->L.N * s->L.esz;
    // grain index through the free U buffer (N int16 fit in N field values)
    CK(launch_shift_rows(2, s->grain, s->U[oth], nx, ny, nz, rows, 0, 0.0, 0.0, s->st));
    CK(cudaMemcpyAsync(s->grain, s->U[oth], s->L.N * sizeof(int16_t), cudaMemcpyDeviceToDevice, s->st));
    // psi continues as a signed distance into the melt; U continues the steady far field of the
    // moving frame, U0 + C exp(-Vp y / D) (Vp = 0, isothermal: the last row, a zero-gradient far field)
    const double vp = s->p.thermal == PF_FROZEN_GRADIENT ? s->p.Vp : 0.0;
    CK(launch_shift_rows(kind, s->psi[cur], s->psi[oth], nx, ny, nz, rows, 1, -s->p.h, 0.0, s->st));
    CK(launch_shift_rows(kind, s->U[cur], s->U[oth], nx, ny, nz, rows, vp > 0.0 ? 3 : 0, s->p.U0,
                         vp * s->p.h / s->p.D, s->st));
    CK(cudaMemcpyAsync(s->psi[cur], s->psi[oth], b, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(s->U[cur], s->U[oth], b, cudaMemcpyDeviceToDevice, s->st));
    // the frame moved up by rows h: the isotherms sit rows h lower in it
    s->p.yT -= rows * s->p.h;
    InstRec r = make_rec(s, 0);
    CK(cudaMemcpyAsync(s->rec, &r, sizeof(r), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    // remembered tip positions follow the frame, so the next V is continuous,
    // and so do the grains' reference points, so growth angles are unchanged
    for (size_t slot = 0; slot < s->have_prev.size(); ++slot) s->prev[4 * slot + 2] -= rows * s->p.h;
    for (int g = 0; g < s->n_grains; ++g) s->centres_h[3 * g + 1] -= rows * s->p.h;
    return PF_OK;
}

int pf_device_fields(pf_sim* s, void** psi, void** U, void** grain) {
    if (!s) return PF_ERR_INVALID;
    const int cur = (int)(s->step & 1);
    if (psi) *psi = s->psi[cur];
    if (U) *U = s->U[cur];
    if (grain) *grain = s->grain;
    return PF_OK;
}

int pf_set_tile(pf_sim* s, int block_x, int block_y, int sweep) {
    if (!s) return PF_ERR_INVALID;
    if (s->group) return PF_ERR_STATE;
    const int obx = s->bx, oby = s->by, osw = s->sweep;
    if (block_x) s->bx = block_x;
    if (block_y) s->by = block_y;
    if (sweep) s->sweep = sweep;
    bool ok = s->sweep >= 8 && s->sweep <= 1 << 20 && occupancy(s) > 0;
    if (ok) {
        std::vector<WorkItem> tmp;
        build_work(s, 0, tmp);
        ok = (int)tmp.size() <= s->L.max_work;
    }
    if (!ok) {
        s->bx = obx;
        s->by = oby;
        s->sweep = osw;
        return PF_ERR_INVALID;
    }
    return upload_work(s);
}

int pf_get_tile(pf_sim* s, int* block_x, int* block_y, int* sweep) {
    if (!s) return PF_ERR_INVALID;
    if (block_x) *block_x = s->bx;
    if (block_y) *block_y = s->by;
    if (sweep) *sweep = s->sweep;
    return PF_OK;
}

int pf_debug_bounds(unsigned long long* failures, int* first_line) {
    if (!failures || !first_line) return PF_ERR_INVALID;
    unsigned long long c[3] = {0, 0, 0};
    int l[3] = {0, 0, 0};
    const int r0 = bounds_step2d(&c[0], &l[0]);
    const int r1 = bounds_step3d(&c[1], &l[1]);
    const int r2 = bounds_observe(&c[2], &l[2]);
    if (r0 < 0 || r1 < 0 || r2 < 0) return PF_ERR_CUDA;
    *failures = c[0] + c[1] + c[2];
    *first_line = l[0] ? l[0] : (l[1] ? l[1] : l[2]);
    return (r0 == 1 && r1 == 1 && r2 == 1) ? PF_ERR_STATE : PF_OK;
}

int pf_debug_inject_launch_failure(long long after_steps) {
    g_inject.store(after_steps < 0 ? -1 : after_steps);
    return PF_OK;
}

int pf_resident_units(pf_sim* s) {
    if (!s) return PF_ERR_INVALID;
    const int occ = occupancy(s);
    return occ > 0 ? occ * num_sms() : PF_ERR_INVALID;
}

int pf_destroy(pf_sim* s) {
    if (!s) return PF_ERR_INVALID;
    if (s->group) return PF_ERR_STATE;
    cudaStreamSynchronize(s->st);
    delete s;
    return PF_OK;
}

const char* pf_status_string(int code) {
    switch (code) {
        case PF_OK: return "ok";
        case PF_ERR_INVALID: return "invalid argument";
        case PF_ERR_BUDGET: return "device buffer too small";
        case PF_ERR_CUDA: return "CUDA error";
        case PF_ERR_NONFINITE: return "non-finite values in the fields";
        case PF_ERR_TIMEOUT: return "device wait timed out";
        case PF_ERR_STATE: return "call not valid in this state";
        default: return "unknown status";
    }
}

const char* pf_last_cuda_error(void) { return g_last_cuda.c_str(); }

int pf_observe_fields_noalloc(const pf_params* p, const void* psi_dev, const void* U_dev, const int16_t* grain_dev,
                              const double* rot9, const double* centre3, int grain, void* stream, pf_obs* out) {
    if (!p || !psi_dev || !U_dev || !rot9 || !centre3 || !out || grain < -2) return PF_ERR_INVALID;
    if (grain >= 0 && !grain_dev) return PF_ERR_INVALID;
    if (p->dim != 2 && p->dim != 3) return PF_ERR_INVALID;
    if (p->precision != PF_F32 && p->precision != PF_F64) return PF_ERR_INVALID;
    if (p->nx < 1 || p->ny < 1 || (p->dim == 3 && p->nz < 1) || !(p->h > 0) || !(p->k > 0 && p->k < 1))
        return PF_ERR_INVALID;
    const long long N = (long long)p->nx * p->ny * (p->dim == 3 ? p->nz : 1);
    if (N > PF_NOALLOC_MAX_CELLS) return PF_ERR_INVALID;
    const int dim = p->dim;
    // growth axis as in pf_observe: the crystal axis with the largest +y
    // component, or +y itself for grain -2 (the pulling axis)
    double d[3] = {0, 0, 0}, best = -INFINITY;
    if (grain == -2) {
        d[1] = 1.0;
    } else {
        for (int a = 0; a < dim; ++a)
            for (int sg = 1; sg >= -1; sg -= 2) {
                const double yc = sg * rot9[3 + a];
                if (yc > best) {
                    best = yc;
                    for (int q = 0; q < 3; ++q) d[q] = q < dim ? sg * rot9[q * 3 + a] : 0.0;
                }
            }
    }
    int ea = 0;
    for (int a = 1; a < dim; ++a)
        if (std::fabs(d[a]) > std::fabs(d[ea])) ea = a;
    ObsArgs a{};
    a.psi = psi_dev;
    a.U = U_dev;
    a.grain = grain_dev;
    a.prec = p->precision == PF_F64 ? 1 : 0;
    a.dim = dim;
    a.nx = p->nx;
    a.ny = p->ny;
    a.nz = dim == 3 ? p->nz : 1;
    a.grain_filter = grain < 0 ? -1 : grain;
    a.h = p->h;
    a.k = p->k;
    for (int q = 0; q < 3; ++q) {
        a.cg[q] = centre3[q];
        a.d[q] = d[q];
    }
    a.ea = ea;
    a.es = d[ea] >= 0 ? 1 : -1;
    ObsPartial* partials = nullptr;
    ObsPartial* result = nullptr;
    CK(noalloc_scratch(&partials, &result));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(launch_observe(a, partials, result, st));
    ObsPartial r;
    CK(cudaMemcpyAsync(&r, result, sizeof(r), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::memset(out, 0, sizeof(*out));
    const double hd = dim == 3 ? p->h * p->h * p->h : p->h * p->h;
    out->solute = r.solute * hd;
    out->solid_fraction = r.solid / (double)N;
    out->nonfinite = (int32_t)r.nonfinite;
    out->found = r.tip_index >= 0 ? 1 : 0;
    out->tip_index = r.tip_index;
    out->tip_score = r.tip_index >= 0 ? r.score : -INFINITY;
    if (r.tip_index >= 0) {
        for (int q = 0; q < 3; ++q) out->tip[q] = r.tip[q];
        const double rx = r.tip[0] - centre3[0], ry = r.tip[1] - centre3[1], rz = dim == 3 ? r.tip[2] - centre3[2] : 0.0;
        out->angle_xy_deg = std::atan2(-rx, ry) * (180.0 / 3.14159265358979323846);
        out->angle_out_deg = std::atan2(rz, std::sqrt(rx * rx + ry * ry)) * (180.0 / 3.14159265358979323846);
    } else {
        out->tip[0] = out->tip[1] = out->tip[2] = NAN;
        out->angle_xy_deg = out->angle_out_deg = NAN;
    }
    return r.nonfinite > 0 ? PF_ERR_NONFINITE : PF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// groups
// ---------------------------------------------------------------------------
struct pf_group {
    int max_inst, max_work;
    cudaStream_t st;
    char* base;
    InstRec* recs;
    WorkItem* work;
    std::vector<pf_sim*> members;
    int64_t launches;
    bool dirty;
    struct Cls {
        int dim, scheme, prec, bx, by, w0, n, grid;
        int ds;    // 2D kernel variant (ds_of: 0 isothermal T1, 1 frozen temperature / periodic x, 2 isothermal T0)
        bool two;  // two-kernel form: the psi pass, then the U pass
        int occ;   // resident units per SM
        std::vector<int> boff;  // depth 2: work items of band b are [w0 + boff[b], w0 + boff[b + 1])
    };
    std::vector<Cls> classes;
    std::vector<int64_t> gens;  // members' record generations at the last rebuild
    // temporal blocking (pf_group_set_depth): the setting, and whether the
    // current members step as depth-2 wavefronts over n_bands bands
    int depth, band_sweeps;
    bool wave;
    int n_bands;
    // step counter of frozen-temperature members: member m is at step
    // step_base[m] + *clock; the clock is advanced on the device after every
    // launch (also inside captured graphs) when any member is thermal
    long long* clock;
    long long* step_base;
    ObsPartial* obs;  // one reduced observe record per member slot
    ObsJob* jobs;     // observe arguments of every member (pf_group_observe)
    bool thermal_any;
    cudaGraphExec_t graph;
    int graph_len;
    int graph_parity;
};

namespace {

int group_rebuild(pf_group* g) {
    std::vector<InstRec> recs;
    std::vector<WorkItem> work;
    g->classes.clear();
    // sort members into classes
    std::vector<int> order(g->members.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    auto key = [&](int i) {
        const pf_sim* s = g->members[i];
        return ((long long)s->p.kernels << 52) | ((long long)ds_of(s->p) << 48) | ((long long)s->p.dim << 40) |
               ((long long)s->p.scheme << 32) |
               ((long long)s->p.precision << 24) | ((long long)s->bx << 12) | (long long)s->by;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key(a) < key(b); });
    g->gens.clear();
    for (size_t m = 0; m < g->members.size(); ++m) {
        const pf_sim* s = g->members[m];
        recs.push_back(make_rec(s, (int)((s->step ^ g->launches) & 1)));
        g->gens.push_back(s->rec_gen);
    }
    long long prev = -1;
    // depth 2 applies when no member has a frozen temperature or the
    // two-kernel form; a band must be at least two rows high (the psi halo),
    // which sweeps of at least 8 rows already guarantee
    g->wave = g->depth == 2;
    for (const pf_sim* s : g->members)
        if (s->p.thermal == PF_FROZEN_GRADIENT || s->p.kernels == PF_TWO_KERNELS || (long long)g->band_sweeps * s->sweep < 2)
            g->wave = false;
    g->n_bands = 0;
    std::vector<int> band_of;  // depth 2: band of every work item, in work order
    for (int i : order) {
        const pf_sim* s = g->members[i];
        const long long k = key(i);
        if (k != prev) {
            pf_group::Cls c{s->p.dim, s->p.scheme, kprec(s->p), s->bx, s->by, (int)work.size(), 0, 0,
                            ds_of(s->p), s->p.kernels == PF_TWO_KERNELS, 0, {}};
            g->classes.push_back(c);
            prev = k;
        }
        const size_t first = work.size();
        build_work(s, i, work);
        g->classes.back().n = (int)work.size() - g->classes.back().w0;
        if (g->wave)
            for (size_t w = first; w < work.size(); ++w) {
                const int c0 = s->p.dim == 2 ? work[w].y0 : work[w].z0;
                band_of.push_back(c0 / s->sweep / g->band_sweeps);
                g->n_bands = std::max(g->n_bands, band_of.back() + 1);
            }
    }
    if ((int)work.size() > g->max_work) return PF_ERR_BUDGET;
    if (g->wave) {
        // each class's items ordered by band (stable: members, then rows, then columns within a band)
        for (auto& c : g->classes) {
            std::vector<int> idx(c.n);
            for (int j = 0; j < c.n; ++j) idx[j] = j;
            std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return band_of[c.w0 + a] < band_of[c.w0 + b]; });
            std::vector<WorkItem> sorted(c.n);
            for (int j = 0; j < c.n; ++j) sorted[j] = work[c.w0 + idx[j]];
            std::copy(sorted.begin(), sorted.end(), work.begin() + c.w0);
            c.boff.assign(g->n_bands + 1, 0);
            for (int j = 0; j < c.n; ++j) ++c.boff[band_of[c.w0 + j] + 1];
            for (int b = 0; b < g->n_bands; ++b) c.boff[b + 1] += c.boff[b];
        }
    }
    for (auto& c : g->classes) {
        int occ = c.dim == 3 ? occupancy_step3d(c.prec, c.scheme, c.bx, c.by)
                  : c.two    ? std::min(occupancy_step2d(c.prec, c.scheme, c.bx, c.ds, 1),
                                        occupancy_step2d(c.prec, c.scheme, c.bx, c.ds, 2))
                             : occupancy_step2d(c.prec, c.scheme, c.bx, c.ds);
        if (occ <= 0) return PF_ERR_INVALID;
        c.occ = occ;
        c.grid = std::min(c.n, occ * num_sms());
    }
    if (!recs.empty()) CK(cudaMemcpyAsync(g->recs, recs.data(), recs.size() * sizeof(InstRec), cudaMemcpyHostToDevice, g->st));
    g->thermal_any = false;
    std::vector<long long> steps(g->members.size() + 1, 0);  // [0] = clock, then the step of each member
    for (size_t m = 0; m < g->members.size(); ++m) {
        steps[m + 1] = g->members[m]->step;
        if (g->members[m]->p.thermal == PF_FROZEN_GRADIENT) g->thermal_any = true;
    }
    CK(cudaMemcpyAsync(g->clock, steps.data(), steps.size() * sizeof(long long), cudaMemcpyHostToDevice, g->st));
    if (!work.empty()) CK(cudaMemcpyAsync(g->work, work.data(), work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, g->st));
    CK(cudaStreamSynchronize(g->st));
    if (g->graph) {
        cudaGraphExecDestroy(g->graph);
        g->graph = nullptr;
    }
    g->dirty = false;
    return PF_OK;
}

bool group_launch_once(pf_group* g, int launch_parity) {
    const StepClock clk{g->clock, g->step_base, 0};
    for (const auto& c : g->classes) {
        if (c.n == 0) continue;
        bool ok;
        if (c.dim == 3)
            ok = launch_step3d(c.prec, c.scheme, c.bx, c.by, c.grid, g->st, g->work + c.w0, c.n, g->recs, launch_parity,
                               clk);
        else if (c.two)
            ok = launch_step2d(c.prec, c.scheme, c.bx, c.grid, g->st, g->work + c.w0, c.n, g->recs, launch_parity, clk,
                               c.ds, 1) &&
                 launch_step2d(c.prec, c.scheme, c.bx, c.grid, g->st, g->work + c.w0, c.n, g->recs, launch_parity, clk,
                               c.ds, 2);
        else
            ok = launch_step2d(c.prec, c.scheme, c.bx, c.grid, g->st, g->work + c.w0, c.n, g->recs, launch_parity, clk,
                               c.ds);
        if (!ok) return false;
    }
    if (g->thermal_any && launch_tick(g->clock, g->st) != cudaSuccess) return false;
    return true;
}

// the work items of band b of every class at one launch parity (depth 2;
// fused kernels only, no frozen temperature: the step clock is not read)
bool group_launch_band(pf_group* g, int launch_parity, int b) {
    const StepClock clk{g->clock, g->step_base, 0};
    for (const auto& c : g->classes) {
        const int lo = c.boff[b], cnt = c.boff[b + 1] - lo;
        if (cnt <= 0) continue;
        const int grid = std::min(cnt, c.occ * num_sms());
        const bool ok = c.dim == 3 ? launch_step3d(c.prec, c.scheme, c.bx, c.by, grid, g->st, g->work + c.w0 + lo, cnt,
                                                   g->recs, launch_parity, clk)
                                   : launch_step2d(c.prec, c.scheme, c.bx, grid, g->st, g->work + c.w0 + lo, cnt,
                                                   g->recs, launch_parity, clk, c.ds);
        if (!ok) return false;
    }
    return true;
}

// two steps as one wavefront over the bands, starting at launch parity lp
bool group_launch_pair(pf_group* g, int lp) {
    const int m = 2 * g->n_bands;
    std::vector<int> level(m), band(m);
    pf_wavefront_order(g->n_bands, level.data(), band.data(), m);
    for (int i = 0; i < m; ++i)
        if (!group_launch_band(g, lp ^ level[i], band[i])) return false;
    return true;
}

}  // namespace

extern "C" {

size_t pf_group_required_bytes(int max_instances, int max_work) {
    if (max_instances < 1 || max_work < 1) return 0;
    return align256((size_t)max_instances * sizeof(InstRec)) + align256((size_t)max_work * sizeof(WorkItem)) +
           align256((size_t)(max_instances + 1) * sizeof(long long)) +
           align256((size_t)max_instances * sizeof(ObsPartial)) + align256((size_t)max_instances * sizeof(ObsJob));
}

int pf_wavefront_order(int n_bands, int* level, int* band, int cap) {
    if (n_bands < 1 || cap < 0 || (cap > 0 && (!level || !band))) return PF_ERR_INVALID;
    int n = 0;
    auto put = [&](int l, int b) {
        if (n < cap) {
            level[n] = l;
            band[n] = b;
        }
        ++n;
    };
    // step n+1 runs one band ahead of step n+2
    for (int b = 0; b <= n_bands; ++b) {
        if (b < n_bands) put(0, b);
        if (b >= 1) put(1, b - 1);
    }
    return n;
}

int pf_group_set_depth(pf_group* g, int depth, int band_sweeps) {
    if (!g || depth < 1 || depth > 2 || band_sweeps < 1) return PF_ERR_INVALID;
    if (depth != g->depth || band_sweeps != g->band_sweeps) {
        g->depth = depth;
        g->band_sweeps = band_sweeps;
        g->dirty = true;
    }
    return PF_OK;
}

int pf_group_get_depth(pf_group* g, int* depth, int* band_sweeps, int* effective) {
    if (!g) return PF_ERR_INVALID;
    if (g->dirty && !g->members.empty()) {
        const int rc = group_rebuild(g);
        if (rc != PF_OK) return rc;
    }
    if (depth) *depth = g->depth;
    if (band_sweeps) *band_sweeps = g->band_sweeps;
    if (effective) *effective = (g->wave && !g->members.empty()) ? 2 : 1;
    return PF_OK;
}

int pf_group_work_items(const pf_sim* s) {
    if (!s) return PF_ERR_INVALID;
    std::vector<WorkItem> tmp;
    build_work(s, 0, tmp);
    return (int)tmp.size();
}

int pf_group_create(int max_instances, int max_work, void* dev_mem, size_t bytes, void* stream, pf_group** out) {
    if (!out) return PF_ERR_INVALID;
    *out = nullptr;
    if (max_instances < 1 || max_work < 1 || !dev_mem || ((uintptr_t)dev_mem & 255)) return PF_ERR_INVALID;
    if (bytes < pf_group_required_bytes(max_instances, max_work)) return PF_ERR_BUDGET;
    pf_group* g = new (std::nothrow) pf_group();
    if (!g) return PF_ERR_INVALID;
    g->max_inst = max_instances;
    g->max_work = max_work;
    g->st = static_cast<cudaStream_t>(stream);
    g->base = static_cast<char*>(dev_mem);
    g->recs = reinterpret_cast<InstRec*>(g->base);
    g->work = reinterpret_cast<WorkItem*>(g->base + align256((size_t)max_instances * sizeof(InstRec)));
    g->clock = reinterpret_cast<long long*>(g->base + align256((size_t)max_instances * sizeof(InstRec)) +
                                            align256((size_t)max_work * sizeof(WorkItem)));
    g->step_base = g->clock + 1;
    g->obs = reinterpret_cast<ObsPartial*>(reinterpret_cast<char*>(g->clock) +
                                           align256((size_t)(max_instances + 1) * sizeof(long long)));
    g->jobs = reinterpret_cast<ObsJob*>(reinterpret_cast<char*>(g->obs) +
                                        align256((size_t)max_instances * sizeof(ObsPartial)));
    g->thermal_any = false;
    g->depth = 1;
    g->band_sweeps = 1;
    g->wave = false;
    g->n_bands = 0;
    g->launches = 0;
    g->dirty = true;
    g->graph = nullptr;
    g->graph_len = 0;
    g->graph_parity = 0;
    *out = g;
    return PF_OK;
}

int pf_group_add(pf_group* g, pf_sim* s) {
    if (!g || !s) return PF_ERR_INVALID;
    if (s->group) return PF_ERR_STATE;
    if ((int)g->members.size() >= g->max_inst) return PF_ERR_BUDGET;
    if (s->work_dirty) {
        int rc = upload_work(s);
        if (rc != PF_OK) return rc;
    }
    CK(cudaStreamSynchronize(s->st));
    g->members.push_back(s);
    s->group = g;
    g->dirty = true;
    return PF_OK;
}

int pf_group_remove(pf_group* g, pf_sim* s) {
    if (!g || !s || s->group != g) return PF_ERR_INVALID;
    CK(cudaStreamSynchronize(g->st));
    g->members.erase(std::find(g->members.begin(), g->members.end(), s));
    s->group = nullptr;
    g->dirty = true;
    return PF_OK;
}

int pf_group_step(pf_group* g, int64_t n, int use_graph) {
    if (!g || n < 0) return PF_ERR_INVALID;
    if (g->members.empty() || n == 0) return PF_OK;
    // a member whose grains changed since the last rebuild needs a new record
    for (size_t m = 0; m < g->members.size() && !g->dirty; ++m)
        if (m >= g->gens.size() || g->members[m]->rec_gen != g->gens[m]) g->dirty = true;
    if (g->dirty) {
        int rc = group_rebuild(g);
        if (rc != PF_OK) return rc;
    }
    int64_t done = 0;
    const int GL = 16;  // steps per graph replay (even)
    // on a failure the group and its members advance by the `done` steps launched
    auto stop = [&](int rc) {
        g->launches += done;
        for (pf_sim* s : g->members) s->step += done;
        return rc;
    };
    // the legacy default stream cannot be captured into a graph
    if (use_graph && n >= GL && g->st != nullptr && g->st != cudaStreamPerThread) {
        if ((g->launches & 1) != 0) {
            if (inject_hits(1)) return stop(PF_ERR_CUDA);
            if (!group_launch_once(g, 1)) return stop(PF_ERR_INVALID);
            ++done;
        }
        if (!g->graph) {
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(g->st, cudaStreamCaptureModeThreadLocal));
            bool ok = true;
            if (g->wave)
                for (int i = 0; i < GL && ok; i += 2) ok = group_launch_pair(g, 0);
            else
                for (int i = 0; i < GL && ok; ++i) ok = group_launch_once(g, i & 1);
            cudaError_t e = cudaStreamEndCapture(g->st, &graph);
            if (!ok) return PF_ERR_INVALID;
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&g->graph, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
            g->graph_len = GL;
        }
        while (n - done >= GL) {
            if (inject_hits(GL)) return stop(PF_ERR_CUDA);
            const cudaError_t e = cudaGraphLaunch(g->graph, g->st);
            if (e != cudaSuccess) return stop(cuda_fail(e, "cudaGraphLaunch"));
            done += GL;
        }
    }
    if (g->wave)
        for (; n - done >= 2; done += 2) {
            if (inject_hits(2)) return stop(PF_ERR_CUDA);
            if (!group_launch_pair(g, (int)((g->launches + done) & 1))) return stop(PF_ERR_INVALID);
        }
    for (; done < n; ++done) {
        if (inject_hits(1)) return stop(PF_ERR_CUDA);
        if (!group_launch_once(g, (int)((g->launches + done) & 1))) return stop(PF_ERR_INVALID);
    }
    CK(cudaGetLastError());
    g->launches += n;
    for (pf_sim* s : g->members) s->step += n;
    return PF_OK;
}

int pf_group_size(const pf_group* g) { return g ? (int)g->members.size() : PF_ERR_INVALID; }

int pf_group_observe(pf_group* g, int grain, pf_obs* out) {
    if (!g || !out || grain < -2) return PF_ERR_INVALID;
    for (pf_sim* s : g->members)
        if (grain >= s->n_grains) return PF_ERR_INVALID;
    const size_t n = g->members.size();
    if (n == 0) return PF_OK;
    std::vector<ObsJob> jobs(n);
    for (size_t i = 0; i < n; ++i) {
        pf_sim* s = g->members[i];
        // the member's fields are current on the group's stream (compensated
        // members are joined there); its partials are its own, the reduced
        // record goes to the group's slot i
        const cudaStream_t keep = s->st;
        s->st = g->st;
        const int rc = observe_args(s, grain, jobs[i].a);
        s->st = keep;
        if (rc != PF_OK) return rc;
        jobs[i].partials = s->partials;
    }
    CK(cudaMemcpyAsync(g->jobs, jobs.data(), n * sizeof(ObsJob), cudaMemcpyHostToDevice, g->st));
    CK(launch_observe_multi(g->jobs, (int)n, g->obs, g->st));
    std::vector<ObsArgs> args(n);
    for (size_t i = 0; i < n; ++i) args[i] = jobs[i].a;
    std::vector<ObsPartial> r(n);
    CK(cudaMemcpyAsync(r.data(), g->obs, n * sizeof(ObsPartial), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    int status = PF_OK;
    for (size_t i = 0; i < n; ++i)
        if (observe_finish(g->members[i], grain, args[i], r[i], out + i) != PF_OK) status = PF_ERR_NONFINITE;
    return status;
}

int pf_group_destroy(pf_group* g) {
    if (!g) return PF_ERR_INVALID;
    cudaStreamSynchronize(g->st);
    for (pf_sim* s : g->members) s->group = nullptr;
    if (g->graph) cudaGraphExecDestroy(g->graph);
    delete g;
    return PF_OK;
}

}  // extern "C"
