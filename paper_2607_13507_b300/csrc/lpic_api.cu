// lpic_api.cu -- host side of liblpic: the C ABI declared in include/lpic.h.
// Descriptor checks, scratch ownership, the fixed-point shift, and the
// launches of the Maxwell, sort, particle and diagnostic kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "lpic.h"
#include "lpic_common.cuh"
#include "lpic_diag.cuh"
#include "lpic_ensemble.cuh"
#include "lpic_field.cuh"
#include "lpic_fp32.cuh"
#include "lpic_fp64.cuh"
#include "lpic_gpd32.h"
#include "lpic_qed.cuh"
#include "lpic_sort.cuh"

using namespace lpic;

namespace {

thread_local std::string g_err;

lpic_status fail(lpic_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define LPIC_CUDA(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return fail(LPIC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// every kernel launch site has the grid `g` in scope and counts the launch
#define LPIC_LAUNCHED(what)                                                               \
    do {                                                                                  \
        ++g->launches;                                                                    \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess) return fail(LPIC_ECUDA, "launch %s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

// Every device allocation of the library goes through dev_alloc, so that
// a test can make the n-th one fail as if the device were out of memory
// (lpic_debug_fail_alloc) and check that each call unwinds and reports
// LPIC_ENOMEM.
std::atomic<long long> g_alloc_fail_at{0};    // 0: off
std::atomic<long long> g_alloc_seen{0};

template <class T>
cudaError_t dev_alloc(T** p, size_t bytes) {
    const long long k = g_alloc_fail_at.load();
    if (k > 0 && g_alloc_seen.fetch_add(1) + 1 == k) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

struct Species {
    double q = 0, m = 1;
    long long cap = 0;
    long long sort_gen = 0;      // sorts so far (the particle order changes with each)
    long long gather_gen = -1;   // sort_gen at the last unfused gather stage
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    int* d_n = nullptr;          // particles in the current buffer
    int* d_count = nullptr;      // ntiles + 1
    int* d_start = nullptr;      // ntiles + 2
    int* d_cursor = nullptr;     // ntiles + 1
    int* d_coff = nullptr;       // ntiles + 1 work-item offsets
    int2* d_items = nullptr;     // work items (tile, chunk)
    int* d_nitems = nullptr;
    int* d_esc = nullptr;        // particles beyond their tile's margin (capacity)
    int* d_nesc = nullptr;
    long long item_cap = 0;
    long long count0 = 0;        // particles at add time
    double wmax = 0;
    bool sorted = false;         // sorted at least once
    int since_sort = 1 << 30;    // pushes since the last sort
    bool counts_fresh = false;   // d_count holds the histogram of the current cells
    bool massless = false;       // m = 0, q = 0: moves at c along u, no fields, no current
    // nonlinear Compton emission inside this species' push (lpic_qed_fuse)
    int q_ph = -1;               // photon species (-1: off)
    float* q_tau = nullptr;
    long long q_nids = 0;
    float* q_phtau = nullptr;
    long long q_phnids = 0;
};

}  // namespace

namespace lpic {
// Lets the other translation units of the library report through lpic_last_error.
__attribute__((visibility("hidden"))) void set_last_error(const char* msg) { g_err = msg; }
}  // namespace lpic

struct lpic_grid {
    lpic_grid_desc d{};
    Laser laser{};
    Geo geo{};
    int T[3] = {1, 1, 1}, nt[3] = {1, 1, 1};
    long long ntiles = 1;
    long long nfield = 0;        // fx * ny * nz
    int F = 0;
    double jscale[3] = {0, 0, 0}, rho_scale = 0;
    std::vector<Species> sp;
    unsigned* d_status = nullptr;
    void* d_mur = nullptr;
    double* d_lprof = nullptr;   // transverse laser profile on the x-min plane
    int cpml = 0;                // CPML layers (absorb_x = 2)
    void* d_psi = nullptr;       // CPML memory: 4 x plane x (2 L + 2) field-precision values
    void* d_pcoef = nullptr;     // CPML coefficients: 1/kappa, a, b at nodes and half nodes (6 x fx)
    double* d_acc = nullptr;
    unsigned long long* d_cnt = nullptr;
    bool started = false;
    int nsm = 0;                 // SMs of the device (queried at create)
    size_t smem32 = 0;
    long long launches = 0;
    int P = 4096;                              // particles per work item (FP32 path)
    int K = 1;                                 // sort interval (steps)
    int m[3] = {0, 0, 0};                      // drift margin of the tiles (cells)
    CellDecode dec{};
    FastDiv fT[3]{};
    double* d_clock = nullptr;                 // device time for graph replays
    // captured steps keyed by every species' buffer parity and sort state
    std::map<unsigned long long, cudaGraphExec_t> graphs;
    std::map<unsigned long long, long long> graph_launches;
    // optional timing of the fused particle kernel (benchmarks)
    bool timing = false;
    std::vector<cudaEvent_t> ev;               // pairs (start, stop)
    size_t ev_used = 0;
    bool attrs_set = false;
    // nonlinear Compton emission (lpic_qed_init)
    bool qed = false;
    double eps_ref = 0;
    uint32_t seed[2] = {0, 0};
    QedTab qtab{};
    float* d_qtab = nullptr;                   // logh | top | cdf
    BwTab btab{};
    float* d_btab = nullptr;                   // g | cdf (Breit-Wheeler)
    unsigned* d_qstep = nullptr;               // counter word of the fused emission (lpic_qed_fuse)
};

namespace {

int grid_blocks(long long work, int nsm, int per_sm = 8) {
    long long b = (work + 255) / 256;
    long long cap = (long long)nsm * per_sm;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

P32 view32(const lpic_grid* g, const Species& s, int b) {
    char* base = static_cast<char*>(s.buf[b]);
    const size_t a = (size_t)s.cap * 4;
    const int dim = g->d.dim;
    P32 p{};
    p.cell = reinterpret_cast<int*>(base);
    for (int d = 0; d < 3; ++d)
        p.off[d] = reinterpret_cast<float*>(base + (1 + (d < dim ? d : dim - 1)) * a);
    for (int c = 0; c < 3; ++c) p.u[c] = reinterpret_cast<float*>(base + (1 + dim + c) * a);
    p.w = reinterpret_cast<float*>(base + (4 + dim) * a);
    p.id = reinterpret_cast<int*>(base + (5 + dim) * a);
    p.n = s.d_n;
    return p;
}

P64 view64(const lpic_grid* g, const Species& s, int b) {
    char* base = static_cast<char*>(s.buf[b]);
    const size_t a = (size_t)s.cap * 8;
    const int dim = g->d.dim;
    P64 p{};
    for (int d = 0; d < 3; ++d) p.x[d] = reinterpret_cast<double*>(base + (d < dim ? d : dim - 1) * a);
    for (int c = 0; c < 3; ++c) p.u[c] = reinterpret_cast<double*>(base + (dim + c) * a);
    p.w = reinterpret_cast<double*>(base + (dim + 3) * a);
    p.id = reinterpret_cast<int*>(base + (dim + 4) * a);
    p.n = s.d_n;
    return p;
}

template <typename T>
Ptr3<T> ptr3(void* const* v) {
    Ptr3<T> p;
    for (int c = 0; c < 3; ++c) p.p[c] = static_cast<T*>(v[c]);
    return p;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

__global__ void k_absmax_f32(const float* w, const int* n, unsigned* out) {
    unsigned m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < *n; i += gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(w[i])));
    atomicMax(out, m);
}

__global__ void k_absmax_f64(const double* w, const int* n, unsigned long long* out) {
    unsigned long long m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < *n; i += gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(fabs(w[i])));
    atomicMax(out, m);
}

// Divisors of the tile kernel's field and current boxes (T + 2m + 3 and
// T + 2m + 5 nodes per dimension).
void box_divisors(const lpic_grid* g, Tiles& t) {
    const TileSmem L = tile_smem(g->d.dim, g->T, g->m);
    t.fG0 = make_fastdiv((unsigned)L.G[0]); t.fG1 = make_fastdiv((unsigned)L.G[1]);
    t.fF = make_fastdiv((unsigned)L.fsz);
    t.fH0 = make_fastdiv((unsigned)L.H[0]); t.fH1 = make_fastdiv((unsigned)L.H[1]);
    t.fJ = make_fastdiv((unsigned)L.jsz);
}

// Bound (units of kBoundUnit) of one move's current at any node for a
// species: S b + 1024 with S = rint(2^F |q| w_max) the largest integer charge
// and b the per-move factor of move_factor().
unsigned move_bound(const lpic_grid* g, const Species& s);
// 2D: rounds of the tile kernel between folds of its int32 current boxes.
int fold_rounds(const lpic_grid_desc& d);

// Arguments of the tile kernel for one species.
GpdArgs gpd_args(lpic_grid* g, Species& s, bool count_next) {
    const P32 p = view32(g, s, s.cur);
    Tiles t{};
    for (int d = 0; d < 3; ++d) { t.T[d] = g->T[d]; t.nt[d] = g->nt[d]; t.m[d] = g->m[d]; t.fT[d] = g->fT[d]; }
    t.next_count = count_next ? s.d_count : nullptr;
    t.esc = s.d_esc;
    t.nesc = s.d_nesc;
    t.start = s.d_start;
    t.items = s.d_items;
    t.nitems = s.d_nitems;
    t.P = g->P;
    t.bmax = move_bound(g, s);
    t.R = fold_rounds(g->d);
    box_divisors(g, t);
    const float k = (float)(s.q * g->d.dt / (2.0 * s.m));
    const float sq = (float)std::ldexp(s.q, g->F);
    const bool f64 = g->d.maxwell_fp64 != 0;
    return GpdArgs{g->geo, ptr3<const float>(g->d.E), ptr3<const float>(g->d.B),
                   ptr3<const double>(g->d.E), ptr3<const double>(g->d.B), f64 ? 1 : 0,
                   ptr3<unsigned long long>(g->d.J),
                   p, t, g->dec, k, sq, (float)(g->d.dt / g->d.dx), (float)(g->d.dt / g->d.dy),
                   (float)(g->d.dt / (g->d.dim == 3 ? g->d.dz : 1.0)), g->d_status, nullptr, 0, 0, QedEmit{}};
}

// The emission state of a species with fused emission (photon buffers of the
// photon species' current parity).
QedEmit qed_emit_args(lpic_grid* g, const Species& s) {
    Species& ph = g->sp[s.q_ph];
    QedEmit q{};
    q.T = g->qtab;
    q.tau = s.q_tau;
    q.n_ids = s.q_nids;
    q.ph = view32(g, ph, ph.cur);
    q.ph_n = ph.d_n;
    q.ph_next_id = ph.d_n + 1;
    q.ph_cap = ph.cap;
    q.ph_tau = s.q_phnids > 0 ? s.q_phtau : nullptr;
    q.ph_n_ids = s.q_phnids;
    q.dt = (float)g->d.dt;
    q.k0 = g->seed[0];
    q.k1 = g->seed[1];
    q.step = g->d_qstep;
    return q;
}

// tile-kernel instance and its dynamic shared memory
template <int DIM, int ORDER>
lpic_status launch_gpd32(lpic_grid* g, Species& s, cudaStream_t st, bool count_next) {
    if (count_next) LPIC_CUDA(cudaMemsetAsync(s.d_count, 0, sizeof(int) * (g->ntiles + 1), st));
    LPIC_CUDA(cudaMemsetAsync(s.d_nesc, 0, sizeof(int), st));
    GpdArgs A = gpd_args(g, s, count_next);
    if (s.q_ph >= 0) {
        A.qed = 1;
        A.q = qed_emit_args(g, s);
        Gpd32Qed<DIM, ORDER>::tile(A, (unsigned)s.item_cap, g->smem32, st);
        LPIC_LAUNCHED("k_gpd32_qed");
    } else {
        Gpd32<DIM, ORDER>::tile(A, (unsigned)s.item_cap, g->smem32, st);
        LPIC_LAUNCHED("k_gpd32");
    }
    Gpd32<DIM, ORDER>::escape(A, (unsigned)(2 * g->nsm), st);
    LPIC_LAUNCHED("k_gpd32_escape");
    if (s.q_ph >= 0) {
        Species& ph = g->sp[s.q_ph];
        k_qed_clamp<<<1, 32, 0, st>>>(ph.d_n, ph.cap);
        LPIC_LAUNCHED("k_qed_clamp");
        ph.counts_fresh = false;
    }
    return LPIC_OK;
}

// One unfused stage (gather: fields written; else push and deposit with the
// fields read) on freshly sorted particles, which never leave their tile.
template <int DIM, int ORDER>
lpic_status launch_stage(lpic_grid* g, Species& s, cudaStream_t st, bool gather, float* fields) {
    GpdArgs A = gpd_args(g, s, false);
    A.fields = fields;
    A.fcap = s.cap;
    if (gather) Gpd32Stages<DIM, ORDER>::gather(A, (unsigned)s.item_cap, g->smem32, st);
    else        Gpd32Stages<DIM, ORDER>::push(A, (unsigned)s.item_cap, g->smem32, st);
    LPIC_LAUNCHED(gather ? "k_gpd32_gather" : "k_gpd32_fields_in");
    return LPIC_OK;
}

template <int DIM, int ORDER>
lpic_status launch_gpd64(lpic_grid* g, Species& s, cudaStream_t st) {
    const P64 p = view64(g, s, s.cur);
    k_gpd64<DIM, ORDER><<<grid_blocks(s.cap, g->nsm, 16), 256, 0, st>>>(
        g->geo, ptr3<const double>(g->d.E), ptr3<const double>(g->d.B), ptr3<double>(g->d.J), p,
        s.q * g->d.dt / (2.0 * s.m), s.q, g->d_status);
    LPIC_LAUNCHED("k_gpd64");
    return LPIC_OK;
}

template <int DIM, int ORDER>
cudaError_t set_smem_attrs(size_t bytes) {
    cudaError_t e = Gpd32<DIM, ORDER>::set_smem(bytes);
    if (e == cudaSuccess) e = Gpd32Stages<DIM, ORDER>::set_smem(bytes);
    return e != cudaSuccess ? e : Gpd32Qed<DIM, ORDER>::set_smem(bytes);
}

// clock != nullptr: the laser time is read from the device clock plus t.
template <int DIM, typename R, typename JT>
lpic_status maxwell_impl(lpic_grid* g, int half, double t, cudaStream_t st, const double* clock) {
    FieldArgs<R, JT> a{};
    for (int c = 0; c < 3; ++c) {
        a.E[c] = static_cast<R*>(g->d.E[c]);
        a.B[c] = static_cast<R*>(g->d.B[c]);
        a.J[c] = static_cast<const JT*>(g->d.J[c]);
    }
    const double tau = 0.5 * g->d.dt;
    a.rdx = (R)(1.0 / g->d.dx);
    a.rdy = (R)(1.0 / g->d.dy);
    a.rdz = (R)(DIM == 3 ? 1.0 / g->d.dz : 0.0);
    a.tau = (R)tau;
    for (int c = 0; c < 3; ++c) a.jfac[c] = tau * (g->d.precision == LPIC_FP32_FIXED ? g->jscale[c] : 1.0);
    a.dfx = make_fastdiv((unsigned)g->geo.fx);
    a.dny = make_fastdiv((unsigned)g->d.ny);
    const int nb = grid_blocks(g->nfield, g->nsm, 16);
    const int plane = g->d.ny * (DIM == 3 ? g->d.nz : 1);
    Ptr3<R> Ep;
    for (int c = 0; c < 3; ++c) Ep.p[c] = a.E[c];
    const bool mur = g->geo.absorb && !g->cpml;
    CpmlArgs<R> cp{};
    Ptr3<const R> Ec, Bc;
    for (int c = 0; c < 3; ++c) { Ec.p[c] = a.E[c]; Bc.p[c] = a.B[c]; }
    Ptr3<R> Bp;
    for (int c = 0; c < 3; ++c) Bp.p[c] = a.B[c];
    const int nbp = grid_blocks((long long)plane * (2 * g->d.pml_cells + 2), g->nsm);
    if (g->cpml) {
        const size_t W = (size_t)plane * (2 * g->d.pml_cells + 2);
        R* psi = static_cast<R*>(g->d_psi);
        const R* cf = static_cast<const R*>(g->d_pcoef);
        const size_t fx = (size_t)g->geo.fx;
        for (int k = 0; k < 4; ++k) cp.psi[k] = psi + k * W;
        for (int h = 0; h < 2; ++h) {
            cp.kinv[h] = cf + (0 + h) * fx;
            cp.a[h] = cf + (2 + h) * fx;
            cp.b[h] = cf + (4 + h) * fx;
        }
        cp.L = g->d.pml_cells;
    }
    auto updE = [&]() -> lpic_status {
        if (mur) {
            k_mur_save<R><<<grid_blocks(8LL * plane, g->nsm), 256, 0, st>>>(g->geo, Ep, static_cast<R*>(g->d_mur));
            LPIC_LAUNCHED("k_mur_save");
        }
        k_update_E<DIM, R, JT><<<nb, 256, 0, st>>>(g->geo, a);
        LPIC_LAUNCHED("k_update_E");
        if (mur) {
            k_mur_apply<R><<<grid_blocks(2LL * plane, g->nsm), 256, 0, st>>>(
                g->geo, Ep, static_cast<const R*>(g->d_mur), g->laser, g->d_lprof, t, clock, tau);
            LPIC_LAUNCHED("k_mur_apply");
        }
        if (g->cpml) {
            k_cpml_E<R><<<nbp, 256, 0, st>>>(g->geo, Ep, Bc, cp, (R)tau);
            LPIC_LAUNCHED("k_cpml_E");
            if (g->laser.on) {
                k_laser_sheet<R><<<grid_blocks(plane, g->nsm), 256, 0, st>>>(
                    g->geo, a.E[1], g->laser, g->d_lprof, g->d.pml_cells + 2, t, clock, tau);
                LPIC_LAUNCHED("k_laser_sheet");
            }
        }
        return LPIC_OK;
    };
    auto updB = [&]() -> lpic_status {
        k_update_B<DIM, R, JT><<<nb, 256, 0, st>>>(g->geo, a);
        LPIC_LAUNCHED("k_update_B");
        if (g->cpml) {
            k_cpml_B<R><<<nbp, 256, 0, st>>>(g->geo, Ec, Bp, cp, (R)tau);
            LPIC_LAUNCHED("k_cpml_B");
        }
        return LPIC_OK;
    };
    lpic_status r;
    if (half == 0) {
        if ((r = updE()) != LPIC_OK) return r;
        if ((r = updB()) != LPIC_OK) return r;
    } else {
        if ((r = updB()) != LPIC_OK) return r;
        if ((r = updE()) != LPIC_OK) return r;
    }
    return LPIC_OK;
}

// use_counts: d_count already holds the tile histogram of the current cells
// (computed by the preceding push), so the counting pass is skipped.
lpic_status sort_one(lpic_grid* g, Species& s, cudaStream_t st, bool use_counts = false) {
    const int other = 1 - s.cur;
    const int nt = (int)g->ntiles;
    if (!use_counts) LPIC_CUDA(cudaMemsetAsync(s.d_count, 0, sizeof(int) * (nt + 1), st));
    LPIC_CUDA(cudaMemsetAsync(s.d_cursor, 0, sizeof(int) * (nt + 1), st));
    const int nb = grid_blocks(s.cap, g->nsm, 16);
    const int dim = g->d.dim;
    if (g->d.precision == LPIC_FP32_FIXED) {
        const P32 src = view32(g, s, s.cur), dst = view32(g, s, other);
        KeyFP32 key{src.cell, g->dec, g->fT[0], g->fT[1], g->fT[2], g->nt[0], g->nt[1], nt};
        if (!use_counts) {
            k_sort_count<<<nb, 256, 0, st>>>(key, s.d_n, s.d_count);
            LPIC_LAUNCHED("k_sort_count");
        }
        k_sort_scan<<<1, 1024, 0, st>>>(s.d_count, s.d_start, nt, g->P, s.d_coff);
        LPIC_LAUNCHED("k_sort_scan");
        k_sort_items<<<grid_blocks(nt, g->nsm), 256, 0, st>>>(s.d_count, s.d_coff, nt, g->P, s.d_items, s.d_nitems);
        LPIC_LAUNCHED("k_sort_items");
        k_sort_scatter<<<nb, 256, 0, st>>>(key, MoveFP32{src, dst, dim}, s.d_n, s.d_start, s.d_cursor, nt);
        LPIC_LAUNCHED("k_sort_scatter");
    } else {
        const P64 src = view64(g, s, s.cur), dst = view64(g, s, other);
        KeyFP64 key{{src.x[0], src.x[1], src.x[2]}, src.w, 1.0 / g->d.dx, 1.0 / g->d.dy,
                    dim == 3 ? 1.0 / g->d.dz : 0.0, g->d.nx, g->d.ny, g->d.nz, g->T[0], g->T[1],
                    g->T[2], g->nt[0], g->nt[1], nt, dim};
        k_sort_count<<<nb, 256, 0, st>>>(key, s.d_n, s.d_count);
        LPIC_LAUNCHED("k_sort_count");
        k_sort_scan<<<1, 1024, 0, st>>>(s.d_count, s.d_start, nt, g->P, s.d_coff);
        LPIC_LAUNCHED("k_sort_scan");
        k_sort_scatter<<<nb, 256, 0, st>>>(key, MoveFP64{src, dst, dim}, s.d_n, s.d_start, s.d_cursor, nt);
        LPIC_LAUNCHED("k_sort_scatter");
    }
    k_sort_finalize<<<1, 32, 0, st>>>(s.d_start, nt, s.d_n);
    LPIC_LAUNCHED("k_sort_finalize");
    s.cur = other;
    s.sorted = true;
    s.since_sort = 0;
    s.counts_fresh = false;
    s.sort_gen += 1;
    return LPIC_OK;
}

lpic_status check_grid(lpic_grid_t g) {
    if (!g) return fail(LPIC_EINVAL, "grid is NULL");
    return LPIC_OK;
}

lpic_status check_species(lpic_grid_t g, int sid) {
    if (!g) return fail(LPIC_EINVAL, "grid is NULL");
    if (sid < 0 || sid >= (int)g->sp.size()) return fail(LPIC_EINVAL, "species id %d out of range", sid);
    return LPIC_OK;
}

// Largest current one move adds to any node, in units of the particle's
// integer charge S.  J_d along d is s (C1 - C0) K with C the running sum of
// the shape weights (|C1 - C0| <= the displacement nu <= c dt / h cells,
// since the running sum of a B-spline's weights moves with slope at most 1)
// and K the transverse factor: 2D A_y <= k, 3D A_y A_z + DS_y DS_z / 12 <=
// k^2 + 1/12 (k = 0.75 TSC, 1 CIC); 2D J_z = s v_z W_z with |v_z| < 1 and
// W_z <= k^2 + 1/12.  Roundings and closures add less than 1024 units.
double move_factor(const lpic_grid_desc& d) {
    double nu = std::max(d.dt / d.dx, d.dt / d.dy);
    if (d.dim == 3) nu = std::max(nu, d.dt / d.dz);
    nu = std::min(nu, 1.0);                     // the kernel rejects longer moves
    const double k = d.shape_order == 2 ? 0.75 : 1.0;
    double b = nu * (d.dim == 3 ? k * k + 1.0 / 12.0 : k);
    if (d.dim == 2) b = std::max(b, k * k + 1.0 / 12.0);
    return b;
}

unsigned move_bound(const lpic_grid* g, const Species& s) {
    const double S = std::rint(std::ldexp(std::fabs(s.q) * s.wmax, g->F));
    return (unsigned)std::ceil((S * move_factor(g->d) + 1024.0) / kBoundUnit) + 1u;
}

// 2D: rounds of 256 moves the int32 current boxes take between folds into
// the int64 boxes, with every particle's integer charge S <= 2^22.
int fold_rounds(const lpic_grid_desc& d) {
    const double per_move = 4194304.0 * move_factor(d) + 1024.0;
    const int R = (int)std::floor(2147483647.0 / (kGpdThreads * per_move));
    return std::max(1, std::min(R, 64));
}

void recompute_shift(lpic_grid* g) {
    double total = 0.0, mx = 0.0;
    for (const auto& s : g->sp) {
        const double b = std::fabs(s.q) * s.wmax;
        total += (double)s.cap * b;
        mx = std::max(mx, b);
    }
    if (mx <= 0.0) { g->F = 0; }
    else {
        // S <= 2^22 (float rounding of the per-particle integers), no int64
        // sum can overflow, and (3D) two deposit phases of the tile kernel
        // (256 moves each) keep the int32 current boxes in range
        const int f1 = (int)std::floor(22.0 - std::log2(mx));
        const int f2 = (int)std::floor(61.0 - std::log2(total));
        const double phase = (g->d.dim == 3 ? 2.0 : 1.0) * kGpdThreads;
        const double smax = (kBoundLimit * (double)kBoundUnit / phase - 2048.0) / move_factor(g->d);
        const int f3 = (int)std::floor(std::log2(smax) - std::log2(mx));
        g->F = std::min(f1, std::min(f2, f3));
    }
    const double u = std::ldexp(1.0, -g->F);
    const lpic_grid_desc& d = g->d;
    if (d.dim == 3) {
        g->jscale[0] = u / (d.dt * d.dy * d.dz);
        g->jscale[1] = u / (d.dt * d.dx * d.dz);
        g->jscale[2] = u / (d.dt * d.dx * d.dy);
        g->rho_scale = u / (d.dx * d.dy * d.dz);
    } else {
        g->jscale[0] = u / (d.dt * d.dy);
        g->jscale[1] = u / (d.dt * d.dx);
        g->jscale[2] = u / (d.dx * d.dy);
        g->rho_scale = u / (d.dx * d.dy);
    }
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

size_t lpic_species_bytes(int dim, int precision, long long capacity) {
    if ((dim != 2 && dim != 3) || capacity < 0) return 0;
    if (precision == LPIC_FP32_FIXED) return (size_t)(dim + 6) * 4 * (size_t)capacity;
    if (precision == LPIC_FP64) return (size_t)(dim + 4) * 8 * (size_t)capacity + 4 * (size_t)capacity;
    return 0;
}

const char* lpic_last_error(void) { return g_err.c_str(); }

lpic_status lpic_create_grid(const lpic_grid_desc* desc, lpic_grid_t* out) {
    if (!desc || !out) return fail(LPIC_EINVAL, "NULL descriptor or output");
    *out = nullptr;
    const lpic_grid_desc& d = *desc;
    if (d.dim != 2 && d.dim != 3) return fail(LPIC_EINVAL, "dim must be 2 or 3 (got %d)", d.dim);
    const int nz = (d.dim == 3) ? d.nz : 1;
    if (d.nx < 4 || d.ny < 4 || nz < 1 || (d.dim == 3 && d.nz < 4))
        return fail(LPIC_EINVAL, "grid too small (%d x %d x %d), need >= 4 cells per dimension", d.nx, d.ny, nz);
    if ((long long)(d.nx + 1) * d.ny * nz >= (1LL << 31))
        return fail(LPIC_EINVAL, "field arrays of 2^31 nodes or more (%d x %d x %d cells)", d.nx, d.ny, nz);
    if (!(d.dx > 0) || !(d.dy > 0) || (d.dim == 3 && !(d.dz > 0)) || !(d.dt > 0))
        return fail(LPIC_EINVAL, "cell sizes and dt must be positive");
    double s2 = 1.0 / (d.dx * d.dx) + 1.0 / (d.dy * d.dy) + (d.dim == 3 ? 1.0 / (d.dz * d.dz) : 0.0);
    if (!(d.dt * std::sqrt(s2) < 1.0))
        return fail(LPIC_EINVAL, "dt = %g violates the Courant limit %g", d.dt, 1.0 / std::sqrt(s2));
    if (d.shape_order != 1 && d.shape_order != 2) return fail(LPIC_EINVAL, "shape_order must be 1 or 2");
    if (d.precision != LPIC_FP64 && d.precision != LPIC_FP32_FIXED) return fail(LPIC_EINVAL, "bad precision");
    if (d.absorb_x < 0 || d.absorb_x > 2) return fail(LPIC_EINVAL, "absorb_x must be 0, 1 or 2");
    if (d.absorb_x == 2) {
        if (d.pml_cells < 1 || 2 * d.pml_cells + 8 > d.nx)
            return fail(LPIC_EINVAL, "pml_cells must be >= 1 with 2 pml_cells + 8 <= nx");
        if (!(d.pml_m >= 0) || !(d.pml_sigma_max >= 0) || !(d.pml_kappa_max >= 1) || !(d.pml_alpha_max >= 0))
            return fail(LPIC_EINVAL, "CPML needs pml_m, pml_sigma_max, pml_alpha_max >= 0 and pml_kappa_max >= 1");
    }
    if (d.absorb_x && d.nx < 8) return fail(LPIC_EINVAL, "absorbing x needs nx >= 8");
    if (d.laser && !d.absorb_x) return fail(LPIC_EINVAL, "a laser needs absorbing x edges");
    if (d.block_particles != 0 && (d.block_particles < 256 || d.block_particles > (1 << 20)))
        return fail(LPIC_EINVAL, "block_particles must be 0 or in [256, 2^20]");
    if (d.sort_interval < 0 || d.sort_interval > 64) return fail(LPIC_EINVAL, "sort_interval must be in [0, 64]");
    if (d.maxwell_fp64 != 0 && d.maxwell_fp64 != 1) return fail(LPIC_EINVAL, "maxwell_fp64 must be 0 or 1");
    if (d.maxwell_fp64 && d.precision != LPIC_FP32_FIXED)
        return fail(LPIC_EINVAL, "maxwell_fp64 applies to the FP32_FIXED path (the FP64 path has FP64 fields)");
    for (int c = 0; c < 3; ++c)
        if (!d.E[c] || !d.B[c] || !d.J[c]) return fail(LPIC_EINVAL, "field pointer %d is NULL", c);
    auto* g = new (std::nothrow) lpic_grid;
    if (!g) return fail(LPIC_ENOMEM, "host allocation failed");
    g->d = d;
    g->d.nz = nz;
    if (d.dim == 2) g->d.dz = 1.0;
    g->laser.on = d.laser ? 1 : 0;
    if (d.laser) {
        g->laser.a0 = d.laser->a0; g->laser.w0 = d.laser->w0; g->laser.tau = d.laser->tau;
        g->laser.omega = d.laser->omega; g->laser.yc = d.laser->yc; g->laser.zc = d.laser->zc;
        if (!(g->laser.w0 > 0) || !(g->laser.tau > 0)) { delete g; return fail(LPIC_EINVAL, "laser w0 and tau must be positive"); }
    }
    g->d.laser = nullptr;
    const int fx = d.absorb_x ? d.nx + 1 : d.nx;
    g->cpml = d.absorb_x == 2;
    g->geo = Geo{d.dim, d.nx, d.ny, nz, fx, d.absorb_x ? 1 : 0, d.dx, d.dy, g->d.dz, d.dt};
    g->nfield = (long long)fx * d.ny * nz;
    const int defT[2][3] = {{16, 16, 1}, {8, 8, 8}};
    const int n3[3] = {d.nx, d.ny, nz};
    g->ntiles = 1;
    for (int k = 0; k < 3; ++k) {
        int T = (k < d.dim) ? (d.tile[k] > 0 ? d.tile[k] : defT[d.dim - 2][k]) : 1;
        if (T > n3[k]) T = n3[k];
        if (k < d.dim && (T < 1 || T > 64)) { delete g; return fail(LPIC_EINVAL, "tile[%d] = %d out of [1, 64]", k, T); }
        g->T[k] = T;
        g->nt[k] = (n3[k] + T - 1) / T;
        g->ntiles *= g->nt[k];
    }
    if (d.dim == 2) { g->T[2] = 1; g->nt[2] = 1; }
    for (int k = 0; k < 3; ++k) g->fT[k] = make_fastdiv((unsigned)g->T[k]);
    g->dec = CellDecode{make_fastdiv((unsigned)d.nx), make_fastdiv((unsigned)d.ny)};
    if (d.block_particles > 0) g->P = d.block_particles;
    g->K = d.sort_interval > 1 ? d.sort_interval : 1;
    {
        // a particle moves less than c dt / h cells per step (Courant limit)
        const double hh[3] = {d.dx, d.dy, d.dim == 3 ? d.dz : 1.0};
        for (int k = 0; k < d.dim; ++k) g->m[k] = (int)std::ceil((g->K - 1) * d.dt / hh[k] - 1e-12);
    }
    // shrink the margin until the tile's boxes fit in shared memory; particles
    // that drift further take the global-memory path
    auto smem_for = [&](const int* m) { return (size_t)tile_smem(d.dim, g->T, m).words * 4; };
    while (smem_for(g->m) > 227 * 1024 && (g->m[0] > 0 || g->m[1] > 0 || g->m[2] > 0))
        for (int k = 0; k < 3; ++k) g->m[k] = g->m[k] > 0 ? g->m[k] - 1 : 0;
    {
        const int D = d.dim;
        (void)D;
        g->smem32 = smem_for(g->m);
        if (d.precision == LPIC_FP32_FIXED && g->smem32 > 227 * 1024) {
            delete g;
            return fail(LPIC_EINVAL, "tile needs %zu bytes of shared memory (> 227 KB)", g->smem32);
        }
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || g->nsm < 1) {
        delete g;
        return fail(LPIC_ECUDA, "cannot query the device's SM count");
    }
    const size_t fbytes = (d.precision == LPIC_FP64 || d.maxwell_fp64) ? 8 : 4;
    const int plane = d.ny * nz;
    if (dev_alloc(&g->d_status, 64) != cudaSuccess ||
        dev_alloc(&g->d_clock, 64) != cudaSuccess ||
        dev_alloc(&g->d_acc, 64) != cudaSuccess ||
        dev_alloc(&g->d_cnt, 64) != cudaSuccess ||
        (d.absorb_x == 1 && dev_alloc(&g->d_mur, fbytes * 8 * plane) != cudaSuccess) ||
        (g->cpml && dev_alloc(&g->d_psi, fbytes * 4 * plane * (2 * d.pml_cells + 2)) != cudaSuccess) ||
        (g->cpml && dev_alloc(&g->d_pcoef, fbytes * 6 * fx) != cudaSuccess) ||
        (g->laser.on && dev_alloc(&g->d_lprof, sizeof(double) * plane) != cudaSuccess)) {
        lpic_destroy_grid(g);
        return fail(LPIC_ENOMEM, "scratch allocation failed");
    }
    if (g->cpml) {
        // coefficients per x index for the half step tau = dt/2: nodes (x = i dx)
        // and half nodes (x = (i + 1/2) dx), depth measured into the layer
        const double tau = 0.5 * d.dt, L = d.pml_cells;
        std::vector<double> cf(6 * (size_t)fx);
        for (int h = 0; h < 2; ++h)
            for (int i = 0; i < fx; ++i) {
                const double xc = i + 0.5 * h;
                double dep = 0.0;
                if (xc < L) dep = (L - xc) / L;
                else if (xc > d.nx - L) dep = (xc - (d.nx - L)) / L;
                const double dm = std::pow(dep, d.pml_m);
                const double sigma = d.pml_sigma_max * dm;
                const double kappa = 1.0 + (d.pml_kappa_max - 1.0) * dm;
                const double alpha = dep > 0.0 ? d.pml_alpha_max * (1.0 - dep) : 0.0;
                const double b = std::exp(-(sigma / kappa + alpha) * tau);
                const double a = sigma > 0.0 ? sigma * (b - 1.0) / (sigma * kappa + kappa * kappa * alpha) : 0.0;
                cf[(0 + h) * fx + i] = 1.0 / kappa;
                cf[(2 + h) * fx + i] = a;
                cf[(4 + h) * fx + i] = b;
            }
        cudaError_t e = cudaSuccess;
        if (fbytes == 8) {
            e = cudaMemcpy(g->d_pcoef, cf.data(), 8 * cf.size(), cudaMemcpyHostToDevice);
        } else {
            std::vector<float> cff(cf.begin(), cf.end());
            e = cudaMemcpy(g->d_pcoef, cff.data(), 4 * cff.size(), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess || cudaMemset(g->d_psi, 0, fbytes * 4 * plane * (2 * d.pml_cells + 2)) != cudaSuccess) {
            lpic_destroy_grid(g);
            return fail(LPIC_ECUDA, "CPML set-up failed");
        }
    }
    if (g->laser.on) {
        k_laser_profile<<<grid_blocks(plane, g->nsm), 256>>>(g->geo, g->laser, g->d_lprof);
        if (cudaGetLastError() != cudaSuccess) { lpic_destroy_grid(g); return fail(LPIC_ECUDA, "laser profile"); }
    }
    if (cudaMemset(g->d_status, 0, 64) != cudaSuccess || cudaMemset(g->d_clock, 0, 64) != cudaSuccess) {
        lpic_destroy_grid(g);
        return fail(LPIC_ECUDA, "memset failed");
    }
    if (d.precision == LPIC_FP32_FIXED) {
        cudaError_t e = d.dim == 2 ? (d.shape_order == 1 ? set_smem_attrs<2, 1>(g->smem32) : set_smem_attrs<2, 2>(g->smem32))
                                   : (d.shape_order == 1 ? set_smem_attrs<3, 1>(g->smem32) : set_smem_attrs<3, 2>(g->smem32));
        if (e != cudaSuccess) { lpic_destroy_grid(g); return fail(LPIC_ECUDA, "shared memory attribute: %s", cudaGetErrorString(e)); }
    }
    recompute_shift(g);
    *out = g;
    return LPIC_OK;
}

lpic_status lpic_destroy_grid(lpic_grid_t g) {
    if (!g) return LPIC_OK;
    cudaDeviceSynchronize();
    for (auto& s : g->sp) {
        cudaFree(s.d_n); cudaFree(s.d_count); cudaFree(s.d_start); cudaFree(s.d_cursor);
        cudaFree(s.d_coff); cudaFree(s.d_items); cudaFree(s.d_nitems);
        cudaFree(s.d_esc); cudaFree(s.d_nesc);
    }
    for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second);
    for (auto e : g->ev) cudaEventDestroy(e);
    cudaFree(g->d_status); cudaFree(g->d_acc); cudaFree(g->d_cnt); cudaFree(g->d_mur); cudaFree(g->d_lprof);
    cudaFree(g->d_psi); cudaFree(g->d_pcoef);
    cudaFree(g->d_clock);
    cudaFree(g->d_qtab);
    cudaFree(g->d_btab);
    cudaFree(g->d_qstep);
    delete g;
    return LPIC_OK;
}

lpic_status lpic_grid_get_info(lpic_grid_t g, lpic_grid_info* out) {
    if (lpic_status r = check_grid(g)) return r;
    if (!out) return fail(LPIC_EINVAL, "NULL output");
    out->fixed_shift = g->F;
    for (int c = 0; c < 3; ++c) { out->j_scale[c] = g->jscale[c]; out->tile[c] = g->T[c]; }
    out->rho_scale = g->rho_scale;
    out->ntiles = g->ntiles;
    out->fx = g->geo.fx;
    out->launches = g->launches;
    return LPIC_OK;
}

lpic_status lpic_add_species(lpic_grid_t g, const lpic_species_desc* desc, cudaStream_t st, int* sid) {
    if (lpic_status r = check_grid(g)) return r;
    if (!desc || !sid) return fail(LPIC_EINVAL, "NULL descriptor or output");
    if (g->started) return fail(LPIC_EUNSUPPORTED, "species must be added before the first push");
    const lpic_species_desc& d = *desc;
    const bool massless = d.m == 0.0 && d.q == 0.0;
    if (!(d.m > 0 || massless) || !std::isfinite(d.m) || !std::isfinite(d.q))
        return fail(LPIC_EINVAL, "mass must be positive (or zero with zero charge), charge finite");
    if (massless && g->d.precision != LPIC_FP32_FIXED)
        return fail(LPIC_EUNSUPPORTED, "massless species need the FP32 path");
    if (d.capacity <= 0 || d.capacity % 64 != 0 || d.capacity >= (1LL << 31))
        return fail(LPIC_EINVAL, "capacity %lld must be a positive multiple of 64 below 2^31", d.capacity);
    if (d.count < 0 || d.count > d.capacity) return fail(LPIC_EINVAL, "count %lld outside [0, capacity]", d.count);
    if (!d.buffers[0] || !d.buffers[1] || d.buffers[0] == d.buffers[1])
        return fail(LPIC_EINVAL, "two distinct particle buffers are required");
    if (!aligned(d.buffers[0], 256) || !aligned(d.buffers[1], 256))
        return fail(LPIC_EINVAL, "particle buffers must be 256-byte aligned");
    Species s;
    s.q = d.q; s.m = d.m; s.cap = d.capacity; s.count0 = d.count; s.massless = massless;
    if (!(d.max_weight >= 0) || !std::isfinite(d.max_weight)) return fail(LPIC_EINVAL, "max_weight must be finite, >= 0");
    s.buf[0] = d.buffers[0]; s.buf[1] = d.buffers[1];
    const int nt = (int)g->ntiles;
    s.item_cap = nt + (d.capacity + g->P - 1) / g->P + 1;
    if (dev_alloc(&s.d_n, sizeof(int) * 4) != cudaSuccess ||
        dev_alloc(&s.d_count, sizeof(int) * (nt + 1)) != cudaSuccess ||
        dev_alloc(&s.d_start, sizeof(int) * (nt + 2)) != cudaSuccess ||
        dev_alloc(&s.d_cursor, sizeof(int) * (nt + 1)) != cudaSuccess ||
        dev_alloc(&s.d_coff, sizeof(int) * (nt + 1)) != cudaSuccess ||
        dev_alloc(&s.d_items, sizeof(int2) * s.item_cap) != cudaSuccess ||
        dev_alloc(&s.d_nitems, sizeof(int) * 4) != cudaSuccess ||
        dev_alloc(&s.d_esc, sizeof(int) * d.capacity) != cudaSuccess ||
        dev_alloc(&s.d_nesc, sizeof(int) * 4) != cudaSuccess) {
        cudaFree(s.d_n); cudaFree(s.d_count); cudaFree(s.d_start); cudaFree(s.d_cursor);
        cudaFree(s.d_coff); cudaFree(s.d_items); cudaFree(s.d_nitems);
        cudaFree(s.d_esc); cudaFree(s.d_nesc);
        return fail(LPIC_ENOMEM, "species scratch allocation failed");
    }
    // d_n[0]: particles; d_n[1]: id of the next particle created on the device
    const int n2[2] = {(int)d.count, (int)d.count};
    LPIC_CUDA(cudaMemcpyAsync(s.d_n, n2, sizeof(n2), cudaMemcpyHostToDevice, st));
    // largest |w|, for the fixed-point bound
    if (g->d.precision == LPIC_FP32_FIXED) {
        const P32 p = view32(g, s, 0);
        unsigned bits = 0;
        LPIC_CUDA(cudaMemsetAsync(g->d_cnt, 0, 8, st));
        k_absmax_f32<<<grid_blocks(s.cap, g->nsm), 256, 0, st>>>(p.w, s.d_n, reinterpret_cast<unsigned*>(g->d_cnt));
        LPIC_LAUNCHED("k_absmax_f32");
        LPIC_CUDA(cudaMemcpyAsync(&bits, g->d_cnt, 4, cudaMemcpyDeviceToHost, st));
        LPIC_CUDA(cudaStreamSynchronize(st));
        float wm;
        std::memcpy(&wm, &bits, 4);
        s.wmax = wm;
    } else {
        const P64 p = view64(g, s, 0);
        unsigned long long bits = 0;
        LPIC_CUDA(cudaMemsetAsync(g->d_cnt, 0, 8, st));
        k_absmax_f64<<<grid_blocks(s.cap, g->nsm), 256, 0, st>>>(p.w, s.d_n, g->d_cnt);
        LPIC_LAUNCHED("k_absmax_f64");
        LPIC_CUDA(cudaMemcpyAsync(&bits, g->d_cnt, 8, cudaMemcpyDeviceToHost, st));
        LPIC_CUDA(cudaStreamSynchronize(st));
        double wm;
        std::memcpy(&wm, &bits, 8);
        s.wmax = wm;
    }
    if (!std::isfinite(s.wmax)) return fail(LPIC_EINVAL, "non-finite particle weight");
    s.wmax = std::max(s.wmax, d.max_weight);   // particles created later (pairs) stay under the bound
    // x^0 -> x^{1/2}
    if (!d.staggered) {
        const int nb = grid_blocks(s.cap, g->nsm);
        if (g->d.precision == LPIC_FP32_FIXED) {
            const P32 p = view32(g, s, 0);
            const float a = (float)(g->d.dt / g->d.dx), b = (float)(g->d.dt / g->d.dy),
                        c = (float)(g->d.dt / g->d.dz);
            if (massless) {
                if (g->d.dim == 3) k_photon32<3><<<nb, 256, 0, st>>>(g->geo, p, g->dec, 0.5f, a, b, c, 0);
                else               k_photon32<2><<<nb, 256, 0, st>>>(g->geo, p, g->dec, 0.5f, a, b, c, 0);
            } else {
                if (g->d.dim == 3) k_advance32<3><<<nb, 256, 0, st>>>(g->geo, p, g->dec, 0.5f, a, b, c);
                else               k_advance32<2><<<nb, 256, 0, st>>>(g->geo, p, g->dec, 0.5f, a, b, c);
            }
        } else {
            const P64 p = view64(g, s, 0);
            if (g->d.dim == 3) k_advance64<3><<<nb, 256, 0, st>>>(g->geo, p, 0.5);
            else               k_advance64<2><<<nb, 256, 0, st>>>(g->geo, p, 0.5);
        }
        LPIC_LAUNCHED("k_advance");
        LPIC_CUDA(cudaStreamSynchronize(st));
    }
    g->sp.push_back(s);
    recompute_shift(g);
    *sid = (int)g->sp.size() - 1;
    return LPIC_OK;
}

lpic_status lpic_species_query(lpic_grid_t g, int sid, cudaStream_t st, int* cur, long long* count) {
    if (lpic_status r = check_species(g, sid)) return r;
    int n = 0;
    LPIC_CUDA(cudaMemcpyAsync(&n, g->sp[sid].d_n, sizeof(int), cudaMemcpyDeviceToHost, st));
    LPIC_CUDA(cudaStreamSynchronize(st));
    if (cur) *cur = g->sp[sid].cur;
    if (count) *count = n;
    return LPIC_OK;
}

lpic_status lpic_sort_particles(lpic_grid_t g, int sid, cudaStream_t st) {
    if (sid == -1) {
        if (lpic_status r = check_grid(g)) return r;
        for (auto& s : g->sp)
            if (lpic_status r = sort_one(g, s, st)) return r;
        return LPIC_OK;
    }
    if (lpic_status r = check_species(g, sid)) return r;
    return sort_one(g, g->sp[sid], st);
}

lpic_status lpic_zero_current(lpic_grid_t g, cudaStream_t st) {
    if (lpic_status r = check_grid(g)) return r;
    for (int c = 0; c < 3; ++c) LPIC_CUDA(cudaMemsetAsync(g->d.J[c], 0, 8 * (size_t)g->nfield, st));
    return LPIC_OK;
}

static lpic_status gpd_impl(lpic_grid_t g, int sid, cudaStream_t st, bool count_next) {
    Species& s = g->sp[sid];
    g->started = true;
    const int D = g->d.dim, O = g->d.shape_order;
    lpic_status r;
    if (s.massless) {
        // ballistic push over [0, n): needs no tile order and no fields (not
        // a launch of the fused kernel, so not timed with it)
        const P32 p = view32(g, s, s.cur);
        const int nb = grid_blocks(s.cap, g->nsm, 16);
        const float a = (float)(g->d.dt / g->d.dx), b = (float)(g->d.dt / g->d.dy),
                    c = (float)(g->d.dt / (D == 3 ? g->d.dz : 1.0));
        const int edge = g->d.absorb_x ? 2 : 0;
        if (D == 3) k_photon32<3><<<nb, 256, 0, st>>>(g->geo, p, g->dec, 1.0f, a, b, c, edge);
        else        k_photon32<2><<<nb, 256, 0, st>>>(g->geo, p, g->dec, 1.0f, a, b, c, edge);
        LPIC_LAUNCHED("k_photon32");
        s.since_sort += 1;
        s.counts_fresh = false;
        return LPIC_OK;
    }
    if (g->d.precision == LPIC_FP32_FIXED) {
        if (!s.sorted || s.since_sort >= g->K)
            return fail(LPIC_EINVAL, "species %d must be sorted by tile at least every %d pushes", sid, g->K);
        const bool timed = g->timing && g->ev_used + 2 <= g->ev.size();
        if (timed) LPIC_CUDA(cudaEventRecord(g->ev[g->ev_used], st));
        if (D == 2) r = (O == 1) ? launch_gpd32<2, 1>(g, s, st, count_next) : launch_gpd32<2, 2>(g, s, st, count_next);
        else        r = (O == 1) ? launch_gpd32<3, 1>(g, s, st, count_next) : launch_gpd32<3, 2>(g, s, st, count_next);
        if (timed) { LPIC_CUDA(cudaEventRecord(g->ev[g->ev_used + 1], st)); g->ev_used += 2; }
        s.since_sort += 1;
        s.counts_fresh = count_next && r == LPIC_OK;
    } else {
        const bool timed = g->timing && g->ev_used + 2 <= g->ev.size();
        if (timed) LPIC_CUDA(cudaEventRecord(g->ev[g->ev_used], st));
        if (D == 2) r = (O == 1) ? launch_gpd64<2, 1>(g, s, st) : launch_gpd64<2, 2>(g, s, st);
        else        r = (O == 1) ? launch_gpd64<3, 1>(g, s, st) : launch_gpd64<3, 2>(g, s, st);
        if (timed) { LPIC_CUDA(cudaEventRecord(g->ev[g->ev_used + 1], st)); g->ev_used += 2; }
    }
    return r;
}

lpic_status lpic_gather_push_deposit(lpic_grid_t g, int sid, cudaStream_t st) {
    if (lpic_status r = check_species(g, sid)) return r;
    return gpd_impl(g, sid, st, false);
}

lpic_status lpic_gather_fields(lpic_grid_t g, int sid, float* fields, cudaStream_t st) {
    if (lpic_status r = check_species(g, sid)) return r;
    if (g->d.precision != LPIC_FP32_FIXED) return fail(LPIC_EUNSUPPORTED, "the unfused stages need the FP32 path");
    if (g->sp[sid].massless) return fail(LPIC_EUNSUPPORTED, "a massless species has no field stages");
    if (g->sp[sid].q_ph >= 0) return fail(LPIC_EUNSUPPORTED, "species %d emits inside its fused push (no stages)", sid);
    if (!fields) return fail(LPIC_EINVAL, "fields is NULL");
    Species& s = g->sp[sid];
    g->started = true;
    if (!s.sorted || s.since_sort > 0)
        if (lpic_status r = sort_one(g, s, st, false)) return r;
    const int D = g->d.dim, O = g->d.shape_order;
    lpic_status r;
    const bool timed = g->timing && g->ev_used + 2 <= g->ev.size();
    if (timed) LPIC_CUDA(cudaEventRecord(g->ev[g->ev_used], st));
    if (D == 2) r = (O == 1) ? launch_stage<2, 1>(g, s, st, true, fields) : launch_stage<2, 2>(g, s, st, true, fields);
    else        r = (O == 1) ? launch_stage<3, 1>(g, s, st, true, fields) : launch_stage<3, 2>(g, s, st, true, fields);
    if (timed) { LPIC_CUDA(cudaEventRecord(g->ev[g->ev_used + 1], st)); g->ev_used += 2; }
    if (r == LPIC_OK) s.gather_gen = s.sort_gen;
    return r;
}

lpic_status lpic_push_deposit_fields(lpic_grid_t g, int sid, const float* fields, cudaStream_t st) {
    if (lpic_status r = check_species(g, sid)) return r;
    if (g->d.precision != LPIC_FP32_FIXED) return fail(LPIC_EUNSUPPORTED, "the unfused stages need the FP32 path");
    if (g->sp[sid].massless) return fail(LPIC_EUNSUPPORTED, "a massless species has no field stages");
    if (g->sp[sid].q_ph >= 0) return fail(LPIC_EUNSUPPORTED, "species %d emits inside its fused push (no stages)", sid);
    if (!fields) return fail(LPIC_EINVAL, "fields is NULL");
    Species& s = g->sp[sid];
    if (s.gather_gen != s.sort_gen || s.since_sort != 0)
        return fail(LPIC_EINVAL, "species %d: call lpic_gather_fields first (the particles were re-sorted or "
                    "pushed since)", sid);
    const int D = g->d.dim, O = g->d.shape_order;
    float* f = const_cast<float*>(fields);
    lpic_status r;
    const bool timed = g->timing && g->ev_used + 2 <= g->ev.size();
    if (timed) LPIC_CUDA(cudaEventRecord(g->ev[g->ev_used], st));
    if (D == 2) r = (O == 1) ? launch_stage<2, 1>(g, s, st, false, f) : launch_stage<2, 2>(g, s, st, false, f);
    else        r = (O == 1) ? launch_stage<3, 1>(g, s, st, false, f) : launch_stage<3, 2>(g, s, st, false, f);
    if (timed) { LPIC_CUDA(cudaEventRecord(g->ev[g->ev_used + 1], st)); g->ev_used += 2; }
    s.since_sort += 1;
    s.counts_fresh = false;
    s.gather_gen = -1;
    return r;
}

static lpic_status maxwell_any(lpic_grid_t g, int half, double t, cudaStream_t st, const double* clock) {
    if (g->d.precision == LPIC_FP32_FIXED && g->d.maxwell_fp64)
        return g->d.dim == 3 ? maxwell_impl<3, double, long long>(g, half, t, st, clock)
                             : maxwell_impl<2, double, long long>(g, half, t, st, clock);
    if (g->d.precision == LPIC_FP32_FIXED)
        return g->d.dim == 3 ? maxwell_impl<3, float, long long>(g, half, t, st, clock)
                             : maxwell_impl<2, float, long long>(g, half, t, st, clock);
    return g->d.dim == 3 ? maxwell_impl<3, double, double>(g, half, t, st, clock)
                         : maxwell_impl<2, double, double>(g, half, t, st, clock);
}

lpic_status lpic_maxwell_half_step(lpic_grid_t g, int half, double t, cudaStream_t st) {
    if (lpic_status r = check_grid(g)) return r;
    if (half != 0 && half != 1) return fail(LPIC_EINVAL, "half must be 0 or 1");
    return maxwell_any(g, half, t, st, nullptr);
}

// One step; with a device clock the laser time is *clock (+ dt/2 in the
// second half) and the clock advances by dt at the end.
// The counter word of the fused emission advances once per full step.
static lpic_status advance_qed_step(lpic_grid_t g, cudaStream_t st) {
    for (const Species& s : g->sp)
        if (s.q_ph >= 0) {
            k_add_uint<<<1, 32, 0, st>>>(g->d_qstep, 1u);
            LPIC_LAUNCHED("k_add_uint");
            break;
        }
    return LPIC_OK;
}

static lpic_status step_impl(lpic_grid_t g, double t, cudaStream_t st, double* clock) {
    if (lpic_status r = maxwell_any(g, 0, clock ? 0.0 : t, st, clock)) return r;
    if (lpic_status r = lpic_zero_current(g, st)) return r;
    for (int s = 0; s < (int)g->sp.size(); ++s) {
        Species& sp = g->sp[s];
        bool count_next = false;
        if (g->d.precision == LPIC_FP32_FIXED) {
            // sort every K steps; the push before a sort counts its tile keys
            if (!sp.sorted || sp.since_sort >= g->K)
                if (lpic_status r = sort_one(g, sp, st, sp.sorted && sp.counts_fresh)) return r;
            count_next = sp.since_sort + 1 >= g->K;
        }
        if (lpic_status r = gpd_impl(g, s, st, count_next)) return r;
    }
    if (lpic_status r = maxwell_any(g, 1, (clock ? 0.0 : t) + 0.5 * g->d.dt, st, clock)) return r;
    if (clock) {
        k_clock_add<<<1, 32, 0, st>>>(clock, g->d.dt);
        LPIC_LAUNCHED("k_clock_add");
    }
    return advance_qed_step(g, st);
}

lpic_status lpic_step(lpic_grid_t g, double t, cudaStream_t st) {
    if (lpic_status r = check_grid(g)) return r;
    return step_impl(g, t, st, nullptr);
}

// A step that also advances `aux` with the current of species sid alone: the
// species is deposited first, its current copied into aux's J, then the
// other species deposit on top; aux's Maxwell halves use the grid's
// fixed-point scale.
lpic_status lpic_step_resolved(lpic_grid_t g, double t, int sid, lpic_grid_t aux, cudaStream_t st) {
    if (lpic_status r = check_species(g, sid)) return r;
    if (!aux || aux == g) return fail(LPIC_EINVAL, "aux must be another grid");
    const lpic_grid_desc &a = aux->d, &d = g->d;
    if (a.dim != d.dim || a.nx != d.nx || a.ny != d.ny || a.nz != d.nz || a.dx != d.dx || a.dy != d.dy ||
        a.dz != d.dz || a.dt != d.dt || a.precision != d.precision || a.absorb_x != d.absorb_x ||
        (a.absorb_x == 2 && a.pml_cells != d.pml_cells) || a.maxwell_fp64 != d.maxwell_fp64)
        return fail(LPIC_EINVAL, "aux must have the grid's geometry, time step, precision, field precision and x boundary");
    if (!aux->sp.empty()) return fail(LPIC_EINVAL, "aux must hold no species");
    auto aux_half = [&](int half, double th) -> lpic_status {
        for (int c = 0; c < 3; ++c) aux->jscale[c] = g->jscale[c];
        return maxwell_any(aux, half, th, st, nullptr);
    };
    if (lpic_status r = maxwell_any(g, 0, t, st, nullptr)) return r;
    if (lpic_status r = aux_half(0, t)) return r;
    if (lpic_status r = lpic_zero_current(g, st)) return r;
    const int n = (int)g->sp.size();
    const size_t jbytes = (size_t)g->nfield * (d.precision == LPIC_FP64 ? sizeof(double) : sizeof(long long));
    for (int k = 0; k < n; ++k) {
        const int s = k == 0 ? sid : (k <= sid ? k - 1 : k);
        Species& sp = g->sp[s];
        bool count_next = false;
        if (d.precision == LPIC_FP32_FIXED) {
            if (!sp.sorted || sp.since_sort >= g->K)
                if (lpic_status r = sort_one(g, sp, st, sp.sorted && sp.counts_fresh)) return r;
            count_next = sp.since_sort + 1 >= g->K;
        }
        if (lpic_status r = gpd_impl(g, s, st, count_next)) return r;
        if (k == 0)
            for (int c = 0; c < 3; ++c)
                LPIC_CUDA(cudaMemcpyAsync(aux->d.J[c], g->d.J[c], jbytes, cudaMemcpyDeviceToDevice, st));
    }
    if (lpic_status r = maxwell_any(g, 1, t + 0.5 * d.dt, st, nullptr)) return r;
    if (lpic_status r = aux_half(1, t + 0.5 * d.dt)) return r;
    return advance_qed_step(g, st);
}

lpic_status lpic_set_clock(lpic_grid_t g, double t, cudaStream_t st) {
    if (lpic_status r = check_grid(g)) return r;
    k_clock_set<<<1, 32, 0, st>>>(g->d_clock, t);
    LPIC_LAUNCHED("k_clock_set");
    return LPIC_OK;
}

lpic_status lpic_graph_steps(lpic_grid_t g, int nsteps, cudaStream_t st) {
    if (lpic_status r = check_grid(g)) return r;
    if (nsteps < 0) return fail(LPIC_EINVAL, "nsteps must be >= 0");
    if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread)
        return fail(LPIC_EINVAL, "graph capture needs a created (non-default) stream");
    for (int k = 0; k < nsteps; ++k) {
        // FNV-1a over each species' buffer parity and sort state: species can
        // be out of step with one another (a pair-creation pass marks its pair
        // species for a sort), and the captured step must match all of them
        unsigned long long key = 1469598103934665603ULL;
        auto mix = [&key](unsigned long long v) { key ^= v; key *= 1099511628211ULL; };
        for (const Species& s : g->sp) {
            mix((unsigned long long)s.cur);
            if (g->d.precision == LPIC_FP32_FIXED) {
                const int phase = (!s.sorted || s.since_sort >= g->K) ? 0 : s.since_sort;
                mix((unsigned long long)phase << 2 | (unsigned long long)(s.sorted && s.counts_fresh) << 1 |
                    (unsigned long long)s.sorted);
            }
        }
        auto it = g->graphs.find(key);
        if (it == g->graphs.end()) {
            // capture one step starting from this buffer parity
            std::vector<Species> saved = g->sp;
            const long long l0 = g->launches;
            LPIC_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            lpic_status r = step_impl(g, 0.0, st, g->d_clock);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(st, &graph);
            for (size_t s = 0; s < g->sp.size(); ++s) {
                g->sp[s].cur = saved[s].cur; g->sp[s].sorted = saved[s].sorted;
                g->sp[s].since_sort = saved[s].since_sort; g->sp[s].counts_fresh = saved[s].counts_fresh;
            }
            const long long per_step = g->launches - l0;
            g->launches = l0;
            if (r != LPIC_OK) { if (graph) cudaGraphDestroy(graph); return r; }
            if (e != cudaSuccess) return fail(LPIC_ECUDA, "stream capture: %s", cudaGetErrorString(e));
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return fail(LPIC_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
            g->graphs[key] = exec;
            g->graph_launches[key] = per_step;
            it = g->graphs.find(key);
        }
        LPIC_CUDA(cudaGraphLaunch(it->second, st));
        g->launches += g->graph_launches[key];
        // replay the host-side bookkeeping of the captured step
        if (g->d.precision == LPIC_FP32_FIXED)
            for (auto& s : g->sp) {
                if (!s.sorted || s.since_sort >= g->K) { s.cur = 1 - s.cur; s.sorted = true; s.since_sort = 0; s.sort_gen += 1; }
                s.since_sort += 1;
                s.counts_fresh = s.since_sort >= g->K && !s.massless;
            }
        g->started = true;
    }
    return LPIC_OK;
}

lpic_status lpic_deposit_charge(lpic_grid_t g, int sid, void* rho, cudaStream_t st) {
    if (lpic_status r = check_species(g, sid)) return r;
    if (!rho) return fail(LPIC_EINVAL, "rho is NULL");
    Species& s = g->sp[sid];
    const int nb = grid_blocks(s.cap, g->nsm, 16);
    const int D = g->d.dim, O = g->d.shape_order;
    if (g->d.precision == LPIC_FP32_FIXED) {
        const P32 p = view32(g, s, s.cur);
        const float sq = (float)std::ldexp(s.q, g->F);
        auto* r = static_cast<unsigned long long*>(rho);
        if (D == 2) { if (O == 1) k_charge32<2, 1><<<nb, 256, 0, st>>>(g->geo, p, g->dec, sq, r); else k_charge32<2, 2><<<nb, 256, 0, st>>>(g->geo, p, g->dec, sq, r); }
        else        { if (O == 1) k_charge32<3, 1><<<nb, 256, 0, st>>>(g->geo, p, g->dec, sq, r); else k_charge32<3, 2><<<nb, 256, 0, st>>>(g->geo, p, g->dec, sq, r); }
    } else {
        const P64 p = view64(g, s, s.cur);
        auto* r = static_cast<double*>(rho);
        if (D == 2) { if (O == 1) k_charge64<2, 1><<<nb, 256, 0, st>>>(g->geo, p, s.q, r); else k_charge64<2, 2><<<nb, 256, 0, st>>>(g->geo, p, s.q, r); }
        else        { if (O == 1) k_charge64<3, 1><<<nb, 256, 0, st>>>(g->geo, p, s.q, r); else k_charge64<3, 2><<<nb, 256, 0, st>>>(g->geo, p, s.q, r); }
    }
    LPIC_LAUNCHED("k_charge");
    return LPIC_OK;
}

lpic_status lpic_div_e(lpic_grid_t g, double* out, cudaStream_t st) {
    if (lpic_status r = check_grid(g)) return r;
    if (!out) return fail(LPIC_EINVAL, "out is NULL");
    const FastDiv dfx = make_fastdiv((unsigned)g->geo.fx), dny = make_fastdiv((unsigned)g->d.ny);
    const int nb = grid_blocks(g->nfield, g->nsm, 16);
    if (g->d.precision == LPIC_FP32_FIXED && !g->d.maxwell_fp64)
        k_div_e<float><<<nb, 256, 0, st>>>(g->geo, ptr3<const float>(g->d.E), out, dfx, dny);
    else
        k_div_e<double><<<nb, 256, 0, st>>>(g->geo, ptr3<const double>(g->d.E), out, dfx, dny);
    LPIC_LAUNCHED("k_div_e");
    return LPIC_OK;
}

lpic_status lpic_positions_at_step(lpic_grid_t g, int sid, double* out, cudaStream_t st) {
    if (lpic_status r = check_species(g, sid)) return r;
    if (!out) return fail(LPIC_EINVAL, "out is NULL");
    Species& s = g->sp[sid];
    const int nb = grid_blocks(s.cap, g->nsm, 16);
    if (g->d.precision == LPIC_FP32_FIXED) {
        const P32 p = view32(g, s, s.cur);
        if (g->d.dim == 3) k_positions32<3><<<nb, 256, 0, st>>>(g->geo, p, g->dec, out, s.cap, s.massless);
        else               k_positions32<2><<<nb, 256, 0, st>>>(g->geo, p, g->dec, out, s.cap, s.massless);
    } else {
        const P64 p = view64(g, s, s.cur);
        if (g->d.dim == 3) k_positions64<3><<<nb, 256, 0, st>>>(g->geo, p, out, s.cap);
        else               k_positions64<2><<<nb, 256, 0, st>>>(g->geo, p, out, s.cap);
    }
    LPIC_LAUNCHED("k_positions");
    return LPIC_OK;
}

lpic_status lpic_diagnostics(lpic_grid_t g, lpic_diag* out, cudaStream_t st) {
    if (lpic_status r = check_grid(g)) return r;
    if (!out) return fail(LPIC_EINVAL, "out is NULL");
    LPIC_CUDA(cudaMemsetAsync(g->d_acc, 0, 64, st));
    LPIC_CUDA(cudaMemsetAsync(g->d_cnt, 0, 8, st));
    for (auto& s : g->sp) {
        const int nb = grid_blocks(s.cap, g->nsm, 8);
        if (g->d.precision == LPIC_FP32_FIXED)
            k_diag_p32<<<nb, 256, 0, st>>>(view32(g, s, s.cur), s.q, s.m, g->d_acc, g->d_cnt);
        else
            k_diag_p64<<<nb, 256, 0, st>>>(view64(g, s, s.cur), s.q, s.m, g->d_acc, g->d_cnt);
        LPIC_LAUNCHED("k_diag_p");
    }
    const double dV = g->d.dx * g->d.dy * (g->d.dim == 3 ? g->d.dz : 1.0);
    const int nb = grid_blocks(g->nfield, g->nsm, 8);
    if (g->d.precision == LPIC_FP32_FIXED && !g->d.maxwell_fp64)
        k_diag_field<float><<<nb, 256, 0, st>>>(ptr3<const float>(g->d.E), ptr3<const float>(g->d.B), g->nfield, dV, g->d_acc);
    else
        k_diag_field<double><<<nb, 256, 0, st>>>(ptr3<const double>(g->d.E), ptr3<const double>(g->d.B), g->nfield, dV, g->d_acc);
    LPIC_LAUNCHED("k_diag_field");
    double acc[3];
    unsigned long long cnt = 0;
    LPIC_CUDA(cudaMemcpyAsync(acc, g->d_acc, sizeof acc, cudaMemcpyDeviceToHost, st));
    LPIC_CUDA(cudaMemcpyAsync(&cnt, g->d_cnt, 8, cudaMemcpyDeviceToHost, st));
    LPIC_CUDA(cudaStreamSynchronize(st));
    out->kinetic = acc[0];
    out->charge = acc[1];
    out->field = acc[2];
    out->particles = (long long)cnt;
    return LPIC_OK;
}

lpic_status lpic_kernel_timing(lpic_grid_t g, int max_launches) {
    if (lpic_status r = check_grid(g)) return r;
    if (max_launches < 0) return fail(LPIC_EINVAL, "max_launches must be >= 0");
    for (auto e : g->ev) cudaEventDestroy(e);
    g->ev.clear();
    g->ev_used = 0;
    g->timing = max_launches > 0;
    for (int i = 0; i < 2 * max_launches; ++i) {
        cudaEvent_t e;
        LPIC_CUDA(cudaEventCreate(&e));
        g->ev.push_back(e);
    }
    return LPIC_OK;
}

lpic_status lpic_kernel_time(lpic_grid_t g, double* ms, long long* launches) {
    if (lpic_status r = check_grid(g)) return r;
    double total = 0.0;
    for (size_t i = 0; i + 1 < g->ev_used; i += 2) {
        LPIC_CUDA(cudaEventSynchronize(g->ev[i + 1]));
        float t = 0.0f;
        LPIC_CUDA(cudaEventElapsedTime(&t, g->ev[i], g->ev[i + 1]));
        total += t;
    }
    if (ms) *ms = total;
    if (launches) *launches = (long long)(g->ev_used / 2);
    return LPIC_OK;
}

lpic_status lpic_check_status(lpic_grid_t g, cudaStream_t st, unsigned* bits) {
    if (lpic_status r = check_grid(g)) return r;
    unsigned b = 0;
    LPIC_CUDA(cudaMemcpyAsync(&b, g->d_status, 4, cudaMemcpyDeviceToHost, st));
    LPIC_CUDA(cudaStreamSynchronize(st));
    LPIC_CUDA(cudaMemsetAsync(g->d_status, 0, 4, st));
    LPIC_CUDA(cudaStreamSynchronize(st));
    if (bits) *bits = b;
    if (b) return fail(LPIC_EDEVICE, "device status bits 0x%x", b);
    return LPIC_OK;
}

}  // extern "C"

// ======================================================================= ensembles
struct lpic_ensemble {
    std::vector<lpic_grid_t> grids;
    int dim = 2, order = 1, nsm = 0, blocks = 1;
    int ninst = 0, nslots = 0;
    size_t smem = 0;
    EnsField* d_fields = nullptr;
    EnsSort* d_sort = nullptr;
    GpdArgs* d_args[2] = {nullptr, nullptr};
    int* d_order = nullptr;
    int* d_prefix = nullptr;
    int* d_head = nullptr;
    unsigned* d_status = nullptr;
    std::vector<std::pair<int, int>> slots;     // (grid, species)
    int parity = 0;
    bool counted = false;                        // histograms hold the current cells
    long long launches = 0;
    long long max_ntiles = 1, max_field = 1, max_cap = 1;
    std::map<int, cudaGraphExec_t> graphs;
    std::map<int, long long> graph_launches;
};

namespace {

template <int DIM, int ORDER>
cudaError_t ens_attrs(size_t bytes, const void** fn) {
    *fn = Gpd32<DIM, ORDER>::queue_fn();
    return Gpd32<DIM, ORDER>::set_smem(bytes);
}

template <int DIM, int ORDER>
lpic_status ens_push(lpic_ensemble* e, cudaStream_t st) {
    lpic_ensemble* g = e;   // LPIC_LAUNCHED counts on g
    Gpd32<DIM, ORDER>::queue(e->d_args[e->parity], e->d_order, e->d_prefix, e->nslots, e->d_head,
                             (unsigned)e->blocks, e->smem, st);
    LPIC_LAUNCHED("k_gpd32_queue");
    return LPIC_OK;
}

lpic_status ens_step_impl(lpic_ensemble* e, cudaStream_t st) {
    lpic_ensemble* g = e;
    const dim3 fgrid((unsigned)std::min<long long>((e->max_field + 255) / 256, 1024), (unsigned)e->ninst);
    const dim3 sgrid((unsigned)std::min<long long>((e->max_cap + 255) / 256, 512), (unsigned)e->nslots);
    const dim3 tgrid((unsigned)std::min<long long>((e->max_ntiles + 255) / 256, 64), (unsigned)e->nslots);
    if (e->dim == 3) k_update_E_many<3><<<fgrid, 256, 0, st>>>(e->d_fields);
    else             k_update_E_many<2><<<fgrid, 256, 0, st>>>(e->d_fields);
    LPIC_LAUNCHED("k_update_E_many");
    if (e->dim == 3) k_update_B_many<3><<<fgrid, 256, 0, st>>>(e->d_fields);
    else             k_update_B_many<2><<<fgrid, 256, 0, st>>>(e->d_fields);
    LPIC_LAUNCHED("k_update_B_many");
    k_zero_J_many<<<fgrid, 256, 0, st>>>(e->d_fields);
    LPIC_LAUNCHED("k_zero_J_many");
    // sort every slot from buffer `parity` into the other one
    k_sort_zero_many<<<tgrid, 256, 0, st>>>(e->d_sort, e->counted ? 0 : 1);
    LPIC_LAUNCHED("k_sort_zero_many");
    if (!e->counted) {
        k_sort_count_many<<<sgrid, 256, 0, st>>>(e->d_sort, e->parity);
        LPIC_LAUNCHED("k_sort_count_many");
    }
    k_sort_scan_many<<<e->nslots, 1024, 0, st>>>(e->d_sort);
    LPIC_LAUNCHED("k_sort_scan_many");
    k_sort_items_many<<<tgrid, 256, 0, st>>>(e->d_sort);
    LPIC_LAUNCHED("k_sort_items_many");
    k_sort_scatter_many<<<sgrid, 256, 0, st>>>(e->d_sort, e->parity);
    LPIC_LAUNCHED("k_sort_scatter_many");
    k_sort_finalize_many<<<1, 256, 0, st>>>(e->d_sort, e->nslots);
    LPIC_LAUNCHED("k_sort_finalize_many");
    k_count_zero_many<<<tgrid, 256, 0, st>>>(e->d_sort);
    LPIC_LAUNCHED("k_count_zero_many");
    k_queue_prefix<<<1, 1024, 0, st>>>(e->d_sort, e->d_order, e->nslots, e->d_prefix, e->d_head);
    LPIC_LAUNCHED("k_queue_prefix");
    e->parity ^= 1;
    lpic_status r;
    if (e->dim == 2) r = e->order == 1 ? ens_push<2, 1>(e, st) : ens_push<2, 2>(e, st);
    else             r = e->order == 1 ? ens_push<3, 1>(e, st) : ens_push<3, 2>(e, st);
    if (r != LPIC_OK) return r;
    k_check_escapes<<<1, 256, 0, st>>>(e->d_sort, e->nslots, e->d_status);
    LPIC_LAUNCHED("k_check_escapes");
    if (e->dim == 3) k_update_B_many<3><<<fgrid, 256, 0, st>>>(e->d_fields);
    else             k_update_B_many<2><<<fgrid, 256, 0, st>>>(e->d_fields);
    LPIC_LAUNCHED("k_update_B_many");
    if (e->dim == 3) k_update_E_many<3><<<fgrid, 256, 0, st>>>(e->d_fields);
    else             k_update_E_many<2><<<fgrid, 256, 0, st>>>(e->d_fields);
    LPIC_LAUNCHED("k_update_E_many");
    e->counted = true;
    return LPIC_OK;
}

// the grids' own bookkeeping after an ensemble step (every species flipped)
void ens_sync_grids(lpic_ensemble* e) {
    for (auto& sl : e->slots) {
        Species& s = e->grids[sl.first]->sp[sl.second];
        s.cur = e->parity;
        s.sorted = true;
        s.sort_gen += 1;
        s.since_sort = 1;
        s.counts_fresh = true;
        e->grids[sl.first]->started = true;
    }
}

}  // namespace

extern "C" {

lpic_status lpic_create_ensemble(lpic_grid_t* grids, int n, lpic_ensemble_t* out) {
    if (!grids || !out || n < 1) return fail(LPIC_EINVAL, "need at least one grid");
    *out = nullptr;
    const lpic_grid_t g0 = grids[0];
    if (!g0) return fail(LPIC_EINVAL, "grid 0 is NULL");
    for (int i = 0; i < n; ++i) {
        const lpic_grid_t g = grids[i];
        if (!g) return fail(LPIC_EINVAL, "grid %d is NULL", i);
        if (g->d.precision != LPIC_FP32_FIXED) return fail(LPIC_EUNSUPPORTED, "ensembles need the FP32 path");
        if (g->d.maxwell_fp64) return fail(LPIC_EUNSUPPORTED, "grid %d: ensembles keep float fields (no maxwell_fp64)", i);
        if (g->d.dim != g0->d.dim || g->d.shape_order != g0->d.shape_order)
            return fail(LPIC_EINVAL, "grid %d: dimension and shape order must match grid 0", i);
        if (g->K != 1) return fail(LPIC_EUNSUPPORTED, "grid %d: ensembles sort every step (sort_interval <= 1)", i);
        if (g->geo.absorb || g->laser.on) return fail(LPIC_EUNSUPPORTED, "grid %d: ensembles need periodic grids", i);
        if (g->sp.empty()) return fail(LPIC_EINVAL, "grid %d has no species", i);
        for (auto& s : g->sp) {
            if (s.cur != g0->sp[0].cur) return fail(LPIC_EINVAL, "grid %d: species buffer parity differs", i);
            if (s.q_ph >= 0) return fail(LPIC_EUNSUPPORTED, "grid %d: ensembles have no fused emission", i);
        }
        for (int j = 0; j < i; ++j)
            if (grids[j] == g) return fail(LPIC_EINVAL, "grid %d appears twice", i);
    }
    auto* e = new (std::nothrow) lpic_ensemble;
    if (!e) return fail(LPIC_ENOMEM, "host allocation failed");
    e->grids.assign(grids, grids + n);
    e->dim = g0->d.dim; e->order = g0->d.shape_order; e->ninst = n; e->nsm = g0->nsm;
    // members keep their own tile shape and particles per block (each work
    // item lays out its shared memory from its slot's tiles); the persistent
    // kernel is launched with the largest member's shared memory
    e->smem = 0;
    for (int i = 0; i < n; ++i) e->smem = std::max(e->smem, grids[i]->smem32);
    e->parity = g0->sp[0].cur;
    std::vector<EnsField> hf(n);
    std::vector<EnsSort> hs;
    std::vector<GpdArgs> ha[2];
    std::vector<double> density;
    for (int i = 0; i < n; ++i) {
        lpic_grid* g = grids[i];
        EnsField& f = hf[i];
        f.g = g->geo;
        for (int c = 0; c < 3; ++c) {
            f.a.E[c] = static_cast<float*>(g->d.E[c]);
            f.a.B[c] = static_cast<float*>(g->d.B[c]);
            f.a.J[c] = static_cast<const long long*>(g->d.J[c]);
            f.J[c] = static_cast<unsigned long long*>(g->d.J[c]);
        }
        const double tau = 0.5 * g->d.dt;
        f.a.rdx = (float)(1.0 / g->d.dx); f.a.rdy = (float)(1.0 / g->d.dy);
        f.a.rdz = (float)(g->d.dim == 3 ? 1.0 / g->d.dz : 0.0);
        f.a.tau = (float)tau;
        for (int c = 0; c < 3; ++c) f.a.jfac[c] = tau * g->jscale[c];
        f.a.dfx = make_fastdiv((unsigned)g->geo.fx);
        f.a.dny = make_fastdiv((unsigned)g->d.ny);
        f.nfield = g->nfield;
        e->max_field = std::max(e->max_field, g->nfield);
        e->max_ntiles = std::max(e->max_ntiles, g->ntiles);
        for (int sidx = 0; sidx < (int)g->sp.size(); ++sidx) {
            Species& s = g->sp[sidx];
            e->slots.push_back({i, sidx});
            e->max_cap = std::max(e->max_cap, s.cap);
            EnsSort so{};
            for (int b = 0; b < 2; ++b) {
                const P32 src = view32(g, s, b), dst = view32(g, s, 1 - b);
                so.key[b] = KeyFP32{src.cell, g->dec, g->fT[0], g->fT[1], g->fT[2], g->nt[0], g->nt[1], (int)g->ntiles};
                so.mv[b] = MoveFP32{src, dst, g->d.dim};
                Tiles t{};
                for (int d = 0; d < 3; ++d) { t.T[d] = g->T[d]; t.nt[d] = g->nt[d]; t.m[d] = g->m[d]; t.fT[d] = g->fT[d]; }
                t.start = s.d_start; t.items = s.d_items; t.nitems = s.d_nitems; t.P = g->P; t.bmax = move_bound(g, s); t.R = fold_rounds(g->d);
                box_divisors(g, t);
                t.next_count = s.d_count; t.esc = s.d_esc; t.nesc = s.d_nesc;
                // the push runs after the step's sort flipped the parity: it
                // reads the buffer the particles were sorted into
                const P32 pv = view32(g, s, b);
                const float k = (float)(s.q * g->d.dt / (2.0 * s.m));
                const float sq = (float)std::ldexp(s.q, g->F);
                ha[b].push_back(GpdArgs{g->geo, ptr3<const float>(g->d.E), ptr3<const float>(g->d.B),
                                        ptr3<const double>(g->d.E), ptr3<const double>(g->d.B), 0,
                                        ptr3<unsigned long long>(g->d.J), pv, t, g->dec, k, sq,
                                        (float)(g->d.dt / g->d.dx), (float)(g->d.dt / g->d.dy),
                                        (float)(g->d.dt / (g->d.dim == 3 ? g->d.dz : 1.0)), g->d_status});
            }
            so.n = s.d_n; so.count = s.d_count; so.start = s.d_start; so.cursor = s.d_cursor;
            so.coff = s.d_coff; so.items = s.d_items; so.nitems = s.d_nitems; so.nesc = s.d_nesc;
            so.ntiles = (int)g->ntiles; so.P = g->P;
            hs.push_back(so);
            density.push_back((double)s.count0 / (double)((long long)g->d.nx * g->d.ny * g->geo.nz));
        }
    }
    e->nslots = (int)hs.size();
    // queue order: densest slots first (their work items are the fullest)
    std::vector<int> order(e->nslots);
    for (int i = 0; i < e->nslots; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return density[a] > density[b]; });
    auto cleanup = [&](lpic_status st, const char* msg) { lpic_destroy_ensemble(e); return fail(st, "%s", msg); };
    if (dev_alloc(&e->d_fields, sizeof(EnsField) * n) != cudaSuccess ||
        dev_alloc(&e->d_sort, sizeof(EnsSort) * e->nslots) != cudaSuccess ||
        dev_alloc(&e->d_args[0], sizeof(GpdArgs) * e->nslots) != cudaSuccess ||
        dev_alloc(&e->d_args[1], sizeof(GpdArgs) * e->nslots) != cudaSuccess ||
        dev_alloc(&e->d_order, sizeof(int) * e->nslots) != cudaSuccess ||
        dev_alloc(&e->d_prefix, sizeof(int) * (e->nslots + 1)) != cudaSuccess ||
        dev_alloc(&e->d_head, 64) != cudaSuccess ||
        dev_alloc(&e->d_status, 64) != cudaSuccess)
        return cleanup(LPIC_ENOMEM, "ensemble table allocation failed");
    if (cudaMemcpy(e->d_fields, hf.data(), sizeof(EnsField) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e->d_sort, hs.data(), sizeof(EnsSort) * e->nslots, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e->d_args[0], ha[0].data(), sizeof(GpdArgs) * e->nslots, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e->d_args[1], ha[1].data(), sizeof(GpdArgs) * e->nslots, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e->d_order, order.data(), sizeof(int) * e->nslots, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(e->d_status, 0, 64) != cudaSuccess)
        return cleanup(LPIC_ECUDA, "ensemble table upload failed");
    const void* fn = nullptr;
    cudaError_t ce = e->dim == 2 ? (e->order == 1 ? ens_attrs<2, 1>(e->smem, &fn) : ens_attrs<2, 2>(e->smem, &fn))
                                 : (e->order == 1 ? ens_attrs<3, 1>(e->smem, &fn) : ens_attrs<3, 2>(e->smem, &fn));
    if (ce != cudaSuccess) return cleanup(LPIC_ECUDA, "queue kernel shared memory attribute failed");
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, e->smem) != cudaSuccess || per_sm < 1) per_sm = 1;
    e->blocks = per_sm * e->nsm;
    e->counted = false;     // the first step counts the tile keys itself
    *out = e;
    return LPIC_OK;
}

lpic_status lpic_destroy_ensemble(lpic_ensemble_t e) {
    if (!e) return LPIC_OK;
    cudaDeviceSynchronize();
    for (auto& kv : e->graphs) cudaGraphExecDestroy(kv.second);
    cudaFree(e->d_fields); cudaFree(e->d_sort); cudaFree(e->d_args[0]); cudaFree(e->d_args[1]);
    cudaFree(e->d_order); cudaFree(e->d_prefix); cudaFree(e->d_head); cudaFree(e->d_status);
    delete e;
    return LPIC_OK;
}

lpic_status lpic_ensemble_step(lpic_ensemble_t e, cudaStream_t st) {
    if (!e) return fail(LPIC_EINVAL, "ensemble is NULL");
    if (lpic_status r = ens_step_impl(e, st)) return r;
    ens_sync_grids(e);
    return LPIC_OK;
}

lpic_status lpic_ensemble_graph_steps(lpic_ensemble_t e, int nsteps, cudaStream_t st) {
    if (!e) return fail(LPIC_EINVAL, "ensemble is NULL");
    if (nsteps < 0) return fail(LPIC_EINVAL, "nsteps must be >= 0");
    if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread)
        return fail(LPIC_EINVAL, "graph capture needs a created (non-default) stream");
    for (int k = 0; k < nsteps; ++k) {
        const int key = e->parity | (e->counted ? 2 : 0);
        auto it = e->graphs.find(key);
        if (it == e->graphs.end()) {
            const int parity0 = e->parity;
            const bool counted0 = e->counted;
            const long long l0 = e->launches;
            LPIC_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            lpic_status r = ens_step_impl(e, st);
            cudaGraph_t graph = nullptr;
            cudaError_t ce = cudaStreamEndCapture(st, &graph);
            e->parity = parity0; e->counted = counted0;
            const long long per = e->launches - l0;
            e->launches = l0;
            if (r != LPIC_OK) { if (graph) cudaGraphDestroy(graph); return r; }
            if (ce != cudaSuccess) return fail(LPIC_ECUDA, "stream capture: %s", cudaGetErrorString(ce));
            cudaGraphExec_t exec = nullptr;
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return fail(LPIC_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
            e->graphs[key] = exec;
            e->graph_launches[key] = per;
            it = e->graphs.find(key);
        }
        LPIC_CUDA(cudaGraphLaunch(it->second, st));
        e->launches += e->graph_launches[key];
        e->parity ^= 1;
        e->counted = true;
        ens_sync_grids(e);
    }
    return LPIC_OK;
}

lpic_status lpic_ensemble_check_status(lpic_ensemble_t e, cudaStream_t st, unsigned* bits) {
    if (!e) return fail(LPIC_EINVAL, "ensemble is NULL");
    unsigned b = 0;
    LPIC_CUDA(cudaMemcpyAsync(&b, e->d_status, 4, cudaMemcpyDeviceToHost, st));
    LPIC_CUDA(cudaStreamSynchronize(st));
    for (auto g : e->grids) {
        unsigned gb = 0;
        LPIC_CUDA(cudaMemcpyAsync(&gb, g->d_status, 4, cudaMemcpyDeviceToHost, st));
        LPIC_CUDA(cudaStreamSynchronize(st));
        b |= gb;
        LPIC_CUDA(cudaMemsetAsync(g->d_status, 0, 4, st));
    }
    LPIC_CUDA(cudaMemsetAsync(e->d_status, 0, 4, st));
    LPIC_CUDA(cudaStreamSynchronize(st));
    if (bits) *bits = b;
    if (b) return fail(LPIC_EDEVICE, "device status bits 0x%x", b);
    return LPIC_OK;
}

lpic_status lpic_ensemble_launches(lpic_ensemble_t e, long long* launches) {
    if (!e || !launches) return fail(LPIC_EINVAL, "NULL argument");
    *launches = e->launches;
    return LPIC_OK;
}


// ------------------------------------------------- nonlinear Compton (Sec. 3.4)
lpic_status lpic_qed_init(lpic_grid_t g, double eps_ref, uint64_t seed, cudaStream_t st) {
    if (lpic_status r = check_grid(g)) return r;
    if (g->d.precision != LPIC_FP32_FIXED) return fail(LPIC_EUNSUPPORTED, "QED events need the FP32 path");
    if (g->d.maxwell_fp64) return fail(LPIC_EUNSUPPORTED, "QED events read float fields (no maxwell_fp64)");
    if (!(eps_ref > 0) || !std::isfinite(eps_ref)) return fail(LPIC_EINVAL, "eps_ref must be positive");
    if (!g->d_qtab) {
        const QedHostTables H = qed_build_tables(1e-4, 1e3, 32, 513);
        const size_t n = H.logh.size() + H.top.size() + H.cdf.size();
        float* d = nullptr;
        if (dev_alloc(&d, n * sizeof(float)) != cudaSuccess) return fail(LPIC_ENOMEM, "QED table allocation failed");
        g->d_qtab = d;
        LPIC_CUDA(cudaMemcpyAsync(d, H.logh.data(), H.logh.size() * 4, cudaMemcpyHostToDevice, st));
        LPIC_CUDA(cudaMemcpyAsync(d + H.nchi, H.top.data(), H.top.size() * 4, cudaMemcpyHostToDevice, st));
        LPIC_CUDA(cudaMemcpyAsync(d + 2 * H.nchi, H.cdf.data(), H.cdf.size() * 4, cudaMemcpyHostToDevice, st));
        LPIC_CUDA(cudaStreamSynchronize(st));
        QedTab& T = g->qtab;
        T.logh = d; T.top = d + H.nchi; T.cdf = d + 2 * H.nchi;
        T.nchi = H.nchi; T.ny = H.ny;
        T.lchi0 = (float)H.lchi0; T.inv_dl = (float)(1.0 / H.dl); T.chi0 = (float)std::exp(H.lchi0);
    }
    if (!g->d_btab) {
        const BwHostTables H = bw_build_tables(1e-2, 1e3, 32, 513);
        const size_t n = H.g.size() + H.cdf.size();
        float* d = nullptr;
        if (dev_alloc(&d, n * sizeof(float)) != cudaSuccess) return fail(LPIC_ENOMEM, "QED table allocation failed");
        g->d_btab = d;
        LPIC_CUDA(cudaMemcpyAsync(d, H.g.data(), H.g.size() * 4, cudaMemcpyHostToDevice, st));
        LPIC_CUDA(cudaMemcpyAsync(d + H.nchi, H.cdf.data(), H.cdf.size() * 4, cudaMemcpyHostToDevice, st));
        LPIC_CUDA(cudaStreamSynchronize(st));
        BwTab& T = g->btab;
        T.g = d; T.cdf = d + H.nchi;
        T.nchi = H.nchi; T.ny = H.ny;
        T.lchi0 = (float)H.lchi0; T.inv_dl = (float)(1.0 / H.dl); T.chi0 = (float)std::exp(H.lchi0);
    }
    const double alpha = 1.0 / 137.035999084;
    g->qtab.pref = (float)(alpha / (eps_ref * std::sqrt(3.0) * M_PI));
    g->qtab.eps_ref = (float)eps_ref;
    g->btab.pref = g->qtab.pref;
    g->btab.eps_ref = (float)eps_ref;
    g->eps_ref = eps_ref;
    g->seed[0] = (uint32_t)(seed & 0xffffffffu);
    g->seed[1] = (uint32_t)(seed >> 32);
    g->qed = true;
    return LPIC_OK;
}

lpic_status lpic_qed_initial_tau(lpic_grid_t g, float* tau, long long n_ids, int photons, cudaStream_t st) {
    if (lpic_status r = check_grid(g)) return r;
    if (!g->qed) return fail(LPIC_EINVAL, "call lpic_qed_init first");
    if (n_ids < 0 || (n_ids > 0 && !tau)) return fail(LPIC_EINVAL, "tau is NULL or n_ids negative");
    if (n_ids == 0) return LPIC_OK;
    k_qed_tau0<<<grid_blocks(n_ids, g->nsm), 256, 0, st>>>(tau, n_ids, photons ? 3u : 2u, g->seed[0], g->seed[1]);
    LPIC_LAUNCHED("k_qed_tau0");
    return LPIC_OK;
}

lpic_status lpic_qed_compton(lpic_grid_t g, int sid_e, int sid_ph, float* tau, long long n_ids, float* ph_tau,
                             long long ph_n_ids, long long step, cudaStream_t st) {
    if (lpic_status r = check_species(g, sid_e)) return r;
    if (lpic_status r = check_species(g, sid_ph)) return r;
    if (!g->qed) return fail(LPIC_EINVAL, "call lpic_qed_init first");
    if (sid_e == sid_ph) return fail(LPIC_EINVAL, "the emitting and the photon species must differ");
    Species& e = g->sp[sid_e];
    Species& ph = g->sp[sid_ph];
    if (e.massless) return fail(LPIC_EINVAL, "species %d is massless and cannot emit", sid_e);
    if (!ph.massless) return fail(LPIC_EINVAL, "species %d must be massless and charge-free", sid_ph);
    if (n_ids < 0 || (n_ids > 0 && !tau)) return fail(LPIC_EINVAL, "tau is NULL or n_ids negative");
    if (step < 0 || step > 0xffffffffLL) return fail(LPIC_EINVAL, "step must fit 32 bits");
    if (ph_n_ids < 0 || (ph_n_ids > 0 && !ph_tau)) return fail(LPIC_EINVAL, "photon_tau is NULL or its length negative");
    QedArgs A{};
    A.g = g->geo;
    A.E = ptr3<const float>(g->d.E);
    A.B = ptr3<const float>(g->d.B);
    A.e = view32(g, e, e.cur);
    A.ph = view32(g, ph, ph.cur);
    A.ph_n = ph.d_n;
    A.ph_next_id = ph.d_n + 1;
    A.ph_cap = ph.cap;
    A.dec = g->dec;
    A.T = g->qtab;
    A.tau = tau;
    A.n_ids = n_ids;
    A.ph_tau = ph_n_ids > 0 ? ph_tau : nullptr;
    A.ph_n_ids = ph_n_ids;
    A.dt = (float)g->d.dt;
    A.dth0 = (float)(g->d.dt / g->d.dx);
    A.dth1 = (float)(g->d.dt / g->d.dy);
    A.dth2 = (float)(g->d.dt / (g->d.dim == 3 ? g->d.dz : 1.0));
    A.k0 = g->seed[0]; A.k1 = g->seed[1];
    A.step = (uint32_t)step;
    A.st = g->d_status;
    const int nb = grid_blocks(e.cap, g->nsm, 16);
    const int D = g->d.dim, O = g->d.shape_order;
    if (D == 2) { if (O == 1) k_qed_compton32<2, 1><<<nb, 256, 0, st>>>(A); else k_qed_compton32<2, 2><<<nb, 256, 0, st>>>(A); }
    else        { if (O == 1) k_qed_compton32<3, 1><<<nb, 256, 0, st>>>(A); else k_qed_compton32<3, 2><<<nb, 256, 0, st>>>(A); }
    LPIC_LAUNCHED("k_qed_compton32");
    k_qed_clamp<<<1, 32, 0, st>>>(ph.d_n, ph.cap);
    LPIC_LAUNCHED("k_qed_clamp");
    ph.counts_fresh = false;
    return LPIC_OK;
}

lpic_status lpic_qed_fuse(lpic_grid_t g, int sid_e, int sid_ph, float* tau, long long n_ids, float* ph_tau,
                          long long ph_n_ids, long long first_step, cudaStream_t st) {
    if (lpic_status r = check_species(g, sid_e)) return r;
    if (!g->qed) return fail(LPIC_EINVAL, "call lpic_qed_init first");
    Species& e = g->sp[sid_e];
    if (e.massless) return fail(LPIC_EINVAL, "species %d is massless and cannot emit", sid_e);
    if (sid_ph >= 0) {
        if (lpic_status r = check_species(g, sid_ph)) return r;
        if (!g->sp[sid_ph].massless) return fail(LPIC_EINVAL, "species %d must be massless and charge-free", sid_ph);
        if (sid_ph < sid_e)
            return fail(LPIC_EINVAL, "the photon species (%d) must come after the emitting species (%d): a step "
                        "moves the photons emitted at x^{n+1/2} with the photon push that follows", sid_ph, sid_e);
        if (n_ids < 0 || (n_ids > 0 && !tau)) return fail(LPIC_EINVAL, "tau is NULL or n_ids negative");
        if (ph_n_ids < 0 || (ph_n_ids > 0 && !ph_tau)) return fail(LPIC_EINVAL, "photon_tau is NULL or its length negative");
        if (first_step < 0 || first_step > 0xffffffffLL) return fail(LPIC_EINVAL, "first_step must fit 32 bits");
    }
    // captured steps launch the kernel form of each species: drop them
    LPIC_CUDA(cudaDeviceSynchronize());
    for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second);
    g->graphs.clear();
    g->graph_launches.clear();
    if (sid_ph < 0) {
        e.q_ph = -1;
        return LPIC_OK;
    }
    if (!g->d_qstep && dev_alloc(&g->d_qstep, 64) != cudaSuccess)
        return fail(LPIC_ENOMEM, "step counter allocation failed");
    e.q_ph = sid_ph;
    e.q_tau = tau;
    e.q_nids = n_ids;
    e.q_phtau = ph_tau;
    e.q_phnids = ph_n_ids;
    k_set_uint<<<1, 32, 0, st>>>(g->d_qstep, (unsigned)first_step);
    LPIC_LAUNCHED("k_set_uint");
    return LPIC_OK;
}

lpic_status lpic_qed_set_step(lpic_grid_t g, long long step, cudaStream_t st) {
    if (lpic_status r = check_grid(g)) return r;
    if (!g->d_qstep) return fail(LPIC_EINVAL, "no species emits inside its push (lpic_qed_fuse)");
    if (step < 0 || step > 0xffffffffLL) return fail(LPIC_EINVAL, "step must fit 32 bits");
    k_set_uint<<<1, 32, 0, st>>>(g->d_qstep, (unsigned)step);
    LPIC_LAUNCHED("k_set_uint");
    return LPIC_OK;
}

lpic_status lpic_debug_fail_alloc(long long nth) {
    if (nth < 0) return fail(LPIC_EINVAL, "nth must be >= 0");
    g_alloc_seen.store(0);
    g_alloc_fail_at.store(nth);
    return LPIC_OK;
}

lpic_status lpic_qed_eval(lpic_grid_t g, const double* chi, const double* r, long long n, double* h, double* xi,
                          cudaStream_t st) {
    if (lpic_status rr = check_grid(g)) return rr;
    if (!g->qed) return fail(LPIC_EINVAL, "call lpic_qed_init first");
    if (n < 0 || (n > 0 && (!chi || !r || !h || !xi))) return fail(LPIC_EINVAL, "NULL array or negative n");
    if (n == 0) return LPIC_OK;
    k_qed_eval<<<grid_blocks(n, g->nsm), 256, 0, st>>>(g->qtab, chi, r, n, h, xi);
    LPIC_LAUNCHED("k_qed_eval");
    return LPIC_OK;
}


lpic_status lpic_qed_breit_wheeler(lpic_grid_t g, int sid_ph, int sid_el, int sid_po, float* tau, long long n_ids,
                                   long long step, cudaStream_t st) {
    if (lpic_status r = check_species(g, sid_ph)) return r;
    if (lpic_status r = check_species(g, sid_el)) return r;
    if (lpic_status r = check_species(g, sid_po)) return r;
    if (!g->qed) return fail(LPIC_EINVAL, "call lpic_qed_init first");
    Species& ph = g->sp[sid_ph];
    Species& el = g->sp[sid_el];
    Species& po = g->sp[sid_po];
    if (!ph.massless) return fail(LPIC_EINVAL, "species %d must be massless and charge-free", sid_ph);
    if (el.massless || po.massless) return fail(LPIC_EINVAL, "the pair species must be massive");
    if (n_ids < 0 || (n_ids > 0 && !tau)) return fail(LPIC_EINVAL, "tau is NULL or n_ids negative");
    if (step < 0 || step > 0xffffffffLL) return fail(LPIC_EINVAL, "step must fit 32 bits");
    BwArgs A{};
    QedArgs& Q = A.q;
    Q.g = g->geo;
    Q.E = ptr3<const float>(g->d.E);
    Q.B = ptr3<const float>(g->d.B);
    Q.e = view32(g, ph, ph.cur);
    Q.dec = g->dec;
    Q.tau = tau;
    Q.n_ids = n_ids;
    Q.dt = (float)g->d.dt;
    Q.dth0 = (float)(g->d.dt / g->d.dx);
    Q.dth1 = (float)(g->d.dt / g->d.dy);
    Q.dth2 = (float)(g->d.dt / (g->d.dim == 3 ? g->d.dz : 1.0));
    Q.k0 = g->seed[0]; Q.k1 = g->seed[1];
    Q.step = (uint32_t)step;
    Q.st = g->d_status;
    A.T = g->btab;
    A.el = view32(g, el, el.cur);
    A.po = view32(g, po, po.cur);
    A.el_n = el.d_n; A.po_n = po.d_n;
    A.el_next_id = el.d_n + 1; A.po_next_id = po.d_n + 1;
    A.el_cap = el.cap; A.po_cap = po.cap;
    A.el_wmax = (float)el.wmax; A.po_wmax = (float)po.wmax;
    const int nb = grid_blocks(ph.cap, g->nsm, 16);
    const int D = g->d.dim, O = g->d.shape_order;
    if (D == 2) { if (O == 1) k_qed_bw32<2, 1><<<nb, 256, 0, st>>>(A); else k_qed_bw32<2, 2><<<nb, 256, 0, st>>>(A); }
    else        { if (O == 1) k_qed_bw32<3, 1><<<nb, 256, 0, st>>>(A); else k_qed_bw32<3, 2><<<nb, 256, 0, st>>>(A); }
    LPIC_LAUNCHED("k_qed_bw32");
    k_qed_clamp<<<1, 32, 0, st>>>(el.d_n, el.cap);
    LPIC_LAUNCHED("k_qed_clamp");
    if (&po != &el) {
        k_qed_clamp<<<1, 32, 0, st>>>(po.d_n, po.cap);
        LPIC_LAUNCHED("k_qed_clamp");
    }
    // the new particles sit after the tiles' ranges: sort before the next push
    for (Species* s : {&el, &po}) {
        s->since_sort = std::max(s->since_sort, g->K);
        s->counts_fresh = false;
    }
    ph.counts_fresh = false;
    return LPIC_OK;
}

lpic_status lpic_qed_pair_eval(lpic_grid_t g, const double* chi, const double* r, long long n, double* h,
                               double* eta, cudaStream_t st) {
    if (lpic_status rr = check_grid(g)) return rr;
    if (!g->qed) return fail(LPIC_EINVAL, "call lpic_qed_init first");
    if (n < 0 || (n > 0 && (!chi || !r || !h || !eta))) return fail(LPIC_EINVAL, "NULL array or negative n");
    if (n == 0) return LPIC_OK;
    k_bw_eval<<<grid_blocks(n, g->nsm), 256, 0, st>>>(g->btab, chi, r, n, h, eta);
    LPIC_LAUNCHED("k_bw_eval");
    return LPIC_OK;
}


lpic_status lpic_species_checkpoint_info(lpic_grid_t g, int sid, cudaStream_t st, double* max_weight,
                                         long long* next_id) {
    if (lpic_status r = check_species(g, sid)) return r;
    if (!max_weight || !next_id) return fail(LPIC_EINVAL, "NULL output");
    int n2[2] = {0, 0};
    LPIC_CUDA(cudaMemcpyAsync(n2, g->sp[sid].d_n, sizeof(n2), cudaMemcpyDeviceToHost, st));
    LPIC_CUDA(cudaStreamSynchronize(st));
    *max_weight = g->sp[sid].wmax;
    *next_id = n2[1];
    return LPIC_OK;
}

lpic_status lpic_species_set_next_id(lpic_grid_t g, int sid, long long next_id, cudaStream_t st) {
    if (lpic_status r = check_species(g, sid)) return r;
    if (next_id < 0 || next_id >= (1LL << 31)) return fail(LPIC_EINVAL, "next_id %lld outside [0, 2^31)", next_id);
    k_set_int<<<1, 32, 0, st>>>(g->sp[sid].d_n + 1, (int)next_id);
    LPIC_LAUNCHED("k_set_int");
    return LPIC_OK;
}

}  // extern "C"
