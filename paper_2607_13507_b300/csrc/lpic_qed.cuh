// Nonlinear Compton emission (Sec. 3.4) on the FP32 path, and the ballistic
// push of massless, charge-free species (the emitted photons).
//
// Physics (locally-constant-field approximation, normalised units: momenta
// in m c, fields in m c omega_ref / e, eps_ref = hbar omega_ref / (m c^2)):
//   chi_e = eps_ref gamma sqrt((E + beta x B)^2 - (beta . E)^2),
//   dW / dxi = alpha / (eps_ref sqrt(3) pi gamma) S(xi, chi),
//   S = (1 - xi + 1 / (1 - xi)) K_{2/3}(delta) - int_delta^inf K_{1/3},
//   delta = 2 xi / (3 chi (1 - xi)),
// W = int_0^1 dW/dxi.  Each particle carries an optical depth tau (indexed by
// its id); per step tau decreases by W dt and when it reaches zero a photon of
// energy fraction xi (drawn from the normalised cumulative of S) is emitted
// along the particle's momentum, the particle recoils and tau restarts at
// -ln r.  Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
// counter (id, step, kind, 0), key (seed_lo, seed_hi).
//
// Tables (built on the host at lpic_qed_init, read from global memory, where
// they stay L2-resident):
//   logh[i]  = ln h(chi_i), h(chi) = int_0^1 S(xi, chi) dxi, chi_i = chi_0 e^{i dl}
//   cdf[i][j] = normalised cumulative of S at xi = top_i m_i(y_j), y_j = j/(ny-1),
//   top_i = min(1, 60 chi_i) (the spectrum is negligible beyond 40 e-folds),
//   m(y) = y^3 (top < 1) or y^3 (10 - 15 y + 6 y^2) (top = 1, which also
//   resolves the (1 - xi)^{-1/3} edge of the spectrum at large chi).
// Below chi_0 the classical limit is used: h and xi are proportional to chi.
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>
#include "lpic_fp32.cuh"

namespace lpic {

// --------------------------------------------------------------- the kernels
// Initial optical depths tau[id] = -ln r, r from counter (id, 0, kind, 0):
// kind 2 for emitting particles, 3 for photons (pair creation).
__global__ void k_qed_tau0(float* tau, long long n_ids, uint32_t kind, uint32_t k0, uint32_t k1) {
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n_ids;
         id += (long long)gridDim.x * blockDim.x) {
        const U4 o = philox4x32_10(U4{(uint32_t)id, 0u, kind, 0u}, k0, k1);
        tau[id] = neg_log_u01(o.x);
    }
}

// Table lookups for given (chi, r): h(chi) and xi(chi, r).
__global__ void k_qed_eval(QedTab T, const double* chi, const double* r, long long n, double* h,
                           double* xi) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float c = (float)chi[i];
        const float rr = fminf((float)r[i], 0.99999994f);
        h[i] = c > 0.0f ? (double)qed_h(T, c) : 0.0;
        xi[i] = c > 0.0f ? (double)qed_xi(T, c, rr) : 0.0;
    }
}

struct QedArgs {
    Geo g;
    Ptr3<const float> E, B;
    P32 e;                 // emitting species (current buffer)
    P32 ph;                // photon species (current buffer); ph.n is appended to
    int* ph_n;             // == ph.n, writable
    int* ph_next_id;       // id of the next created photon
    long long ph_cap;
    CellDecode dec;
    QedTab T;
    float* tau;
    long long n_ids;
    float* ph_tau;         // optional: pair-creation depths of new photons, by photon id
    long long ph_n_ids;
    float dt, dth0, dth1, dth2;
    uint32_t k0, k1, step;
    unsigned* st;
};

// E and B at a particle in cell gc with offsets f, read from global memory
// (the grid's shape functions, staggering as in the particle push).  The
// stencil covers nodes gc - 1 .. gc + ORDER of each dimension: their wrapped
// indices are formed once, and every read is unconditional so that the 6
// (ORDER + 1)^DIM loads issue together.  Returns false (nothing read) when
// the stencil crosses an absorbing x edge.
template <int DIM, int ORDER>
__device__ __forceinline__ bool qed_gather(const QedArgs& A, const int (&gc)[3], const float (&f)[3],
                                           float (&fld)[6]) {
    constexpr int K = ORDER + 2;
    const Geo& g = A.g;
    int ix[K];
    long long ry[K], rz[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        int i = gc[0] - 1 + k;
        if (g.absorb) { if (i < 0 || i >= g.fx) return false; }
        else          { i = wrapn(i, g.nx); }
        ix[k] = i;
        ry[k] = (long long)wrapn(gc[1] - 1 + k, g.ny) * g.fx;
        rz[k] = DIM == 3 ? (long long)wrapn(gc[2] - 1 + k, g.nz) * g.ny * g.fx : 0;
    }
    const NodeW<ORDER> nx_(1, f[0]), ny_(1, f[1]), nz_(1, f[2]);
    const HalfW<ORDER> hx_(1, f[0]), hy_(1, f[1]), hz_(1, f[2]);
    const float* F[6] = {A.E.p[0], A.E.p[1], A.E.p[2], A.B.p[0], A.B.p[1], A.B.p[2]};
#pragma unroll
    for (int comp = 0; comp < 6; ++comp) {
        // E_x (h,n,n), E_y (n,h,n), E_z (n,n,h), B_x (n,h,h), B_y (h,n,h), B_z (h,h,n)
        const bool hx = (comp == 0 || comp == 4 || comp == 5);
        const bool hy = (comp == 1 || comp == 3 || comp == 5);
        const bool hz = (comp == 2 || comp == 3 || comp == 4);
        const int bx = hx ? hx_.base : nx_.base, by = hy ? hy_.base : ny_.base;
        const int bz = hz ? hz_.base : nz_.base;
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < (DIM == 3 ? ORDER + 1 : 1); ++c) {
            const long long oz = DIM == 3 ? (bz ? rz[c + 1] : rz[c]) : 0;
            float accb = 0.0f;
#pragma unroll
            for (int b = 0; b <= ORDER; ++b) {
                const long long oy = oz + (by ? ry[b + 1] : ry[b]);
                float r = 0.0f;
#pragma unroll
                for (int a = 0; a <= ORDER; ++a) {
                    const float v = __ldg(F[comp] + oy + (bx ? ix[a + 1] : ix[a]));
                    r = __fmaf_rn(v, hx ? hx_.w[a] : nx_.w[a], r);
                }
                accb = __fmaf_rn(r, hy ? hy_.w[b] : ny_.w[b], accb);
            }
            acc = DIM == 3 ? __fmaf_rn(accb, hz ? hz_.w[c] : nz_.w[c], acc) : accb;
        }
        fld[comp] = acc;
    }
    return true;
}

// One pass over the emitting species after its push.  The fields are
// gathered at x - (dt/2) v, the particle's position at the time of its
// momentum u (the stored position is half a step ahead of it).
template <int DIM, int ORDER>
__global__ void __launch_bounds__(256) k_qed_compton32(QedArgs A) {
    const P32& p = A.e;
    const int n = *p.n;
    const float dth[3] = {A.dth0, A.dth1, A.dth2};
    const QedEmit Q{A.T, A.tau, A.n_ids, A.ph, A.ph_n, A.ph_next_id, A.ph_cap, A.ph_tau, A.ph_n_ids, A.dt,
                    A.k0, A.k1, nullptr};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int cell = p.cell[i];
        if (cell < 0) continue;
        const int id = p.id[i];
        if (id < 0 || (long long)id >= A.n_ids) { set_status(A.st, LPIC_ST_OVERFLOW); continue; }
        float u[3] = {p.u[0][i], p.u[1][i], p.u[2][i]};
        const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const float ig = 1.0f / sqrtf(1.0f + u2);
        int gc[3];
        A.dec(cell, gc);
        if (DIM == 2) gc[2] = 0;
        float f[3] = {0.0f, 0.0f, 0.0f}, off[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            off[d] = p.off[d][i];
            float fd = off[d] - 0.5f * dth[d] * u[d] * ig;
            if (fd < 0.0f) { fd += 1.0f; gc[d] -= 1; if (fd >= 1.0f) fd = 0.99999994f; }
            else if (fd >= 1.0f) { fd -= 1.0f; gc[d] += 1; }
            f[d] = fd;
        }
        float fld[6];
        if (!qed_gather<DIM, ORDER>(A, gc, f, fld)) { set_status(A.st, LPIC_ST_OUTSIDE); continue; }
        // the photon is stored at the emitter's stored position
        if (qed_emit(Q, A.step, DIM, id, A.tau[id], cell, off, p.w[i], u, fld, A.st)) {
#pragma unroll
            for (int c = 0; c < 3; ++c) p.u[c][i] = u[c];
        }
    }
}

// One int written on the device (stream-ordered, no host buffer to keep alive).
__global__ void k_set_int(int* p, int v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

// After the emission pass: a photon count past the capacity is cut back.
__global__ void k_qed_clamp(int* n, long long cap) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && (long long)*n > cap) *n = (int)cap;
}

// Massless particles move at c along u: offsets advance by frac dt u / (|u| h)
// with carries into the cell (at most one per dimension under the Courant
// limit).  With absorbing x edges a particle is removed once its cell is
// within `edge` cells of an edge (2 in a step, as for charged particles,
// whose deposit stencils must stay on the grid; 0 at the initial half push).
template <int DIM>
__global__ void k_photon32(Geo g, P32 p, CellDecode dec, float frac, float dth0, float dth1, float dth2,
                           int edge) {
    const int n = *p.n;
    const float dth[3] = {dth0, dth1, dth2};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int cell = p.cell[i];
        if (cell < 0) continue;
        int gc[3];
        dec(cell, gc);
        const float uu[3] = {p.u[0][i], p.u[1][i], p.u[2][i]};
        const float um = sqrtf(uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
        const float iu = um > 0.0f ? 1.0f / um : 0.0f;
        const int nn[3] = {g.nx, g.ny, g.nz};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const float fr = p.off[d][i] + frac * uu[d] * iu * dth[d];
            int carry = (int)floorf(fr);
            float fn = fr - (float)carry;
            if (fn >= 1.0f) { fn -= 1.0f; carry += 1; }
            gc[d] += carry;
            if (!(d == 0 && g.absorb)) gc[d] = wrapi(gc[d], nn[d]);
            p.off[d][i] = fn;
        }
        if (DIM == 2) gc[2] = 0;
        p.cell[i] = (gc[0] < edge || gc[0] >= g.nx - edge) ? -1 : (gc[2] * g.ny + gc[1]) * g.nx + gc[0];
    }
}

// ------------------------------------------------- Breit-Wheeler (Sec. 3.4)
// Pair creation by a photon of momentum k along khat:
//   chi_g = eps_ref k sqrt((E + khat x B)^2 - (khat . E)^2),
//   dW/deta = alpha / (eps_ref sqrt(3) pi k) F(eta, chi_g),
//   F = (eta/(1 - eta) + (1 - eta)/eta) K_{2/3}(z) + int_z^inf K_{1/3},
//   z = 2 / (3 chi_g eta (1 - eta)),
// eta the electron's energy share (F is symmetric in eta <-> 1 - eta).
// Tables: g_i = ln H(chi_i) + 8 / (3 chi_i), H = int_0^1 F deta (smooth in
// ln chi: the exp(-8 / (3 chi)) of the small-chi limit is taken out), and the
// normalised cumulative of F over eta in [0, 1/2] at eta = y^{3/2} / 2, y
// uniform (the cumulative grows like eta^{2/3} near 0 at large chi).  Below
// chi_0 = 0.01 the rate is below 1e-110 of its scale and is taken as 0.
struct BwTab {
    const float* g;        // [nchi]
    const float* cdf;      // [nchi][ny]
    int nchi, ny;
    float lchi0, inv_dl, chi0;
    float pref;            // alpha / (eps_ref sqrt(3) pi): W = pref H(chi) / k
    float eps_ref;
};

__device__ inline float bw_h(const BwTab& T, float chi) {
    if (!(chi >= T.chi0)) return 0.0f;
    const float u = (logf(chi) - T.lchi0) * T.inv_dl;
    const int i = min((int)u, T.nchi - 2);
    const float f = u - (float)i;
    return expf(T.g[i] + f * (T.g[i + 1] - T.g[i]) - 8.0f / (3.0f * chi));
}

// share in [0, 1/2] of half-cumulative probability s in row i
__device__ inline float bw_row_eta(const BwTab& T, int i, float s) {
    const float* P = T.cdf + (long long)i * T.ny;
    int lo = 0, hi = T.ny - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (P[mid] <= s) lo = mid; else hi = mid;
    }
    const float pa = P[lo], pb = P[hi];
    const float f = pb > pa ? fminf((s - pa) / (pb - pa), 1.0f) : 0.0f;
    const float y = ((float)lo + f) / (float)(T.ny - 1);
    return 0.5f * y * sqrtf(y);
}

// eta(chi, r): the half of the symmetric spectrum from r < 1/2 or not, the
// share within it from the half-cumulative, rows blended linearly in ln chi.
__device__ inline float bw_eta(const BwTab& T, float chi, float r) {
    float u = (logf(fmaxf(chi, T.chi0)) - T.lchi0) * T.inv_dl;
    u = fminf(fmaxf(u, 0.0f), (float)(T.nchi - 1));
    const int i = min((int)u, T.nchi - 2);
    const float f = u - (float)i;
    const bool low = r < 0.5f;
    const float s = low ? 2.0f * r : 2.0f * (1.0f - r);
    const float a = bw_row_eta(T, i, s), b = bw_row_eta(T, i + 1, s);
    const float e = a + f * (b - a);
    return low ? e : 1.0f - e;
}

__global__ void k_bw_eval(BwTab T, const double* chi, const double* r, long long n, double* h, double* eta) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float c = (float)chi[i];
        const float rr = fminf((float)r[i], 0.99999994f);
        h[i] = (double)bw_h(T, c);
        eta[i] = (double)bw_eta(T, c, rr);
    }
}

struct BwArgs {
    QedArgs q;             // geometry, fields, photon species as q.e, keys, step, status
    BwTab T;
    P32 el, po;            // receiving species (current buffers)
    int *el_n, *po_n, *el_next_id, *po_next_id;
    long long el_cap, po_cap;
    float el_wmax, po_wmax;  // weight bounds of the receiving species (fixed-point current)
};

// One pass over a photon species: photons at or below the pair threshold
// (|k| <= 2) never convert; a converted photon is removed (cell -1) and an
// electron (eta k) and a positron ((1 - eta) k) appear at its stored position
// with its weight.
template <int DIM, int ORDER>
__global__ void __launch_bounds__(256) k_qed_bw32(BwArgs A) {
    const QedArgs& Q = A.q;
    const P32& p = Q.e;
    const int n = *p.n;
    const float dth[3] = {Q.dth0, Q.dth1, Q.dth2};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int cell = p.cell[i];
        if (cell < 0) continue;
        const float k[3] = {p.u[0][i], p.u[1][i], p.u[2][i]};
        const float km = sqrtf(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        if (!(km > 2.0f)) continue;
        const int id = p.id[i];
        if (id < 0 || (long long)id >= Q.n_ids) { set_status(Q.st, LPIC_ST_OVERFLOW); continue; }
        const float ik = 1.0f / km;
        const float nn[3] = {k[0] * ik, k[1] * ik, k[2] * ik};
        int gc[3];
        Q.dec(cell, gc);
        if (DIM == 2) gc[2] = 0;
        float f[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            float fd = p.off[d][i] - 0.5f * dth[d] * nn[d];
            if (fd < 0.0f) { fd += 1.0f; gc[d] -= 1; if (fd >= 1.0f) fd = 0.99999994f; }
            else if (fd >= 1.0f) { fd -= 1.0f; gc[d] += 1; }
            f[d] = fd;
        }
        float fld[6];
        if (!qed_gather<DIM, ORDER>(Q, gc, f, fld)) { set_status(Q.st, LPIC_ST_OUTSIDE); continue; }
        const float F0 = fld[0] + nn[1] * fld[5] - nn[2] * fld[4];
        const float F1 = fld[1] + nn[2] * fld[3] - nn[0] * fld[5];
        const float F2 = fld[2] + nn[0] * fld[4] - nn[1] * fld[3];
        const float ne = nn[0] * fld[0] + nn[1] * fld[1] + nn[2] * fld[2];
        const float q2 = F0 * F0 + F1 * F1 + F2 * F2 - ne * ne;
        const float chi = A.T.eps_ref * km * sqrtf(fmaxf(q2, 0.0f));
        if (!(chi > 0.0f)) continue;
        const float t = Q.tau[id] - A.T.pref * bw_h(A.T, chi) * ik * Q.dt;
        Q.tau[id] = t;
        if (t > 0.0f) continue;
        const U4 o = philox4x32_10(U4{(uint32_t)id, Q.step, 1u, 0u}, Q.k0, Q.k1);
        const float r = u01f(o.x);
        const float eta = bw_eta(A.T, chi, r);
        const float w = p.w[i];
        const int je = atomicAdd(A.el_n, 1), jp = atomicAdd(A.po_n, 1);
        // a pair that does not fit (capacity, or a weight above the receiving
        // species' fixed-point bound) is not created: the photon stays, with
        // its spent depth, and converts at a later pass; a slot already taken
        // is written as a removed particle, which the next sort discards
        const bool fits = (long long)je < A.el_cap && (long long)jp < A.po_cap && w <= A.el_wmax &&
                          w <= A.po_wmax;
        if (!fits) {
            set_status(Q.st, LPIC_ST_OVERFLOW);
            if ((long long)je < A.el_cap) A.el.cell[je] = -1;
            if ((long long)jp < A.po_cap) A.po.cell[jp] = -1;
            continue;
        }
        p.cell[i] = -1;
        A.el.cell[je] = cell;
        A.po.cell[jp] = cell;
#pragma unroll
        for (int d = 0; d < DIM; ++d) { A.el.off[d][je] = p.off[d][i]; A.po.off[d][jp] = p.off[d][i]; }
#pragma unroll
        for (int c = 0; c < 3; ++c) { A.el.u[c][je] = eta * k[c]; A.po.u[c][jp] = k[c] - eta * k[c]; }
        A.el.w[je] = w;
        A.po.w[jp] = w;
        A.el.id[je] = atomicAdd(A.el_next_id, 1);
        A.po.id[jp] = atomicAdd(A.po_next_id, 1);
    }
}

// ---------------------------------------------------- host: building tables
// K_nu(x) and int_x^inf K_nu from K_nu(x) = int_0^inf e^{-x cosh t} cosh(nu t) dt
// (and the same integrand over cosh t for the tail integral).  The integrands
// are analytic in the strip |Im t| < pi/2 and decay double-exponentially, so
// the trapezoid rule with step 1/8 is accurate to far below double rounding.
inline void qed_bessel_pair(double x, double& k23, double& ik13) {
    const double h = 0.125;
    const double tmax = std::acosh(std::fmax(1.0, 80.0 / x)) + 1.0;
    double a = 0.5 * std::exp(-x), b = 0.5 * std::exp(-x);
    for (int m = 1; m * h <= tmax; ++m) {
        const double t = m * h, ch = std::cosh(t), e = std::exp(-x * ch);
        a += e * std::cosh(t * (2.0 / 3.0));
        b += e * std::cosh(t * (1.0 / 3.0)) / ch;
    }
    k23 = a * h;
    ik13 = b * h;
}

inline double qed_spectrum(double xi, double chi) {
    if (!(xi > 0.0) || !(xi < 1.0)) return 0.0;
    const double delta = 2.0 * xi / (3.0 * chi * (1.0 - xi));
    if (delta > 700.0) return 0.0;
    double k23, ik13;
    qed_bessel_pair(delta, k23, ik13);
    return (1.0 - xi + 1.0 / (1.0 - xi)) * k23 - ik13;
}

struct QedHostTables {
    int nchi = 0, ny = 0;
    double lchi0 = 0, dl = 0;
    std::vector<float> logh, cdf, top;
};

// Rows chi_i = chi_min 10^{i / per_decade} up to chi_max; cumulative by the
// trapezoid rule over y (the integrand S dxi/dy is finite at y = 0, where its
// limit is 3 Gamma(2/3) (3 chi)^{2/3} (c top)^{1/3} with xi ~ c top y^3).
inline QedHostTables qed_build_tables(double chi_min, double chi_max, int per_decade, int ny) {
    QedHostTables T;
    T.dl = std::log(10.0) / per_decade;
    T.lchi0 = std::log(chi_min);
    T.nchi = (int)std::floor((std::log(chi_max) - T.lchi0) / T.dl + 1e-9) + 1;
    T.ny = ny;
    T.logh.resize(T.nchi);
    T.top.resize(T.nchi);
    T.cdf.resize((size_t)T.nchi * ny);
    std::vector<double> g(ny), cum(ny);
    for (int i = 0; i < T.nchi; ++i) {
        const double chi = std::exp(T.lchi0 + i * T.dl);
        const double top = std::fmin(1.0, 60.0 * chi);
        const bool step = !(top < 1.0);
        const double c = step ? 10.0 : 1.0;
        g[0] = 3.0 * std::tgamma(2.0 / 3.0) * std::pow(3.0 * chi, 2.0 / 3.0) * std::cbrt(c * top);
        for (int j = 1; j < ny; ++j) {
            const double y = (double)j / (ny - 1);
            const double m = step ? y * y * y * (10.0 + y * (-15.0 + 6.0 * y)) : y * y * y;
            const double dm = step ? 30.0 * y * y * (1.0 - y) * (1.0 - y) : 3.0 * y * y;
            g[j] = (j == ny - 1 && step) ? 0.0 : qed_spectrum(top * m, chi) * top * dm;
        }
        cum[0] = 0.0;
        for (int j = 1; j < ny; ++j) cum[j] = cum[j - 1] + 0.5 * (g[j - 1] + g[j]) / (ny - 1);
        const double total = cum[ny - 1];
        T.logh[i] = (float)std::log(total);
        T.top[i] = (float)top;
        for (int j = 0; j < ny; ++j) T.cdf[(size_t)i * ny + j] = (float)(cum[j] / total);
        T.cdf[(size_t)i * ny + ny - 1] = 1.0f;
    }
    return T;
}


inline double bw_spectrum(double eta, double chi) {
    if (!(eta > 0.0) || !(eta < 1.0)) return 0.0;
    const double z = 2.0 / (3.0 * chi * eta * (1.0 - eta));
    if (z > 700.0) return 0.0;
    double k23, ik13;
    qed_bessel_pair(z, k23, ik13);
    return (eta / (1.0 - eta) + (1.0 - eta) / eta) * k23 + ik13;
}

struct BwHostTables {
    int nchi = 0, ny = 0;
    double lchi0 = 0, dl = 0;
    std::vector<float> g, cdf;
};

// Rows chi_i = chi_min 10^{i / per_decade}; the half-cumulative over
// eta = y^{3/2} / 2 by the trapezoid rule in y (the integrand vanishes at
// y = 0, where z grows without bound); H = twice the half integral.
inline BwHostTables bw_build_tables(double chi_min, double chi_max, int per_decade, int ny) {
    BwHostTables T;
    T.dl = std::log(10.0) / per_decade;
    T.lchi0 = std::log(chi_min);
    T.nchi = (int)std::floor((std::log(chi_max) - T.lchi0) / T.dl + 1e-9) + 1;
    T.ny = ny;
    T.g.resize(T.nchi);
    T.cdf.resize((size_t)T.nchi * ny);
    std::vector<double> v(ny), cum(ny);
    for (int i = 0; i < T.nchi; ++i) {
        const double chi = std::exp(T.lchi0 + i * T.dl);
        v[0] = 0.0;
        for (int j = 1; j < ny; ++j) {
            const double y = (double)j / (ny - 1);
            v[j] = bw_spectrum(0.5 * y * std::sqrt(y), chi) * 0.75 * std::sqrt(y);
        }
        cum[0] = 0.0;
        for (int j = 1; j < ny; ++j) cum[j] = cum[j - 1] + 0.5 * (v[j - 1] + v[j]) / (ny - 1);
        const double half = cum[ny - 1];
        T.g[i] = (float)(std::log(2.0 * half) + 8.0 / (3.0 * chi));
        for (int j = 0; j < ny; ++j) T.cdf[(size_t)i * ny + j] = (float)(cum[j] / half);
        T.cdf[(size_t)i * ny + ny - 1] = 1.0f;
    }
    return T;
}

}  // namespace lpic
