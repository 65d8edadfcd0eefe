// lpic_fp32.cuh -- FP32 particle path with an int64 fixed-point current.
//
// Particles: int32 linear cell + FP32 in-cell offsets (f in [0, 1)), FP32 u
// and w, stored leapfrog-style (x^{n+1/2}, u^n).  They are sorted by cell tile
// before the push; a work item is a tile, or a chunk of at most P particles of
// a crowded tile, and one thread block handles one item: it stages the tile's
// E/B halo in shared memory, pushes the item's particles (gather, Boris,
// straight path x^{n+1/2} -> x^{n+3/2}, Sec. 3.1) and accumulates their
// Esirkepov current in shared memory, which it flushes once to the global
// int64 J with integer atomics.  Integer sums do not depend on the order of
// the additions, so the result is bitwise deterministic.
//
// Shared-memory accumulation: rounds of 256 particles add into an int32 box
// with native 32-bit atomics.  In 2D the box is folded into an int64 box
// every R rounds (R from a host bound on one move's current per node, a
// fraction of S set by the Courant number and the shape); in 3D it is
// flushed to the global int64 current whenever a running bound of the moves
// deposited since the last flush says the next phase could overflow it.  The
// shift F keeps every particle's integer charge S <= 2^22.
//
// Exact charge conservation in integers.  The unit of charge is 2^-F.  A
// particle of charge s = 2^F q w carries the integer charge S = rint(s),
// split over its stencil level by level: qx(a) = rint(s Sx(a)) with the
// remainder S - sum qx at stencil index 1; qxy(a, b) = rint(qx(a) Sy(b)) with
// each row's remainder at b = 1 (so sum_b qxy(a, .) = qx(a)); in 3D
// q(a, b, c) = rint(qxy(a, b) Sz(c)) likewise.  Every particle's integer
// charge is then the same S at every position, and its marginals are exact
// integers that follow the 1D shapes to within a unit or two.  Weights are
// computed from the stored (cell, offset) pair with explicitly rounded
// arithmetic, so the charge at the end of one step's path is bit-identical
// to the charge at the start of the next step's path.  The Esirkepov fluxes
// (Sec. 3.1) are rounded directly and closed level by level (1D flow, 2D
// column sums, 3D nodes; see the deposit below), so that node by node
// sum_d J_d(i+1/2) - J_d(i-1/2) = -(Q1 - Q0) exactly.
#pragma once
#include "lpic_common.cuh"
#include "lpic_qed_tab.cuh"

// Checked build (compiled into a library of its own): every data-dependent
// shared-memory index of the gather and of the current box is tested against
// its box; an index outside it raises LPIC_ST_BOUNDS and the access is
// skipped.  Off in the product library.
#ifndef LPIC_CHECK
#define LPIC_CHECK 0
#endif

namespace lpic {

struct P32 {
    int* cell;
    float* off[3];
    float* u[3];
    float* w;
    int* id;
    const int* n;
};

// Nonlinear Compton emission (Sec. 3.4) of one emitting species into one
// photon species: the tables, the optical depths by particle id, the photon
// buffer (appended to), the step's counter word and the Philox key.
struct QedEmit {
    QedTab T;
    float* tau;            // [n_ids] optical depth by particle id
    long long n_ids;
    P32 ph;                // photon species (current buffer)
    int* ph_n;             // == ph.n, appended to
    int* ph_next_id;       // id of the next created photon
    long long ph_cap;
    float* ph_tau;         // optional: pair-creation depths of new photons, by photon id
    long long ph_n_ids;
    float dt;
    uint32_t k0, k1;
    const unsigned* step;  // fused kernel: device counter holding the counter word
};

// One particle's emission event in fields fld = (E, B) at its position, with
// momentum u (m c) and depth tau0 = tau[id] (read by the caller, which can
// issue that load early): chi = eps_ref gamma sqrt((E + beta x B)^2 -
// (beta . E)^2), tau[id] = tau0 - W(chi, gamma) dt, and when tau reaches zero a photon of energy
// k = xi gamma (xi from the spectrum's inverse cumulative at the first Philox
// word of counter (id, step, 0, 0)) is appended along u at (cell, off) with
// weight w, u recoils to u (1 - k/|u|) and tau restarts at -ln of the second
// word.  A photon that finds no room raises LPIC_ST_OVERFLOW and leaves the
// particle untouched with its spent depth (it emits at a later step).
// Returns true when u changed.
__device__ __forceinline__ bool qed_emit(const QedEmit& Q, uint32_t step, int dim, int id, float tau0,
                                         int cell, const float (&off)[3], float w, float (&u)[3],
                                         const float (&fld)[6], unsigned* st) {
    const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float gam = sqrtf(1.0f + u2);
    const float ig = 1.0f / gam;
    const float b0 = u[0] * ig, b1 = u[1] * ig, b2 = u[2] * ig;
    const float F0 = fld[0] + b1 * fld[5] - b2 * fld[4];
    const float F1 = fld[1] + b2 * fld[3] - b0 * fld[5];
    const float F2 = fld[2] + b0 * fld[4] - b1 * fld[3];
    const float be = b0 * fld[0] + b1 * fld[1] + b2 * fld[2];
    const float q2 = F0 * F0 + F1 * F1 + F2 * F2 - be * be;
    const float chi = Q.T.eps_ref * gam * sqrtf(fmaxf(q2, 0.0f));
    if (!(chi > 0.0f)) return false;
    const float t = tau0 - Q.T.pref * qed_h(Q.T, chi) * ig * Q.dt;
    if (t > 0.0f) { Q.tau[id] = t; return false; }
    // emission: xi from the first word, the new depth from the second
    const U4 o = philox4x32_10(U4{(uint32_t)id, step, 0u, 0u}, Q.k0, Q.k1);
    const float r1 = u01f(o.x);
    const float xi = qed_xi(Q.T, chi, r1);
    const float umag = sqrtf(u2);
    const float k = xi * gam;
    const int j = atomicAdd(Q.ph_n, 1);
    if ((long long)j >= Q.ph_cap) {
        set_status(st, LPIC_ST_OVERFLOW);
        Q.tau[id] = t;
        return false;
    }
    const float s = k / umag;
    Q.ph.cell[j] = cell;
    for (int d = 0; d < dim; ++d) Q.ph.off[d][j] = off[d];
#pragma unroll
    for (int c = 0; c < 3; ++c) Q.ph.u[c][j] = s * u[c];
    Q.ph.w[j] = w;
    const int pid = atomicAdd(Q.ph_next_id, 1);
    Q.ph.id[j] = pid;
    if (Q.ph_tau) {
        // the new photon's depth for pair creation: counter (id, 0, 3, 0)
        if (pid >= 0 && (long long)pid < Q.ph_n_ids) {
            const U4 q = philox4x32_10(U4{(uint32_t)pid, 0u, 3u, 0u}, Q.k0, Q.k1);
            Q.ph_tau[pid] = neg_log_u01(q.x);
        } else {
            set_status(st, LPIC_ST_OVERFLOW);
        }
    }
    const float keep = 1.0f - k / umag;
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] *= keep;
    Q.tau[id] = neg_log_u01(o.y);
    return true;
}

struct Tiles {
    int T[3];            // cells per tile
    int nt[3];           // tiles per dimension
    int m[3];            // margin (cells) the particles may have drifted since the sort
    const int* start;    // ntiles + 1 prefix offsets (after the sort)
    const int2* items;   // (tile, chunk) work items
    const int* nitems;   // device count of work items
    int P;               // particles per chunk
    unsigned bmax;       // 3D: bound of one move's current at any node, units of 256 (int32 box guard)
    int R;               // 2D: rounds of 256 moves between folds of the int32 current boxes
    FastDiv fT[3];       // division by T (tile keys of the next sort)
    FastDiv fG0, fG1, fF;  // division by the field box rows, planes, size
    FastDiv fH0, fH1, fJ;  // and by those of the current box
    int* next_count;     // if set: histogram of the new tile keys for the next sort
    int* esc;            // indices of particles beyond the tile's margin ...
    int* nesc;           // ... and their count (pushed by k_gpd32_escape)
};

template <int ORDER, class W>
__device__ __forceinline__ void place32(float (&S)[ORDER + 2], const W& w, int off) {
#pragma unroll
    for (int a = 0; a < ORDER + 2; ++a) {
        const float lo = (a <= ORDER) ? w.w[a < ORDER + 1 ? a : 0] : 0.0f;
        const float hi = (a >= 1) ? w.w[a >= 1 ? a - 1 : 0] : 0.0f;
        S[a] = off ? hi : lo;
    }
}

// Adds a lane's value to the int32 current box with a shared-memory
// reduction.  SKIP_ZERO: predicated on a nonzero value, without a branch (2D:
// slowly moving particles leave most window values at zero; 3D: most values
// are nonzero).
template <bool SKIP_ZERO>
struct Acc32 {
    int* sJ;
    int lim = 0;                 // checked build: words in the box
    unsigned* st = nullptr;
    __device__ __forceinline__ void operator()(int idx, int v) const {
#if LPIC_CHECK
        if ((unsigned)idx >= (unsigned)lim) { set_status(st, LPIC_ST_BOUNDS); return; }
#endif
        if constexpr (SKIP_ZERO) {
            const unsigned a = (unsigned)__cvta_generic_to_shared(sJ + idx);
            asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %1, 0;\n\t@q red.shared.add.s32 [%0], %1;\n\t}"
                         :: "r"(a), "r"(v));
        } else {
            atomicAdd(sJ + idx, v);
        }
    }
};

// Hierarchical integer charge of one stencil placed in a window of WN nodes
// per dimension (weights zero outside the stencil; o = stencil offset in the
// window, the remainder of each level goes to stencil index 1).
template <int WN>
__device__ inline void charge_levels_1d(float s, int S, const float (&Sx)[WN], int o, int (&qx)[WN]) {
    int sum = 0;
#pragma unroll
    for (int a = 0; a < WN; ++a) { qx[a] = rint22_mul(s, Sx[a]); sum += qx[a]; }
#pragma unroll
    for (int a = 0; a < WN; ++a) qx[a] += (a == o + 1) ? S - sum : 0;
}

template <int WN>
__device__ inline void charge_levels_2d(const int (&qx)[WN], const float (&Sy)[WN], int o,
                                        int (&qxy)[WN][WN]) {
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        int sum = 0;
        const float fa = (float)qx[a];
#pragma unroll
        for (int b = 0; b < WN; ++b) { qxy[a][b] = rint22_mul(fa, Sy[b]); sum += qxy[a][b]; }
#pragma unroll
        for (int b = 0; b < WN; ++b) qxy[a][b] += (b == o + 1) ? qx[a] - sum : 0;
    }
}

// ----------------------------------------------------------- deposit (Sec. 3.1)
// Integer Esirkepov current of one move, written directly as fluxes.
//
// Window of WN nodes per dimension (WN = ORDER + 1: both stencils start at
// the same node; WN = ORDER + 2: they differ by one in some dimension), the
// start / end stencils at offsets o0 / o1 in it.  With A = (S0 + S1) / 2,
// DS = S1 - S0 and C(a) = sum_{a' <= a} DS(a') per dimension, the exact
// Esirkepov fluxes are J_x(a+1/2, b, c) = -s C_x(a) (A_y A_z + DS_y DS_z / 12)
// and cyclically (2D: J_x = -s C_x(a) A_y(b), J_y likewise).  The integer
// construction, level by level:
//   1D: the x flow Mx(a+1/2) = -sum_{a' <= a} (qx1 - qx0)(a').
//   2D: X(a+1/2, b) = rint(-s C_x(a) A_y(b)) except on the closure column
//       b = cy, fixed so that sum_b X(a+1/2, .) = Mx(a+1/2); Y(a, b+1/2) is
//       the running sum over b of -(dqxy + X(a+1/2) - X(a-1/2)), which closes
//       to zero at the window's end because every row sum of X is the 1D flow.
//       (In 2D X and Y are the currents J_x and J_y.)
//   3D: J_x(a+1/2, b, c) = rint(-s C_x(a) K_x(b, c)) except on c = cz, fixed
//       so that sum_c J_x = X(a+1/2, b); J_y likewise with sum_c J_y =
//       Y(a, b+1/2); J_z(a, b, c+1/2) is the running sum over c of
//       -(dQ + dJ_x/dx + dJ_y/dy), which closes at both window ends.
// The closure column of each dimension is the stencil's last node when both
// stencils start at the same node in that dimension, else the window's last
// node, and every rounded value off the stencils is rint(0) = 0: a
// same-stencil move gives identical integers in both window sizes.  Node by
// node, sum_d J_d(+1/2) - J_d(-1/2) = -(Q1 - Q0) exactly.

constexpr float kRound = 12582912.0f;      // 1.5 * 2^23
// nearest integer of a * b (|a b| < 2^22)
__device__ __forceinline__ int irnd_mul(float a, float b) { return __float_as_int(__fmaf_rn(a, b, kRound)) - 0x4B400000; }

// One level of the hierarchical charge: out[k] = rint(scale S[k]) except at
// the stencil's index 1 (window index o + 1), which takes total - the sum of
// the others (the same integers as charge_levels_1d / _2d).
template <int WN, bool FIXED>
__device__ __forceinline__ void leveli(float scale, int total, const float (&S)[WN], int o, int (&out)[WN]) {
    if constexpr (FIXED) {
        int sum = 0;
#pragma unroll
        for (int k = 0; k < WN; ++k)
            if (k != 1) { out[k] = irnd_mul(scale, S[k]); sum += out[k]; }
        out[1] = total - sum;
    } else {
        int sum = 0;
#pragma unroll
        for (int k = 0; k < WN; ++k) { out[k] = irnd_mul(scale, S[k]); sum += out[k]; }
#pragma unroll
        for (int k = 0; k < WN; ++k)
            if (k == o + 1) out[k] += total - sum;
    }
}

// 2D.  SAME: WN = ORDER + 1 and all offsets 0 (compile-time closures).
// Node (a, b) of component c lives at c * jsz + n0 + b * H0 + a of the box.
// Evaluated column by column in x, so that only the previous column's J_x
// crosses columns.
template <int ORDER, int WN, bool SAME, class Acc>
__device__ __forceinline__ void deposit2d_core(const Acc& acc, int jsz, int H0, int n0, int o0x, int o1x, int o0y,
                                      int o1y, const float (&S0x)[WN], const float (&S1x)[WN],
                                      const float (&S0y)[WN], const float (&S1y)[WN], float s, float vz) {
    constexpr int L = WN - 1;
    const int S = rint22(s);
    int qx0[WN], qx1[WN];
    leveli<WN, SAME>(s, S, S0x, o0x, qx0);
    leveli<WN, SAME>(s, S, S1x, o1x, qx1);
    const int cy = SAME ? ORDER : ((o0y == o1y) ? o0y + ORDER : L);
    const float svz = s * vz, svz12 = svz * (1.0f / 12.0f);
    int jxp[WN];                       // J_x(a - 1/2, b)
#pragma unroll
    for (int b = 0; b < WN; ++b) jxp[b] = 0;
    float Cx = 0.0f;
    int Mx = 0;
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        // J_x(a+1/2, b) with the closure column cy
        int jx[WN];
        if (a < L) {
            Cx = Cx + (S1x[a] - S0x[a]);
            Mx += qx0[a] - qx1[a];
            const float sc = -s * Cx;
            int row = 0;
#pragma unroll
            for (int b = 0; b < WN; ++b) {
                jx[b] = (b == cy) ? 0 : irnd_mul(sc, 0.5f * (S0y[b] + S1y[b]));
                row += jx[b];
            }
#pragma unroll
            for (int b = 0; b < WN; ++b)
                if (b == cy) jx[b] = Mx - row;
#pragma unroll
            for (int b = 0; b < WN; ++b) acc(n0 + b * H0 + a, jx[b]);
        } else {
#pragma unroll
            for (int b = 0; b < WN; ++b) jx[b] = 0;
        }
        // J_y(a, b+1/2), b < L: running sums of -(dq + dJ_x)
        int r0[WN], r1[WN];
        leveli<WN, SAME>((float)qx0[a], qx0[a], S0y, o0y, r0);
        leveli<WN, SAME>((float)qx1[a], qx1[a], S1y, o1y, r1);
        int run = 0;
#pragma unroll
        for (int b = 0; b < L; ++b) {
            run -= (r1[b] - r0[b]) + jx[b] - jxp[b];
            acc(jsz + n0 + b * H0 + a, run);
        }
        // J_z: s v_z W_z, W_z = A_x A_y + DS_x DS_y / 12 (no closure in 2D; the
        // DS term is added to the rounding constant first, then the A term)
        const float pa = svz * (0.5f * (S0x[a] + S1x[a])), qa = svz12 * (S1x[a] - S0x[a]);
#pragma unroll
        for (int b = 0; b < WN; ++b) {
            const float t = __fmaf_rn(qa, S1y[b] - S0y[b], kRound);
            acc(2 * jsz + n0 + b * H0 + a,
                __float_as_int(__fmaf_rn(pa, 0.5f * (S0y[b] + S1y[b]), t)) - 0x4B400000);
        }
#pragma unroll
        for (int b = 0; b < WN; ++b) jxp[b] = jx[b];
    }
}

// From the start and end stencils' weights: SAME (both start at the same
// node in both dimensions) uses the stencil-sized window, else the window of
// ORDER + 2 nodes.
template <int ORDER, bool SAME, class Acc>
__device__ __forceinline__ void deposit2d_w(const Acc& acc, int jsz, int H0, const NodeW<ORDER>& ax, const NodeW<ORDER>& ay,
                                   const NodeW<ORDER>& bx, const NodeW<ORDER>& by, float s, float vz) {
    if constexpr (SAME) {
        constexpr int WN = ORDER + 1;
        float S0x[WN], S1x[WN], S0y[WN], S1y[WN];
#pragma unroll
        for (int a = 0; a < WN; ++a) { S0x[a] = ax.w[a]; S1x[a] = bx.w[a]; S0y[a] = ay.w[a]; S1y[a] = by.w[a]; }
        deposit2d_core<ORDER, WN, true>(acc, jsz, H0, (ay.base + 2) * H0 + ax.base + 2, 0, 0, 0, 0, S0x, S1x,
                                        S0y, S1y, s, vz);
    } else {
        constexpr int WN = ORDER + 2;
        const int basex = min(ax.base, bx.base), basey = min(ay.base, by.base);
        const int o0x = ax.base - basex, o1x = bx.base - basex;
        const int o0y = ay.base - basey, o1y = by.base - basey;
        float S0x[WN], S1x[WN], S0y[WN], S1y[WN];
        place32<ORDER>(S0x, ax, o0x); place32<ORDER>(S1x, bx, o1x);
        place32<ORDER>(S0y, ay, o0y); place32<ORDER>(S1y, by, o1y);
        deposit2d_core<ORDER, WN, false>(acc, jsz, H0, (basey + 2) * H0 + basex + 2, o0x, o1x, o0y, o1y, S0x,
                                         S1x, S0y, S1y, s, vz);
    }
}

// General case from (cell, offset) pairs: the window of ORDER + 2 nodes.
template <int ORDER, class Acc>
__device__ __forceinline__ void deposit2d(const Acc& acc, int jsz, int H0, const int* lc, const float* f,
                                 const int* ce, const float* fe, float s, float vz) {
    deposit2d_w<ORDER, false>(acc, jsz, H0, NodeW<ORDER>(lc[0], f[0]), NodeW<ORDER>(lc[1], f[1]),
                              NodeW<ORDER>(ce[0], fe[0]), NodeW<ORDER>(ce[1], fe[1]), s, vz);
}

// Both stencils start at the same node in both dimensions (the particle kept
// its nearest node): the window is the stencil itself, ORDER + 1 nodes.
template <int ORDER, class Acc>
__device__ __forceinline__ void deposit2d_same(const Acc& acc, int jsz, int H0, const int* lc, const float* f,
                                      const int* ce, const float* fe, float s, float vz) {
    deposit2d_w<ORDER, true>(acc, jsz, H0, NodeW<ORDER>(lc[0], f[0]), NodeW<ORDER>(lc[1], f[1]),
                             NodeW<ORDER>(ce[0], fe[0]), NodeW<ORDER>(ce[1], fe[1]), s, vz);
}

// 3D.  Node (a, b, c) of component k lives at k * jsz + n0 + (c H1 + b) H0 + a.
// Evaluated slab by slab in x and column by column in y inside a slab, so
// that only the previous slab's J_x, the previous column's J_y and the
// previous slab's X cross.  SAME: WN = ORDER + 1, all offsets 0; then the 3D
// charge level is needed only off the stencil's index 1 (J_z runs forward
// below it and backward above it).
template <int ORDER, int WN, bool SAME, class Acc>
__device__ __forceinline__ void deposit3d_core(const Acc& acc, int jsz, int H0, int H1, int n0,
                                      int ox0, int ox1, int oy0, int oy1, int oz0, int oz1,
                                      const float (&S0x)[WN], const float (&S1x)[WN],
                                      const float (&S0y)[WN], const float (&S1y)[WN],
                                      const float (&S0z)[WN], const float (&S1z)[WN], float s) {
    constexpr int L = WN - 1;
    const int P = H0 * H1;
    const int S = rint22(s);
    int qx0[WN], qx1[WN];
    leveli<WN, SAME>(s, S, S0x, ox0, qx0);
    leveli<WN, SAME>(s, S, S1x, ox1, qx1);
    const int cy = SAME ? ORDER : ((oy0 == oy1) ? oy0 + ORDER : L);
    const int cz = SAME ? ORDER : ((oz0 == oz1) ? oz0 + ORDER : L);
    int Xp[WN];                        // X(a - 1/2, b)
    // SAME: J_x(a - 1/2, b, c) kept for the next slab's J_z; otherwise each
    // J_x column's running sum over c is added to the next slab's J_z at once
    // (fewer live registers for the larger window)
    int jxp[SAME ? WN : 1][SAME ? WN : 1];
#pragma unroll
    for (int b = 0; b < WN; ++b) {
        Xp[b] = 0;
        if constexpr (SAME) {
#pragma unroll
            for (int c = 0; c < WN; ++c) jxp[b][c] = 0;
        }
    }
    float Cx = 0.0f;
    int Mx = 0;
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        // 2D charges of slab a, X(a+1/2, .) with the closure column cy
        int r0[WN], r1[WN];
        leveli<WN, SAME>((float)qx0[a], qx0[a], S0y, oy0, r0);
        leveli<WN, SAME>((float)qx1[a], qx1[a], S1y, oy1, r1);
        int X[WN];
        float sCx = 0.0f;
        if (a < L) {
            Cx = Cx + (S1x[a] - S0x[a]);
            Mx += qx0[a] - qx1[a];
            sCx = -s * Cx;
            int row = 0;
#pragma unroll
            for (int b = 0; b < WN; ++b) {
                X[b] = (b == cy) ? 0 : irnd_mul(sCx, 0.5f * (S0y[b] + S1y[b]));
                row += X[b];
            }
#pragma unroll
            for (int b = 0; b < WN; ++b)
                if (b == cy) X[b] = Mx - row;
        } else {
#pragma unroll
            for (int b = 0; b < WN; ++b) X[b] = 0;
        }
        const float ax = 0.5f * (S0x[a] + S1x[a]), dx12 = (S1x[a] - S0x[a]) * (1.0f / 12.0f);
        int Y = 0;                     // Y(a, b+1/2), running over b
        float Cy = 0.0f;
        int jyp[WN];                   // J_y(a, b - 1/2, c)
#pragma unroll
        for (int c = 0; c < WN; ++c) jyp[c] = 0;
#pragma unroll
        for (int b = 0; b < WN; ++b) {
            const int nb = n0 + b * H0 + a;
            // J_x(a+1/2, b, c) with the closure row cz: sum_c = X(a+1/2, b)
            int jx[WN];
            if (a < L) {
                const float ay = 0.5f * (S0y[b] + S1y[b]), dy12 = (S1y[b] - S0y[b]) * (1.0f / 12.0f);
                int col = 0;
#pragma unroll
                for (int c = 0; c < WN; ++c) {
                    jx[c] = (c == cz) ? 0 : irnd_mul(sCx, __fmaf_rn(ay, 0.5f * (S0z[c] + S1z[c]), dy12 * (S1z[c] - S0z[c])));
                    col += jx[c];
                }
#pragma unroll
                for (int c = 0; c < WN; ++c) {
                    if (c == cz) jx[c] = X[b] - col;
                    acc(nb + c * P, jx[c]);
                }
                if constexpr (!SAME) {
                    // -J_x(a+1/2) enters D of slab a + 1: its running sum over c,
                    // with the sign of J_z = -sum D, goes to J_z(a + 1, b, .)
                    int px = 0;
#pragma unroll
                    for (int c = 0; c < L; ++c) {
                        px += jx[c];
                        acc(2 * jsz + nb + 1 + c * P, px);
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < WN; ++c) jx[c] = 0;
            }
            // J_y(a, b+1/2, c) with the closure row cz: sum_c = Y(a, b+1/2)
            int jy[WN];
            if (b < L) {
                Y -= (r1[b] - r0[b]) + X[b] - Xp[b];
                Cy = Cy + (S1y[b] - S0y[b]);
                const float sCy = -s * Cy;
                int col = 0;
#pragma unroll
                for (int c = 0; c < WN; ++c) {
                    jy[c] = (c == cz) ? 0 : irnd_mul(sCy, __fmaf_rn(ax, 0.5f * (S0z[c] + S1z[c]), dx12 * (S1z[c] - S0z[c])));
                    col += jy[c];
                }
#pragma unroll
                for (int c = 0; c < WN; ++c) {
                    if (c == cz) jy[c] = Y - col;
                    acc(jsz + nb + c * P, jy[c]);
                }
            } else {
#pragma unroll
                for (int c = 0; c < WN; ++c) jy[c] = 0;
            }
            // J_z(a, b, c+1/2): D(c) = dQ + J_x(a+1/2) - J_x(a-1/2) + J_y(b+1/2) - J_y(b-1/2)
            if constexpr (SAME) {
                int fw = 0;
#pragma unroll
                for (int c = 0; c < 1; ++c) {
                    const int dq = irnd_mul((float)r1[b], S1z[c]) - irnd_mul((float)r0[b], S0z[c]);
                    fw -= dq + jx[c] - jxp[b][c] + jy[c] - jyp[c];
                    acc(2 * jsz + nb + c * P, fw);
                }
                int bw = 0;
#pragma unroll
                for (int c = L; c >= 2; --c) {
                    const int dq = irnd_mul((float)r1[b], S1z[c]) - irnd_mul((float)r0[b], S0z[c]);
                    bw += dq + jx[c] - jxp[b][c] + jy[c] - jyp[c];
                    acc(2 * jsz + nb + (c - 1) * P, bw);
                }
            } else {
                int z0[WN], z1[WN];
                leveli<WN, false>((float)r0[b], r0[b], S0z, oz0, z0);
                leveli<WN, false>((float)r1[b], r1[b], S1z, oz1, z1);
                int fw = 0;
#pragma unroll
                for (int c = 0; c < L; ++c) {
                    fw -= (z1[c] - z0[c]) + jx[c] + jy[c] - jyp[c];
                    acc(2 * jsz + nb + c * P, fw);
                }
            }
#pragma unroll
            for (int c = 0; c < WN; ++c) {
                if constexpr (SAME) jxp[b][c] = jx[c];
                jyp[c] = jy[c];
            }
        }
#pragma unroll
        for (int b = 0; b < WN; ++b) Xp[b] = X[b];
    }
}

// General case: the window of ORDER + 2 nodes per dimension holds both stencils.
template <int ORDER, class Acc>
__device__ __forceinline__ void deposit3d(const Acc& acc, int jsz, int H0, int H1, const int* lc,
                                 const float* f, const int* ce, const float* fe, float s) {
    constexpr int WN = ORDER + 2;
    const NodeW<ORDER> a0(lc[0], f[0]), a1(lc[1], f[1]), a2(lc[2], f[2]);
    const NodeW<ORDER> b0(ce[0], fe[0]), b1(ce[1], fe[1]), b2(ce[2], fe[2]);
    const int bs0 = min(a0.base, b0.base), bs1 = min(a1.base, b1.base), bs2 = min(a2.base, b2.base);
    float S0x[WN], S1x[WN], S0y[WN], S1y[WN], S0z[WN], S1z[WN];
    place32<ORDER>(S0x, a0, a0.base - bs0); place32<ORDER>(S1x, b0, b0.base - bs0);
    place32<ORDER>(S0y, a1, a1.base - bs1); place32<ORDER>(S1y, b1, b1.base - bs1);
    place32<ORDER>(S0z, a2, a2.base - bs2); place32<ORDER>(S1z, b2, b2.base - bs2);
    deposit3d_core<ORDER, WN, false>(acc, jsz, H0, H1, ((bs2 + 2) * H1 + bs1 + 2) * H0 + bs0 + 2,
                                     a0.base - bs0, b0.base - bs0, a1.base - bs1, b1.base - bs1,
                                     a2.base - bs2, b2.base - bs2, S0x, S1x, S0y, S1y, S0z, S1z, s);
}

// Both stencils start at the same node in every dimension: the window is the
// stencil itself, ORDER + 1 nodes per dimension (from the stencils' weights).
template <int ORDER, class Acc>
__device__ __forceinline__ void deposit3d_w(const Acc& acc, int jsz, int H0, int H1, const NodeW<ORDER>& a0,
                                   const NodeW<ORDER>& a1, const NodeW<ORDER>& a2, const NodeW<ORDER>& b0,
                                   const NodeW<ORDER>& b1, const NodeW<ORDER>& b2, float s) {
    constexpr int WN = ORDER + 1;
    float S0x[WN], S1x[WN], S0y[WN], S1y[WN], S0z[WN], S1z[WN];
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        S0x[a] = a0.w[a]; S1x[a] = b0.w[a]; S0y[a] = a1.w[a]; S1y[a] = b1.w[a];
        S0z[a] = a2.w[a]; S1z[a] = b2.w[a];
    }
    deposit3d_core<ORDER, WN, true>(acc, jsz, H0, H1, ((a2.base + 2) * H1 + a1.base + 2) * H0 + a0.base + 2,
                                    0, 0, 0, 0, 0, 0, S0x, S1x, S0y, S1y, S0z, S1z, s);
}

template <int ORDER, class Acc>
__device__ __forceinline__ void deposit3d_same(const Acc& acc, int jsz, int H0, int H1, const int* lc,
                                      const float* f, const int* ce, const float* fe, float s) {
    deposit3d_w<ORDER>(acc, jsz, H0, H1, NodeW<ORDER>(lc[0], f[0]), NodeW<ORDER>(lc[1], f[1]),
                       NodeW<ORDER>(lc[2], f[2]), NodeW<ORDER>(ce[0], fe[0]), NodeW<ORDER>(ce[1], fe[1]),
                       NodeW<ORDER>(ce[2], fe[2]), s);
}

// Whether the start and end stencils of a move begin at the same node in
// every dimension (then the stencil-sized window holds the whole deposit).
template <int DIM, int ORDER>
__device__ __forceinline__ bool same_stencils(const int* lc, const float* f, const int* ce, const float* fe) {
    bool same = true;
#pragma unroll
    for (int d = 0; d < DIM; ++d) same &= NodeW<ORDER>(lc[d], f[d]).base == NodeW<ORDER>(ce[d], fe[d]).base;
    return same;
}

// Integer charge of one particle (the Q of the deposit: same levels, same
// arithmetic) added to rho_int.
template <int DIM, int ORDER>
__device__ inline void charge_int(unsigned long long* rho, const Geo& g, const int* gc,
                                  const float* f, float s) {
    constexpr int WN = ORDER + 2;
    const NodeW<ORDER> wx(gc[0], f[0]), wy(gc[1], f[1]), wz(DIM == 3 ? gc[2] : 0, DIM == 3 ? f[2] : 0.0f);
    float Sx[WN], Sy[WN], Sz[WN];
    place32<ORDER>(Sx, wx, 0); place32<ORDER>(Sy, wy, 0); place32<ORDER>(Sz, wz, 0);
    const int sint = rint22(s);
    int qx[WN], qxy[WN][WN];
    charge_levels_1d<WN>(s, sint, Sx, 0, qx);
    charge_levels_2d<WN>(qx, Sy, 0, qxy);
#pragma unroll
    for (int a = 0; a <= ORDER; ++a)
#pragma unroll
        for (int b = 0; b <= ORDER; ++b) {
            if (DIM == 2) {
                const long long m = fidx(g, wx.base + a, wy.base + b, 0);
                if (m >= 0 && qxy[a][b] != 0)
                    atomicAdd(rho + m, static_cast<unsigned long long>(static_cast<long long>(qxy[a][b])));
                continue;
            }
            int q[WN], sum = 0;
            const float fab = (float)qxy[a][b];
#pragma unroll
            for (int c = 0; c < WN; ++c) { q[c] = rint22_mul(fab, Sz[c]); sum += q[c]; }
            q[1] += qxy[a][b] - sum;
#pragma unroll
            for (int c = 0; c <= ORDER; ++c) {
                const long long m = fidx(g, wx.base + a, wy.base + b, wz.base + c);
                if (m >= 0 && q[c] != 0)
                    atomicAdd(rho + m, static_cast<unsigned long long>(static_cast<long long>(q[c])));
            }
        }
}

// ----------------------------------------------------------- gather
// Interpolates the six Yee components at the particle: staggering E_x (h,n,n),
// E_y (n,h,n), E_z (n,n,h), B_x (n,h,h), B_y (h,n,h), B_z (h,h,n) with h the
// half-node and n the node weights of each dimension.  The sum is separable:
// rows along x first, then along y, then z, with explicit roundings so that
// the tile kernel (fields staged in shared memory) and the global-memory path
// for escaped particles give identical bits.  ld(comp, x, y, z) returns the
// component at node (x, y, z) of the particle's local frame (z = 0 in 2D).
template <int DIM, int ORDER, class Load>
__device__ __forceinline__ void gather32(const Load& ld, const NodeW<ORDER>& nx_, const NodeW<ORDER>& ny_,
                                         const NodeW<ORDER>& nz_, const HalfW<ORDER>& hx_,
                                         const HalfW<ORDER>& hy_, const HalfW<ORDER>& hz_, float (&fld)[6]) {
#pragma unroll
    for (int comp = 0; comp < 6; ++comp) {
        const bool hx = (comp == 0 || comp == 4 || comp == 5);
        const bool hy = (comp == 1 || comp == 3 || comp == 5);
        const bool hz = (comp == 2 || comp == 3 || comp == 4);
        const int bx = hx ? hx_.base : nx_.base, by = hy ? hy_.base : ny_.base;
        const int bz = (DIM == 3) ? (hz ? hz_.base : nz_.base) : 0;
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < (DIM == 3 ? ORDER + 1 : 1); ++c) {
            float accb = 0.0f;
#pragma unroll
            for (int b = 0; b <= ORDER; ++b) {
                float r = 0.0f;
#pragma unroll
                for (int a = 0; a <= ORDER; ++a) {
                    const float wx = hx ? hx_.w[a] : nx_.w[a];
                    const float v = ld(comp, bx + a, by + b, DIM == 3 ? bz + c : 0);
                    r = (a == 0) ? __fmul_rn(v, wx) : __fmaf_rn(v, wx, r);
                }
                const float wy = hy ? hy_.w[b] : ny_.w[b];
                accb = (b == 0) ? __fmul_rn(r, wy) : __fmaf_rn(r, wy, accb);
            }
            if (DIM == 3) {
                const float wz = hz ? hz_.w[c] : nz_.w[c];
                acc = (c == 0) ? __fmul_rn(accb, wz) : __fmaf_rn(accb, wz, acc);
            } else {
                acc = accb;
            }
        }
        fld[comp] = acc;
    }
}

// Field components staged in shared memory: box of G0 x G1 (x G2) nodes per
// component from local node -1, local node (x, y, z) at ((z+1) G1 + y+1) G0 + x+1
// (2D: (y+1) G0 + x+1).
template <int DIM>
struct LoadShared {
    const float* sF;
    int fsz, G0, G1;
    unsigned* st = nullptr;      // checked build: status word
    __device__ inline float operator()(int comp, int x, int y, int z) const {
        const int idx = comp * fsz + ((DIM == 3 ? z + 1 : 0) * G1 + (y + 1)) * G0 + (x + 1);
#if LPIC_CHECK
        if ((unsigned)idx >= (unsigned)(6 * fsz)) { set_status(st, LPIC_ST_BOUNDS); return 0.0f; }
#endif
        return sF[idx];
    }
};

// Field components read from global memory around a particle whose cell is
// gc, local frame with the particle's cell at 2; nodes outside the grid
// (absorbing x) read 0 and raise the flag.
template <int DIM>
struct LoadGlobal {
    const Geo* g;
    const float* F[6];
    const double* F64[6];     // FP64 master fields, rounded to float (when set)
    int gc[3];
    bool* outside;
    __device__ inline float operator()(int comp, int x, int y, int z) const {
        const long long m = fidx(*g, gc[0] + x - 2, gc[1] + y - 2, DIM == 3 ? gc[2] + z - 2 : 0);
        if (m < 0) { *outside = true; return 0.0f; }
        return F64[0] ? (float)F64[comp][m] : F[comp][m];
    }
};

// ----------------------------------------------------------- the tile kernel
// Blocks per SM the register allocation targets (2D: 64 registers, 4 blocks
// of 256; 3D: 80 registers, 3 blocks, which the shared memory of an 8x8x4
// tile also allows).
#ifndef LPIC_GPD2D_MINB
#define LPIC_GPD2D_MINB 4
#endif
#ifndef LPIC_GPD3D_MINB
#define LPIC_GPD3D_MINB 3
#endif

// Shared memory of one work item, in 4-byte words, each part 16-byte aligned:
//   fields     6 boxes of G0 x G1 (x G2) floats, G = T + 2m + 3: local nodes
//              -1 .. T + 2m + 1, which hold the gather stencil of any particle
//              in local cells [0, T + 2m) for either shape order;
//   current    3 boxes of H0 x H1 (x H2) int32, H = T + 2m + 5: local nodes
//              -2 .. T + 2m + 2, which hold both stencils of any move;
//   current64  (2D) the same boxes in int64, into which the int32 boxes are
//              folded when they could overflow (in 3D they are flushed to the
//              global current instead: its boxes are large and shared memory
//              bounds the blocks per SM);
//   particles  two round buffers of DIM + 6 arrays (cell, offsets, momenta,
//              weight, and the id for the form with emission) of kRoundWords
//              words: the next round's particles are copied in asynchronously
//              while the current round runs;
//   ring       (3D) moves whose two stencils start at different nodes, deposited
//              256 at a time so that every warp runs one form of the deposit;
//   counters   the bound of the current accumulated in the int32 boxes
//              (three, by round modulo 3) and the ring's fill count.
constexpr int kGpdThreads = 256;
constexpr int kRoundWords = kGpdThreads + 8;
constexpr int kRing = 2 * kGpdThreads;
constexpr int kCntWords = 8;
enum { kCntBound = 0, kCntRing = 3 };

struct TileSmem {
    int G[3], H[3], fsz, jsz, off_r, off_64, off_p, off_ring, off_cnt, words;
};

__host__ __device__ inline int up4(int w) { return (w + 3) & ~3; }

__host__ __device__ inline TileSmem tile_smem(int dim, const int* T, const int* m) {
    TileSmem s{};
    s.fsz = 1;
    s.jsz = 1;
    for (int d = 0; d < 3; ++d) {
        s.G[d] = d < dim ? T[d] + 2 * m[d] + 3 : 1;
        s.H[d] = d < dim ? T[d] + 2 * m[d] + 5 : 1;
        s.fsz *= s.G[d];
        s.jsz *= s.H[d];
    }
    s.off_r = up4(6 * s.fsz);
    s.off_64 = s.off_r + up4(3 * s.jsz);
    s.off_p = s.off_64 + (dim == 2 ? 2 * up4(3 * s.jsz) : 0);
    s.off_ring = s.off_p + 2 * (dim + 6) * kRoundWords;
    s.off_cnt = s.off_ring + (dim == 3 ? (dim + 5) * kRing : 0);
    s.words = s.off_cnt + kCntWords;
    return s;
}

// Overflow guard of the int32 current boxes.  One move adds at most
// S |d|max (k^2 + 1/12) + 1024 to any node in 3D (S the particle's integer
// charge, |d|max its largest displacement in cells, k the largest 1D shape
// weight; the slack covers roundings and closures), and in 2D at most
// S max(|d|max k, |v_z| (k^2 + 1/12)) + 1024.  3D: the kernel sums these
// bounds (in units of 256) over the moves deposited since the boxes were
// last flushed, and flushes before a phase whose worst case could take the
// sum past 2^31 - 1 (a thermal plasma never needs to within a work item).
// 2D: the boxes are folded into the int64 boxes every R rounds, R from the
// largest move (host side).
constexpr unsigned kBoundUnit = 256;
constexpr unsigned kBoundLimit = 0x7fffffffu / kBoundUnit;

__device__ inline void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ inline void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// A move in DIM + 5 words at stride `stride`: word 0 packs the start cell in
// the box's local frame (8 bits per dimension) with the end cell's carries
// (2 bits each, from bit 24) and bit 30 set when both stencils start at the
// same node in every dimension (-1: no move); then the start offsets, the
// end offsets, the charge s and (2D) v_z.
template <int DIM>
struct Move {
    int lc[3], ce[3];
    float f[3], fe[3], s, vz;
    bool same;
    __device__ __forceinline__ static bool valid(const int* w) { return w[0] >= 0; }
    __device__ __forceinline__ void write(int* w, int stride) const {
        int carries = 0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) carries |= (ce[d] - lc[d] + 1) << (2 * d);
        int h = lc[0] | (lc[1] << 8) | (carries << 24) | (same ? (1 << 30) : 0);
        if (DIM == 3) h |= lc[2] << 16;
        w[0] = h;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            w[(1 + d) * stride] = __float_as_int(f[d]);
            w[(1 + DIM + d) * stride] = __float_as_int(fe[d]);
        }
        w[(1 + 2 * DIM) * stride] = __float_as_int(s);
        if (DIM == 2) w[(2 + 2 * DIM) * stride] = __float_as_int(vz);
    }
    __device__ __forceinline__ void read(const int* w, int stride) {
        const int h = w[0];
        lc[0] = h & 0xff; lc[1] = (h >> 8) & 0xff; lc[2] = DIM == 3 ? (h >> 16) & 0xff : 0;
        same = (h >> 30) & 1;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ce[d] = d < DIM ? lc[d] + ((h >> (24 + 2 * d)) & 3) - 1 : 0;
            f[d] = d < DIM ? __int_as_float(w[(1 + d) * stride]) : 0.0f;
            fe[d] = d < DIM ? __int_as_float(w[(1 + DIM + d) * stride]) : 0.0f;
        }
        s = __int_as_float(w[(1 + 2 * DIM) * stride]);
        vz = DIM == 2 ? __int_as_float(w[(2 + 2 * DIM) * stride]) : 0.0f;
    }
    // bound of this move's current at any node (units of kBoundUnit)
    template <int ORDER>
    __device__ __forceinline__ unsigned bound() const {
        constexpr float k = ORDER == 2 ? 0.75f : 1.0f;
        constexpr float k2 = k * k + 1.0f / 12.0f;
        float dm = 0.0f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) dm = fmaxf(dm, fabsf((float)(ce[d] - lc[d]) + (fe[d] - f[d])));
        const float b = DIM == 3 ? dm * k2 : fmaxf(dm * k, fabsf(vz) * k2);
        return __float2uint_ru(b * fabsf(s) * (1.0f / kBoundUnit)) + 5u;
    }
};

// Everything the fused kernel needs for one species of one grid.
struct GpdArgs {
    Geo g;
    Ptr3<const float> E, B;
    Ptr3<const double> E64, B64;   // FP64 master fields (used when f64 is set)
    int f64;
    Ptr3<unsigned long long> J;
    P32 p;
    Tiles t;
    CellDecode dec;
    float k, sq, dth0, dth1, dth2;
    unsigned* st;
    float* fields;       // unfused stages: per-particle E_x..B_z, [6][fcap]
    long long fcap;
    int qed;             // emission inside the push (kGpdQed form and the escape kernel)
    QedEmit q;
};

// Forms of the tile kernel: the fused gather/push/deposit, and the two
// stages of the unfused path (the gather alone, writing each particle's
// fields; the push and deposit with fields read back).  Between them the
// caller may change the fields (an external field, a diagnostic).
enum { kGpdFused = 0, kGpdGather = 1, kGpdFieldsIn = 2, kGpdQed = 3 };

// One work item (a tile, or a chunk of a crowded tile) of one species.
template <int DIM, int ORDER, int MODE = kGpdFused>
__device__ __forceinline__ void gpd_item(const GpdArgs& A, int item_index, float4* smem4) {
    const Geo& g = A.g;
    const Ptr3<unsigned long long>& J = A.J;
    const P32& p = A.p;
    const Tiles& t = A.t;
    const CellDecode& dec = A.dec;
    unsigned* st = A.st;
    const int tid = threadIdx.x;

    const int2 item = t.items[item_index];
    const int tile = item.x;
    const int tbeg = t.start[tile], tend = t.start[tile + 1];
    const int beg = tbeg + item.y * t.P;
    const int end = min(beg + t.P, tend);
    if (beg >= end) return;
    // box origin: the tile origin less the drift margin; particles sit in
    // local cells [0, T + 2m) of it
    const int t0[3] = {(tile % t.nt[0]) * t.T[0] - t.m[0], ((tile / t.nt[0]) % t.nt[1]) * t.T[1] - t.m[1],
                       DIM == 3 ? (tile / (t.nt[0] * t.nt[1])) * t.T[2] - t.m[2] : 0};
    const int Te[3] = {t.T[0] + 2 * t.m[0], t.T[1] + 2 * t.m[1], t.T[2] + 2 * t.m[2]};
    const TileSmem L = tile_smem(DIM, t.T, t.m);
    const int G0 = L.G[0], G1 = L.G[1], H0 = L.H[0], H1 = L.H[1];
    const int fsz = L.fsz, jsz = L.jsz;
    int* smw = reinterpret_cast<int*>(smem4);
    float* sF = reinterpret_cast<float*>(smw);
    int* sR = smw + L.off_r;
    int* sP = smw + L.off_p;
    int* sRing = smw + L.off_ring;
    int* sCnt = smw + L.off_cnt;

    // the next round's particles (cell, offsets, momenta, weight; the arrays
    // lie cap words apart).  3D: copied in 16-byte chunks, warp w copying
    // array w (a barrier orders them before use).  2D: each thread copies
    // its own particle's words, so a round needs no barrier.
    constexpr int NARR = DIM + 5 + (MODE == kGpdQed ? 1 : 0);
    constexpr int NBUF = DIM + 6;      // arrays per round buffer
    const long long astride = (long long)(reinterpret_cast<const char*>(p.off[0]) - reinterpret_cast<const char*>(p.cell));
    const int nround = (end - beg + kGpdThreads - 1) / kGpdThreads;
    auto prefetch = [&](int r) {
        const int rb = beg + r * kGpdThreads, re = min(rb + kGpdThreads, end);
        if constexpr (DIM == 2) {
            if (rb + tid < re) {
                const char* src = reinterpret_cast<const char*>(p.cell) + 4LL * (rb + tid);
                int* dst = sP + (r & 1) * NBUF * kRoundWords + tid;
#pragma unroll
                for (int k = 0; k < NARR; ++k) cp_async4(dst + k * kRoundWords, src + k * astride);
            }
        } else {
            const int a0 = rb & ~3, nch = (re - a0 + 3) >> 2;
            for (int arr = tid >> 5; arr < NARR; arr += kGpdThreads / 32) {
                const char* src = reinterpret_cast<const char*>(p.cell) + arr * astride + 4LL * a0;
                int* dst = sP + ((r & 1) * NBUF + arr) * kRoundWords;
                for (int q = tid & 31; q < nch; q += 32) cp_async16(dst + 4 * q, src + 16 * q);
            }
        }
    };
    prefetch(0);
    cp_async_commit();

    // fields of the box (local node x at index x + 1), zeroed current boxes
    for (int idx = tid; MODE != kGpdFieldsIn && idx < 6 * fsz; idx += kGpdThreads) {
        const int c = fdiv(idx, t.fF), r = idx - c * fsz;
        const int q = fdiv(r, t.fG0), lx = r - q * G0;
        const int lz = (DIM == 3) ? fdiv(q, t.fG1) : 0, ly = q - lz * G1;
        const long long m = fidx_near(g, t0[0] - 1 + lx, t0[1] - 1 + ly, DIM == 3 ? t0[2] - 1 + lz : 0);
        if (A.f64) {
            const double* src = c == 0 ? A.E64.p[0] : c == 1 ? A.E64.p[1] : c == 2 ? A.E64.p[2]
                              : c == 3 ? A.B64.p[0] : c == 4 ? A.B64.p[1] : A.B64.p[2];
            sF[idx] = (m < 0) ? 0.0f : (float)__ldg(src + m);
        } else {
            const float* src = c == 0 ? A.E.p[0] : c == 1 ? A.E.p[1] : c == 2 ? A.E.p[2]
                             : c == 3 ? A.B.p[0] : c == 4 ? A.B.p[1] : A.B.p[2];
            sF[idx] = (m < 0) ? 0.0f : __ldg(src + m);
        }
    }
    for (int q = tid; q < (L.off_p - L.off_r) / 4; q += kGpdThreads)
        reinterpret_cast<int4*>(sR)[q] = make_int4(0, 0, 0, 0);
    if (tid < kCntWords) sCnt[tid] = 0;
    constexpr bool BOX64 = DIM == 2;
    const int n4 = (L.off_64 - L.off_r) / 4;          // int32 boxes in groups of 4 nodes
    int4* sR4 = reinterpret_cast<int4*>(sR);
    longlong2* s64 = reinterpret_cast<longlong2*>(smw + L.off_64);

    // flush of the current boxes into the global int64 current (all threads;
    // callers place the barriers): the int64 boxes (2D), or the int32 boxes
    auto flush = [&]() {
        bool outside = false;
        for (int idx = tid; idx < 3 * jsz; idx += kGpdThreads) {
            long long v;
            if constexpr (BOX64) {
                v = reinterpret_cast<const long long*>(s64)[idx];
            } else {
                v = sR[idx];
                if (v != 0) sR[idx] = 0;
            }
            if (v == 0) continue;
            const int c = fdiv(idx, t.fJ), r = idx - c * jsz;
            const int q = fdiv(r, t.fH0), lx = r - q * H0;
            const int lz = (DIM == 3) ? fdiv(q, t.fH1) : 0, ly = q - lz * H1;
            const long long m = fidx_near(g, t0[0] - 2 + lx, t0[1] - 2 + ly, DIM == 3 ? t0[2] - 2 + lz : 0);
            if (m < 0) { outside = true; continue; }
            unsigned long long* dst = c == 0 ? J.p[0] : c == 1 ? J.p[1] : J.p[2];
            atomicAdd(dst + m, static_cast<unsigned long long>(v));
        }
        if (outside) set_status(st, LPIC_ST_OUTSIDE);
    };
    // 2D: adds the int32 boxes into the int64 boxes, four nodes at a time, and
    // clears them (callers place the barriers)
    auto fold = [&]() {
        for (int q = tid; q < n4; q += kGpdThreads) {
            const int4 v = sR4[q];
            if ((v.x | v.y | v.z | v.w) != 0) {
                longlong2 a = s64[2 * q], b = s64[2 * q + 1];
                a.x += v.x; a.y += v.y; b.x += v.z; b.y += v.w;
                s64[2 * q] = a; s64[2 * q + 1] = b;
                sR4[q] = make_int4(0, 0, 0, 0);
            }
        }
    };
    // makes room in the int32 boxes
    auto drain = [&]() {
        if constexpr (BOX64) fold(); else flush();
    };
    // 3D: the ring's general-form moves (full warps of one form)
    auto deposit_ring = [&](int slot) -> unsigned {
        Move<DIM> mv;
        mv.read(sRing + (slot & (kRing - 1)), kRing);
        deposit3d<ORDER>(Acc32<false>{sR, 3 * jsz, st}, jsz, H0, H1, mv.lc, mv.f, mv.ce, mv.fe, mv.s);
        return mv.template bound<ORDER>();
    };

    const float dth[3] = {A.dth0, A.dth1, A.dth2};
    const unsigned bmax = t.bmax;          // bound of any one move (units)
    unsigned total = 0;                    // bound accumulated since the boxes were emptied (block-uniform)
    int consumed = 0;                      // 3D ring entries deposited (block-uniform)

    // bound counters: round r adds to [r % 3], which every thread reads after
    // the first barrier of round r + 1; thread 0 clears [(r + 1) % 3] in round
    // r, after all threads read it (round r - 1) and before anyone adds to it
    int cc = 0;
    for (int rnd = 0; rnd < nround; ++rnd, cc = (cc == 2) ? 0 : cc + 1) {
        const int cprev = (cc == 0) ? 2 : cc - 1, cnext = (cc == 2) ? 0 : cc + 1;
        cp_async_wait_all();
        if (DIM == 3 || rnd == 0) __syncthreads();
        if (rnd + 1 < nround) prefetch(rnd + 1);
        cp_async_commit();
        if (DIM == 3 && MODE != kGpdGather) {
            // the previous round's moves are all accounted for: empty the boxes
            // if this round's (its own moves and a batch from the ring) could
            // overflow them (the host keeps 2 x 256 bmax within the limit)
            if (rnd > 0) total += (unsigned)sCnt[kCntBound + cprev];
            if (total + 2u * kGpdThreads * bmax > kBoundLimit) {
                drain();
                __syncthreads();
                total = 0;
            }
            if (tid == 0) sCnt[kCntBound + cnext] = 0;
        }

        const int rb = beg + rnd * kGpdThreads;
        const int i = rb + tid;
        const int* slot = sP + (rnd & 1) * NBUF * kRoundWords + (DIM == 3 ? rb - (rb & ~3) : 0) + tid;
        int cell = -1;
        float f[3] = {0.0f, 0.0f, 0.0f}, ux = 0.0f, uy = 0.0f, uz = 0.0f, w = 0.0f;
        if (i < end) {
            cell = slot[0];
#pragma unroll
            for (int d = 0; d < DIM; ++d) f[d] = __int_as_float(slot[(1 + d) * kRoundWords]);
            ux = __int_as_float(slot[(1 + DIM) * kRoundWords]);
            uy = __int_as_float(slot[(2 + DIM) * kRoundWords]);
            uz = __int_as_float(slot[(3 + DIM) * kRoundWords]);
            w = __int_as_float(slot[(4 + DIM) * kRoundWords]);
        }
        // form with emission: the particle's id and depth, loaded before the
        // gather so that the depth's latency overlaps it
        int qid = -1;
        float qtau = 0.0f;
        if (MODE == kGpdQed && cell >= 0) {
            qid = slot[(5 + DIM) * kRoundWords];
            if (qid >= 0 && (long long)qid < A.q.n_ids) qtau = A.q.tau[qid];
        }
        int cell_out = cell;            // the particle's cell after this round (-1: removed)
        unsigned bnd = 0;               // bound of the move this thread deposited
        if (cell >= 0) {
            int gc[3];
            dec(cell, gc);
            int lc[3] = {gc[0] - t0[0], gc[1] - t0[1], DIM == 3 ? gc[2] - t0[2] : 0};
            bool inside = true;
            const int nn[3] = {g.nx, g.ny, g.nz};
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                // a particle that crossed a periodic edge since the sort is
                // taken at its image next to the tile
                if (!(d == 0 && g.absorb)) {
                    if (lc[d] < 0) lc[d] += nn[d];
                    else if (lc[d] >= Te[d]) lc[d] -= nn[d];
                }
                inside &= (lc[d] >= 0 && lc[d] < Te[d]);
            }
            if (!inside) {
                if (MODE == kGpdFused || MODE == kGpdQed) {
                    // beyond the tile's drift margin: queued for the global-memory
                    // path, which also counts its new tile key
                    t.esc[atomicAdd(t.nesc, 1)] = i;
                } else {
                    // the unfused stages run on freshly sorted particles only
                    set_status(st, LPIC_ST_HALO);
                }
                cell_out = -1;
            } else {
                // gather at x^{n+1/2} from the shared-memory halo
                const NodeW<ORDER> nx_(lc[0], f[0]), ny_(lc[1], f[1]), nz_(lc[2], f[2]);
                const HalfW<ORDER> hx_(lc[0], f[0]), hy_(lc[1], f[1]), hz_(lc[2], f[2]);
                float fld[6];
                if constexpr (MODE == kGpdFieldsIn) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) fld[c] = A.fields[c * A.fcap + i];
                } else {
                    gather32<DIM, ORDER>(LoadShared<DIM>{sF, fsz, G0, G1, st}, nx_, ny_, nz_, hx_, hy_, hz_, fld);
                }
                if constexpr (MODE == kGpdGather) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) A.fields[c * A.fcap + i] = fld[c];
                } else {
                if constexpr (MODE == kGpdQed) {
                    // emission between the interpolation and the momentum push
                    // (Algorithm 1), with u^n and the fields at x^{n+1/2}; the
                    // photon leaves from x^{n+1/2}
                    if (qid < 0 || (long long)qid >= A.q.n_ids) {
                        set_status(st, LPIC_ST_OVERFLOW);
                    } else {
                        float uq[3] = {ux, uy, uz};
                        if (qed_emit(A.q, *A.q.step, DIM, qid, qtau, cell, f, w, uq, fld, st)) {
                            ux = uq[0]; uy = uq[1]; uz = uq[2];
                        }
                    }
                }
                boris_f32(ux, uy, uz, A.k, fld[0], fld[1], fld[2], fld[3], fld[4], fld[5]);
                if (!isfinite(ux) || !isfinite(uy) || !isfinite(uz)) {
                    set_status(st, LPIC_ST_NAN);
                    p.cell[i] = -1;
                    cell_out = -1;
                } else {
                    const float ig = rsqrtf(1.0f + ux * ux + uy * uy + uz * uz);
                    const float uu[3] = {ux, uy, uz};
                    Move<DIM> mv;
                    bool cfl = false;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        mv.lc[d] = lc[d]; mv.f[d] = f[d]; mv.ce[d] = lc[d]; mv.fe[d] = f[d];
                        if (d >= DIM) continue;
                        const float dl = uu[d] * ig * dth[d];
                        cfl |= !(fabsf(dl) < 1.0f);
                        const float fr = f[d] + dl;
                        int carry = (int)floorf(fr);
                        float fn = fr - (float)carry;
                        if (fn >= 1.0f) { fn -= 1.0f; carry += 1; }
                        mv.ce[d] = lc[d] + carry;
                        mv.fe[d] = fn;
                    }
                    if (cfl) {
                        set_status(st, LPIC_ST_CFL);
                        p.cell[i] = -1;
                        cell_out = -1;
                    } else {
                        // store x^{n+3/2} and u^{n+1}
                        int ng[3];
#pragma unroll
                        for (int d = 0; d < 3; ++d) ng[d] = (d < DIM) ? t0[d] + mv.ce[d] : 0;
                        bool dead = false;
                        if (g.absorb) dead = (ng[0] < 2 || ng[0] >= g.nx - 2);
                        else ng[0] = wrapi(ng[0], g.nx);
                        ng[1] = wrapi(ng[1], g.ny);
                        if (DIM == 3) ng[2] = wrapi(ng[2], g.nz);
                        cell_out = dead ? -1 : (ng[2] * g.ny + ng[1]) * g.nx + ng[0];
                        p.cell[i] = cell_out;
#pragma unroll
                        for (int d = 0; d < DIM; ++d) p.off[d][i] = mv.fe[d];
                        p.u[0][i] = ux; p.u[1][i] = uy; p.u[2][i] = uz;

                        mv.s = A.sq * w;
                        mv.vz = uz * ig;
                        const NodeW<ORDER> ex(mv.ce[0], mv.fe[0]), ey(mv.ce[1], mv.fe[1]), ez(mv.ce[2], mv.fe[2]);
                        mv.same = ex.base == nx_.base && ey.base == ny_.base && (DIM == 2 || ez.base == nz_.base);
                        if constexpr (DIM == 2) {
                            const Acc32<true> acc{sR, 3 * jsz, st};
                            // the stencil-sized window when every converged lane allows it
                            if (__all_sync(__activemask(), mv.same))
                                deposit2d_w<ORDER, true>(acc, jsz, H0, nx_, ny_, ex, ey, mv.s, mv.vz);
                            else
                                deposit2d_w<ORDER, false>(acc, jsz, H0, nx_, ny_, ex, ey, mv.s, mv.vz);
                        } else {
                            if (mv.same) {
                                bnd = mv.template bound<ORDER>();
                                deposit3d_w<ORDER>(Acc32<false>{sR, 3 * jsz, st}, jsz, H0, H1, nx_, ny_, nz_, ex, ey, ez, mv.s);
                            } else {
                                // staged: deposited with the other general-form moves
                                const int to = atomicAdd(sCnt + kCntRing, 1) & (kRing - 1);
                                mv.write(sRing + to, kRing);
                            }
                        }
                    }
                }
                }   // not the gather stage
            }
        }
        // histogram of the tile keys for the next sort (all lanes take part)
        if (t.next_count) {
            int key = -1;
            if (cell_out >= 0) {
                int gc2[3];
                dec(cell_out, gc2);
                key = (fdiv(gc2[2], t.fT[2]) * t.nt[1] + fdiv(gc2[1], t.fT[1])) * t.nt[0] + fdiv(gc2[0], t.fT[0]);
            }
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            if (key >= 0 && (tid & 31) == __ffs(peers) - 1)
                atomicAdd(t.next_count + key, __popc(peers));
        }
        if (MODE == kGpdGather) continue;
        if constexpr (DIM == 3) {
            // a full batch of general-form moves from the ring
            __syncthreads();
            if (sCnt[kCntRing] - consumed >= kGpdThreads) {
                bnd += deposit_ring(consumed + tid);
                consumed += kGpdThreads;
            }
            const unsigned wb = __reduce_add_sync(0xffffffffu, bnd);
            if ((tid & 31) == 0 && wb) atomicAdd(reinterpret_cast<unsigned*>(sCnt) + kCntBound + cc, wb);
        } else {
            // 2D: every R rounds (and after the last) fold the int32 boxes
            // into the int64 boxes (the host's R keeps them in range)
            if ((rnd + 1) % t.R == 0 || rnd + 1 == nround) { __syncthreads(); fold(); __syncthreads(); }
        }
    }
    if (MODE == kGpdGather) return;
    if constexpr (DIM == 3) {
        __syncthreads();
        // the moves still in the ring (fewer than 512), in batches of 256
        total += (unsigned)sCnt[kCntBound + (nround - 1) % 3];
        const int queued = sCnt[kCntRing];
        while (queued - consumed > 0) {
            if (total + kGpdThreads * bmax > kBoundLimit) { drain(); __syncthreads(); total = 0; }
            if (tid < queued - consumed) deposit_ring(consumed + tid);
            consumed += kGpdThreads;
            total += kGpdThreads * bmax;
            __syncthreads();
        }
    }
    // one flush of the item's current to the global int64 arrays (2D: the
    // int64 boxes, folded after the last round)
    flush();
}

template <int DIM, int ORDER, int MODE = kGpdFused>
__global__ void __launch_bounds__(256, DIM == 2 ? LPIC_GPD2D_MINB : LPIC_GPD3D_MINB) k_gpd32(GpdArgs A) {
    extern __shared__ float4 smem4[];
    if ((int)blockIdx.x >= *A.t.nitems) return;
    gpd_item<DIM, ORDER, MODE>(A, blockIdx.x, smem4);
}

// Persistent form for a batch of grids: blocks pull work items from one
// device queue that runs over the species slots in the given order (densest
// first), slots[order[r]] owning queue entries prefix[r] .. prefix[r+1]-1.
template <int DIM, int ORDER>
__global__ void __launch_bounds__(256, DIM == 2 ? LPIC_GPD2D_MINB : LPIC_GPD3D_MINB)
k_gpd32_queue(const GpdArgs* slots, const int* order, const int* prefix, int nslots, int* head) {
    extern __shared__ float4 smem4[];
    __shared__ int s_q;
    const int total = prefix[nslots];
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(head, 1);
        __syncthreads();
        const int q = s_q;
        __syncthreads();
        if (q >= total) break;
        int lo = 0, hi = nslots;             // prefix[lo] <= q < prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (prefix[mid] <= q) lo = mid; else hi = mid;
        }
        gpd_item<DIM, ORDER>(slots[order[lo]], q - prefix[lo], smem4);
        __syncthreads();
    }
}

// Accumulates a deposit straight into the global int64 J.  The deposit's box
// index is read in a virtual box of HV nodes per dimension whose local frame
// puts the particle's cell at 2: box coordinate X is global node gc + X - 4.
template <int DIM>
struct AccGlobal {
    static constexpr int HV = 10;
    const Geo* g;
    Ptr3<unsigned long long> J;
    int gc[3];
    unsigned* st;
    __device__ __forceinline__ void operator()(int idx, int v) const {
        if (v == 0) return;
        constexpr int jsz = (DIM == 3) ? HV * HV * HV : HV * HV;
        const int c = idx / jsz, r = idx - c * jsz;
        const int X = r % HV, Y = (r / HV) % HV, Z = r / (HV * HV);
        const long long m = fidx(*g, gc[0] + X - 4, gc[1] + Y - 4, DIM == 3 ? gc[2] + Z - 4 : 0);
        if (m < 0) { set_status(st, LPIC_ST_OUTSIDE); return; }
        unsigned long long* dst = c == 0 ? J.p[0] : c == 1 ? J.p[1] : J.p[2];
        atomicAdd(dst + m, static_cast<unsigned long long>(static_cast<long long>(v)));
    }
};

// The same push for the particles the tile kernel queued: fields gathered from
// global memory, current added with global integer atomics (same integer
// quantisation, so the result is identical to the shared-memory path).
template <int DIM, int ORDER>
__global__ void __launch_bounds__(256) k_gpd32_escape(GpdArgs A) {
    const Geo& g = A.g;
    const Ptr3<const float>& E = A.E;
    const Ptr3<const float>& B = A.B;
    const Ptr3<unsigned long long>& J = A.J;
    const P32& p = A.p;
    const Tiles& t = A.t;
    const CellDecode& dec = A.dec;
    const float k = A.k, sq = A.sq, dth0 = A.dth0, dth1 = A.dth1, dth2 = A.dth2;
    unsigned* st = A.st;
    const int nesc = *t.nesc;
    const float dth[3] = {dth0, dth1, dth2};
    const int stride = gridDim.x * blockDim.x;
    const int nround = (nesc + stride - 1) / stride;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    for (int r = 0; r < nround; ++r, j += stride) {
        int cell_out = -1;
        if (j < nesc) {
            const int i = t.esc[j];
            int gc[3];
            dec(p.cell[i], gc);
            if (DIM == 2) gc[2] = 0;
            float f[3] = {p.off[0][i], p.off[1][i], DIM == 3 ? p.off[2][i] : 0.0f};
            float ux = p.u[0][i], uy = p.u[1][i], uz = p.u[2][i];
            const float w = p.w[i];
            // local frame with the particle's cell at 2 (lc = 2)
            int lc[3] = {2, 2, DIM == 3 ? 2 : 0};
            const NodeW<ORDER> nx_(lc[0], f[0]), ny_(lc[1], f[1]), nz_(lc[2], f[2]);
            const HalfW<ORDER> hx_(lc[0], f[0]), hy_(lc[1], f[1]), hz_(lc[2], f[2]);
            float fld[6];
            bool outside = false;
            const LoadGlobal<DIM> ld{&g, {E.p[0], E.p[1], E.p[2], B.p[0], B.p[1], B.p[2]},
                                     {A.f64 ? A.E64.p[0] : nullptr, A.E64.p[1], A.E64.p[2], A.B64.p[0],
                                      A.B64.p[1], A.B64.p[2]},
                                     {gc[0], gc[1], gc[2]}, &outside};
            gather32<DIM, ORDER>(ld, nx_, ny_, nz_, hx_, hy_, hz_, fld);
            if (outside) set_status(st, LPIC_ST_OUTSIDE);
            if (A.qed) {
                // the emission of the tile kernel's kGpdQed form
                const int id = p.id[i];
                if (id < 0 || (long long)id >= A.q.n_ids) {
                    set_status(st, LPIC_ST_OVERFLOW);
                } else {
                    float uq[3] = {ux, uy, uz};
                    if (qed_emit(A.q, *A.q.step, DIM, id, A.q.tau[id], p.cell[i], f, w, uq, fld, st)) {
                        ux = uq[0]; uy = uq[1]; uz = uq[2];
                    }
                }
            }
            boris_f32(ux, uy, uz, k, fld[0], fld[1], fld[2], fld[3], fld[4], fld[5]);
            if (!isfinite(ux) || !isfinite(uy) || !isfinite(uz)) {
                set_status(st, LPIC_ST_NAN);
                p.cell[i] = -1;
            } else {
                const float ig = rsqrtf(1.0f + ux * ux + uy * uy + uz * uz);
                const float uu[3] = {ux, uy, uz};
                int ce[3] = {lc[0], lc[1], lc[2]};
                float fe[3] = {0.0f, 0.0f, 0.0f};
                bool cfl = false;
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    const float dl = uu[d] * ig * dth[d];
                    cfl |= !(fabsf(dl) < 1.0f);
                    const float fr = f[d] + dl;
                    int carry = (int)floorf(fr);
                    float fn = fr - (float)carry;
                    if (fn >= 1.0f) { fn -= 1.0f; carry += 1; }
                    ce[d] = lc[d] + carry;
                    fe[d] = fn;
                }
                if (cfl) {
                    set_status(st, LPIC_ST_CFL);
                    p.cell[i] = -1;
                } else {
                    const AccGlobal<DIM> acc{&g, J, {gc[0], gc[1], gc[2]}, st};
                    constexpr int HV = AccGlobal<DIM>::HV;
                    const float s = sq * w;
                    // the same form of the deposit as the tile kernel takes
                    const bool same = same_stencils<DIM, ORDER>(lc, f, ce, fe);
                    if (DIM == 3) {
                        if (same) deposit3d_same<ORDER>(acc, HV * HV * HV, HV, HV, lc, f, ce, fe, s);
                        else      deposit3d<ORDER>(acc, HV * HV * HV, HV, HV, lc, f, ce, fe, s);
                    } else {
                        if (same) deposit2d_same<ORDER>(acc, HV * HV, HV, lc, f, ce, fe, s, uz * ig);
                        else      deposit2d<ORDER>(acc, HV * HV, HV, lc, f, ce, fe, s, uz * ig);
                    }
                    int ng[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) ng[d] = (d < DIM) ? gc[d] + ce[d] - lc[d] : 0;
                    bool dead = false;
                    if (g.absorb) dead = (ng[0] < 2 || ng[0] >= g.nx - 2);
                    else ng[0] = wrapi(ng[0], g.nx);
                    ng[1] = wrapi(ng[1], g.ny);
                    if (DIM == 3) ng[2] = wrapi(ng[2], g.nz);
                    cell_out = dead ? -1 : (ng[2] * g.ny + ng[1]) * g.nx + ng[0];
                    p.cell[i] = cell_out;
#pragma unroll
                    for (int d = 0; d < DIM; ++d) p.off[d][i] = fe[d];
                    p.u[0][i] = ux; p.u[1][i] = uy; p.u[2][i] = uz;
                }
            }
        }
        if (t.next_count) {
            int key = -1;
            if (cell_out >= 0) {
                int gc2[3];
                dec(cell_out, gc2);
                key = (fdiv(gc2[2], t.fT[2]) * t.nt[1] + fdiv(gc2[1], t.fT[1])) * t.nt[0] + fdiv(gc2[0], t.fT[0]);
            }
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            if (key >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
                atomicAdd(t.next_count + key, __popc(peers));
        }
    }
}

// x^0 -> x^{1/2}: offsets advance by (dt/2) v / h with carries into the cell.
template <int DIM>
__global__ void k_advance32(Geo g, P32 p, CellDecode dec, float frac, float dth0, float dth1,
                            float dth2) {
    const int n = *p.n;
    const float dth[3] = {dth0, dth1, dth2};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int cell = p.cell[i];
        if (cell < 0) continue;
        int gc[3];
        dec(cell, gc);
        const float ux = p.u[0][i], uy = p.u[1][i], uz = p.u[2][i];
        const float ig = 1.0f / sqrtf(1.0f + ux * ux + uy * uy + uz * uz);
        const float uu[3] = {ux, uy, uz};
        const int nn[3] = {g.nx, g.ny, g.nz};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const float fr = p.off[d][i] + frac * uu[d] * ig * dth[d];
            int carry = (int)floorf(fr);
            float fn = fr - (float)carry;
            if (fn >= 1.0f) { fn -= 1.0f; carry += 1; }
            gc[d] += carry;
            if (!(d == 0 && g.absorb)) gc[d] = wrapi(gc[d], nn[d]);
            p.off[d][i] = fn;
        }
        if (DIM == 2) gc[2] = 0;
        p.cell[i] = (gc[0] < 0 || gc[0] >= g.nx) ? -1 : (gc[2] * g.ny + gc[1]) * g.nx + gc[0];
    }
}

template <int DIM, int ORDER>
__global__ void k_charge32(Geo g, P32 p, CellDecode dec, float sq, unsigned long long* rho) {
    const int n = *p.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int cell = p.cell[i];
        if (cell < 0) continue;
        int gc[3];
        dec(cell, gc);
        const float f[3] = {p.off[0][i], p.off[1][i], DIM == 3 ? p.off[2][i] : 0.0f};
        charge_int<DIM, ORDER>(rho, g, gc, f, sq * p.w[i]);
    }
}

}  // namespace lpic
