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
// with native 32-bit atomics; every R rounds the box is folded into an int64
// box.  The shift F keeps every particle's integer charge S <= 2^22, and the
// host derives R from a bound on one move's current per node (a fraction of
// S set by the Courant number and the shape), so the int32 box cannot
// overflow between folds.
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
// to the charge at the start of the next step's path.  The Esirkepov weights
// W_d (Sec. 3.1) are quantised with closures that make the integer current
// a valid flow for the integer charge change dQ = Q1 - Q0:
//   2D: W_x = rint(s DS_x A_y) except the last column (b), fixed so that
//       sum_b W_x(a, .) = M(a) = qx1(a) - qx0(a), and the last row (a), fixed
//       so that sum_a W_x(., b) = 0; W_y = dQ - W_x.
//   3D: the same construction on the column sums over c (targets X, Y for
//       sum_c W_x, sum_c W_y with X + Y = qxy1 - qxy0), then W_x, W_y per node
//       with closures along c (to X, Y) and along a / b (to 0);
//       W_z = dQ - W_x - W_y.
// J_d is then the running sum of -W_d along d and satisfies, node by node,
// J_d(i+1/2) - J_d(i-1/2) summed over d = -(Q1 - Q0) exactly.
#pragma once
#include "lpic_common.cuh"

namespace lpic {

struct P32 {
    int* cell;
    float* off[3];
    float* u[3];
    float* w;
    int* id;
    const int* n;
};

struct Tiles {
    int T[3];            // cells per tile
    int nt[3];           // tiles per dimension
    int m[3];            // margin (cells) the particles may have drifted since the sort
    const int* start;    // ntiles + 1 prefix offsets (after the sort)
    const int2* items;   // (tile, chunk) work items
    const int* nitems;   // device count of work items
    int P;               // particles per chunk
    int R;               // rounds between folds of the int32 current box
    FastDiv fT[3];       // division by T (tile keys of the next sort)
    FastDiv fG0, fG1, fF;  // division by the field box rows, planes, size
    FastDiv fH0, fH1, fJ;  // and by those of the current box
    int* next_count;     // if set: histogram of the new tile keys for the next sort
    int* esc;            // indices of particles beyond the tile's margin ...
    int* nesc;           // ... and their count (pushed by k_gpd32_escape)
};

template <int ORDER, class W>
__device__ inline void place32(float (&S)[ORDER + 2], const W& w, int off) {
#pragma unroll
    for (int a = 0; a < ORDER + 2; ++a) {
        const float lo = (a <= ORDER) ? w.w[a < ORDER + 1 ? a : 0] : 0.0f;
        const float hi = (a >= 1) ? w.w[a >= 1 ? a - 1 : 0] : 0.0f;
        S[a] = off ? hi : lo;
    }
}

// Adds a lane's value to the int32 round box with a native 32-bit atomic.
// SKIP_ZERO: only nonzero values (2D: slowly moving particles leave most
// window values at zero and lanes of one cell would otherwise all hit the same
// addresses; 3D: most values are nonzero and the test costs more than it saves
// -- both measured).
template <bool SKIP_ZERO>
struct Acc32 {
    int* sJ;
    __device__ inline void operator()(int idx, int v) const {
        if (!SKIP_ZERO || v != 0) atomicAdd(sJ + idx, v);
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

// ----------------------------------------------------------- 2D deposit
// The construction on a window of WN nodes per dimension starting at
// (basex, basey); the start/end stencils sit at offsets o0*/o1* in it.
// Node (a, b) of component c lives at c * jsz + (b + 2) * H0 + (a + 2) of the
// box (coordinates relative to the box's local frame).
// The rounding residuals of W_x go to row cx and column cy: the stencil's
// last node where both stencils coincide in that dimension (so that the
// window size never changes the integers), else the window's last node.
template <int ORDER, int WN, class Acc>
__device__ inline void deposit2d_core(const Acc& acc, int jsz, int H0, int basex, int basey, int o0x,
                                      int o1x, int o0y, int o1y, int cx, int cy,
                                      const float (&S0x)[WN], const float (&S1x)[WN],
                                      const float (&S0y)[WN], const float (&S1y)[WN], float s, float vz) {
    const int sint = rint22(s);
    int qx0[WN], qx1[WN], dQ[WN][WN], M[WN];
    {
        int qxy0[WN][WN], qxy1[WN][WN];
        charge_levels_1d<WN>(s, sint, S0x, o0x, qx0);
        charge_levels_1d<WN>(s, sint, S1x, o1x, qx1);
        charge_levels_2d<WN>(qx0, S0y, o0y, qxy0);
        charge_levels_2d<WN>(qx1, S1y, o1y, qxy1);
#pragma unroll
        for (int a = 0; a < WN; ++a) {
            M[a] = qx1[a] - qx0[a];
#pragma unroll
            for (int b = 0; b < WN; ++b) dQ[a][b] = qxy1[a][b] - qxy0[a][b];
        }
    }

    float DSx[WN], DSy[WN], Ax[WN], Ay[WN];
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        DSx[a] = S1x[a] - S0x[a]; DSy[a] = S1y[a] - S0y[a];
        Ax[a] = 0.5f * (S0x[a] + S1x[a]); Ay[a] = 0.5f * (S0y[a] + S1y[a]);
    }
    // W_x with closures on row cx and column cy; W_y = dQ - W_x
    int Wx[WN][WN];
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        int row = 0;
        const float sdx = s * DSx[a];
#pragma unroll
        for (int b = 0; b < WN; ++b) {
            const int v = (b == cy) ? 0 : rint22_mul(sdx, Ay[b]);
            Wx[a][b] = v; row += v;
        }
#pragma unroll
        for (int b = 0; b < WN; ++b)
            if (b == cy) Wx[a][b] = M[a] - row;
    }
#pragma unroll
    for (int b = 0; b < WN; ++b) {
        int col = 0;
#pragma unroll
        for (int a = 0; a < WN; ++a) col += (a == cx) ? 0 : Wx[a][b];
#pragma unroll
        for (int a = 0; a < WN; ++a)
            if (a == cx) Wx[a][b] = -col;
    }
    // J_x: running sum along a; J_y: running sum along b
#pragma unroll
    for (int b = 0; b < WN; ++b) {
        int run = 0;
#pragma unroll
        for (int a = 0; a < WN - 1; ++a) {
            run -= Wx[a][b];
            acc((basey + b + 2) * H0 + (basex + a + 2), run);
        }
    }
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        int run = 0;
#pragma unroll
        for (int b = 0; b < WN - 1; ++b) {
            run -= dQ[a][b] - Wx[a][b];
            acc(jsz + (basey + b + 2) * H0 + (basex + a + 2), run);
        }
    }
    // J_z: s v_z W_z, W_z = A_x A_y + DS_x DS_y / 12 (needs no closure in 2D,
    // so any fixed integer rounding of it will do: the DS term is rounded to an
    // integer first, then the sum)
    const float svz = s * vz, svz12 = svz * (1.0f / 12.0f);
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        const float pa = svz * Ax[a], qa = svz12 * DSx[a];
#pragma unroll
        for (int b = 0; b < WN; ++b) {
            const float t = __fmaf_rn(qa, DSy[b], 12582912.0f);
            acc(2 * jsz + (basey + b + 2) * H0 + (basex + a + 2),
                __float_as_int(__fmaf_rn(pa, Ay[b], t)) - 0x4B400000);
        }
    }
}

// General case: the window of ORDER + 2 nodes holds both stencils.
template <int ORDER, class Acc>
__device__ inline void deposit2d(const Acc& acc, int jsz, int H0, const int* lc, const float* f,
                                 const int* ce, const float* fe, float s, float vz) {
    constexpr int WN = ORDER + 2;
    const NodeW<ORDER> ax(lc[0], f[0]), ay(lc[1], f[1]), bx(ce[0], fe[0]), by(ce[1], fe[1]);
    const int basex = min(ax.base, bx.base), basey = min(ay.base, by.base);
    const int o0x = ax.base - basex, o1x = bx.base - basex;
    const int o0y = ay.base - basey, o1y = by.base - basey;
    float S0x[WN], S1x[WN], S0y[WN], S1y[WN];
    place32<ORDER>(S0x, ax, o0x); place32<ORDER>(S1x, bx, o1x);
    place32<ORDER>(S0y, ay, o0y); place32<ORDER>(S1y, by, o1y);
    const int cx = (o0x == o1x) ? o0x + ORDER : WN - 1;
    const int cy = (o0y == o1y) ? o0y + ORDER : WN - 1;
    deposit2d_core<ORDER, WN>(acc, jsz, H0, basex, basey, o0x, o1x, o0y, o1y, cx, cy, S0x, S1x, S0y, S1y,
                              s, vz);
}

// Both stencils start at the same node in both dimensions (the particle kept
// its nearest node): the window is the stencil itself, ORDER + 1 nodes.
template <int ORDER, class Acc>
__device__ inline void deposit2d_same(const Acc& acc, int jsz, int H0, const int* lc, const float* f,
                                      const int* ce, const float* fe, float s, float vz) {
    constexpr int WN = ORDER + 1;
    const NodeW<ORDER> ax(lc[0], f[0]), ay(lc[1], f[1]), bx(ce[0], fe[0]), by(ce[1], fe[1]);
    float S0x[WN], S1x[WN], S0y[WN], S1y[WN];
#pragma unroll
    for (int a = 0; a < WN; ++a) { S0x[a] = ax.w[a]; S1x[a] = bx.w[a]; S0y[a] = ay.w[a]; S1y[a] = by.w[a]; }
    deposit2d_core<ORDER, WN>(acc, jsz, H0, ax.base, ay.base, 0, 0, 0, 0, ORDER, ORDER, S0x, S1x, S0y, S1y,
                              s, vz);
}

// ----------------------------------------------------------- 3D deposit
// Same construction as the 2D deposit one level up, evaluated slab by slab
// in y (b) so that only the closure sums cross slabs: X(a, b) (target of
// sum_c W_x) per slab with running row sums, W_y(a, b, c) with running sums
// over b (their negative is J_y), and W_z = dQ - W_x - W_y inside the slab.
// Window of WN nodes per dimension from (bs0, bs1, bs2); the start/end
// stencils sit at offsets o*0 / o*1 in it; residuals go to the window's last
// node.
template <int ORDER, int WN, class Acc>
__device__ inline void deposit3d_core(const Acc& acc, int jsz, int H0, int H1, int bs0, int bs1, int bs2,
                                      int ox0, int ox1, int oy0, int oy1, int oz0, int oz1,
                                      const float (&S0x)[WN], const float (&S1x)[WN],
                                      const float (&S0y)[WN], const float (&S1y)[WN],
                                      const float (&S0z)[WN], const float (&S1z)[WN], float s) {
    constexpr int L = WN - 1;
    const int sint = rint22(s);

    int qx0[WN], qx1[WN], qxy0[WN][WN], qxy1[WN][WN];
    charge_levels_1d<WN>(s, sint, S0x, ox0, qx0);
    charge_levels_1d<WN>(s, sint, S1x, ox1, qx1);
    charge_levels_2d<WN>(qx0, S0y, oy0, qxy0);
    charge_levels_2d<WN>(qx1, S1y, oy1, qxy1);

    int xrow[WN];          // running sum over b of X(a, b), a < L
    int wys[WN][WN];       // running sum over b of W_y(a, b, c)
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        xrow[a] = 0;
#pragma unroll
        for (int c = 0; c < WN; ++c) wys[a][c] = 0;
    }
    float sdx[WN], Az[WN], DSz[WN];
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        sdx[a] = s * (S1x[a] - S0x[a]);
        Az[a] = 0.5f * (S0z[a] + S1z[a]); DSz[a] = S1z[a] - S0z[a];
    }
#pragma unroll
    for (int b = 0; b < WN; ++b) {
        const float ay = 0.5f * (S0y[b] + S1y[b]), dsy = S1y[b] - S0y[b];
        const float sdy = s * dsy, dsy12 = dsy * (1.0f / 12.0f);
        // X(., b) with its closures; Y(., b) = Z(., b) - X(., b)
        int X[WN];
        {
            int col = 0;
#pragma unroll
            for (int a = 0; a < L; ++a) {
                const int v = (b < L) ? rint22_mul(sdx[a], ay) : (qx1[a] - qx0[a]) - xrow[a];
                X[a] = v; xrow[a] += v; col += v;
            }
            X[L] = -col;
        }
        // dQ of the slab (levels continued along z with the column remainders)
        int dq[WN][WN];
#pragma unroll
        for (int a = 0; a < WN; ++a) {
            const float f0 = (float)qxy0[a][b], f1 = (float)qxy1[a][b];
            int sum0 = 0, sum1 = 0;
#pragma unroll
            for (int c = 0; c < WN; ++c) {
                const int q0 = rint22_mul(f0, S0z[c]);
                const int q1 = rint22_mul(f1, S1z[c]);
                dq[a][c] = q1 - q0; sum0 += q0; sum1 += q1;
            }
#pragma unroll
            for (int c = 0; c < WN; ++c)
                dq[a][c] += ((c == oz1 + 1) ? qxy1[a][b] - sum1 : 0) - ((c == oz0 + 1) ? qxy0[a][b] - sum0 : 0);
        }
        // W_x(a, b, c) = s DS_x(a) (A_y A_z + DS_y DS_z / 12); J_x runs along a
        {
            int cs[WN];
#pragma unroll
            for (int a = 0; a < WN; ++a) cs[a] = 0;
#pragma unroll
            for (int c = 0; c < WN; ++c) {
                const float kyz = __fmaf_rn(ay, Az[c], dsy12 * DSz[c]);
                int colsum = 0, run = 0;
#pragma unroll
                for (int a = 0; a < L; ++a) {
                    const int v = (c < L) ? rint22_mul(sdx[a], kyz) : X[a] - cs[a];
                    cs[a] += v; colsum += v;
                    dq[a][c] -= v;
                    run -= v;
                    acc(((bs2 + c + 2) * H1 + (bs1 + b + 2)) * H0 + (bs0 + a + 2), run);
                }
                dq[L][c] += colsum;
            }
        }
        // W_y(a, b, c) = s DS_y(b) (A_x A_z + DS_x DS_z / 12) with sum_c W_y = Y(a, b);
        // the last slab closes sum_b W_y = 0.  J_y is minus the running sum over b.
#pragma unroll
        for (int a = 0; a < WN; ++a) {
            const float ax = 0.5f * (S0x[a] + S1x[a]), dsx12 = (S1x[a] - S0x[a]) * (1.0f / 12.0f);
            const int Y = (qxy1[a][b] - qxy0[a][b]) - X[a];
            int cs = 0;
#pragma unroll
            for (int c = 0; c < WN; ++c) {
                int v;
                if (b < L) {
                    v = (c < L) ? rint22_mul(sdy, __fmaf_rn(ax, Az[c], dsx12 * DSz[c])) : Y - cs;
                    cs += v;
                    wys[a][c] += v;
                    acc(jsz + ((bs2 + c + 2) * H1 + (bs1 + b + 2)) * H0 + (bs0 + a + 2), -wys[a][c]);
                } else {
                    v = -wys[a][c];
                }
                dq[a][c] -= v;
            }
        }
        // W_z = what is left; J_z runs along c
#pragma unroll
        for (int a = 0; a < WN; ++a) {
            int run = 0;
#pragma unroll
            for (int c = 0; c < L; ++c) {
                run -= dq[a][c];
                acc(2 * jsz + ((bs2 + c + 2) * H1 + (bs1 + b + 2)) * H0 + (bs0 + a + 2), run);
            }
        }
    }
}


// General case: the window of ORDER + 2 nodes per dimension holds both stencils.
template <int ORDER, class Acc>
__device__ inline void deposit3d(const Acc& acc, int jsz, int H0, int H1, const int* lc,
                                 const float* f, const int* ce, const float* fe, float s) {
    constexpr int WN = ORDER + 2;
    const NodeW<ORDER> a0(lc[0], f[0]), a1(lc[1], f[1]), a2(lc[2], f[2]);
    const NodeW<ORDER> b0(ce[0], fe[0]), b1(ce[1], fe[1]), b2(ce[2], fe[2]);
    const int bs0 = min(a0.base, b0.base), bs1 = min(a1.base, b1.base), bs2 = min(a2.base, b2.base);
    float S0x[WN], S1x[WN], S0y[WN], S1y[WN], S0z[WN], S1z[WN];
    place32<ORDER>(S0x, a0, a0.base - bs0); place32<ORDER>(S1x, b0, b0.base - bs0);
    place32<ORDER>(S0y, a1, a1.base - bs1); place32<ORDER>(S1y, b1, b1.base - bs1);
    place32<ORDER>(S0z, a2, a2.base - bs2); place32<ORDER>(S1z, b2, b2.base - bs2);
    deposit3d_core<ORDER, WN>(acc, jsz, H0, H1, bs0, bs1, bs2, a0.base - bs0, b0.base - bs0,
                              a1.base - bs1, b1.base - bs1, a2.base - bs2, b2.base - bs2,
                              S0x, S1x, S0y, S1y, S0z, S1z, s);
}

// Both stencils start at the same node in every dimension: the window is the
// stencil itself, ORDER + 1 nodes per dimension.
template <int ORDER, class Acc>
__device__ inline void deposit3d_same(const Acc& acc, int jsz, int H0, int H1, const int* lc,
                                      const float* f, const int* ce, const float* fe, float s) {
    constexpr int WN = ORDER + 1;
    const NodeW<ORDER> a0(lc[0], f[0]), a1(lc[1], f[1]), a2(lc[2], f[2]);
    const NodeW<ORDER> b0(ce[0], fe[0]), b1(ce[1], fe[1]), b2(ce[2], fe[2]);
    float S0x[WN], S1x[WN], S0y[WN], S1y[WN], S0z[WN], S1z[WN];
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        S0x[a] = a0.w[a]; S1x[a] = b0.w[a]; S0y[a] = a1.w[a]; S1y[a] = b1.w[a];
        S0z[a] = a2.w[a]; S1z[a] = b2.w[a];
    }
    deposit3d_core<ORDER, WN>(acc, jsz, H0, H1, a0.base, a1.base, a2.base, 0, 0, 0, 0, 0, 0,
                              S0x, S1x, S0y, S1y, S0z, S1z, s);
}

// Whether the start and end stencils of a move begin at the same node in
// every dimension (then the stencil-sized window holds the whole deposit).
template <int DIM, int ORDER>
__device__ inline bool same_stencils(const int* lc, const float* f, const int* ce, const float* fe) {
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
// component with a halo of 2, local node (x, y, z) at ((z+2) G1 + y+2) G0 + x+2
// (2D: y+2) G0 + x+2).
template <int DIM>
struct LoadShared {
    const float* sF;
    int fsz, G0, G1;
    __device__ inline float operator()(int comp, int x, int y, int z) const {
        return sF[comp * fsz + ((DIM == 3 ? z + 2 : 0) * G1 + (y + 2)) * G0 + (x + 2)];
    }
};

// Field components read from global memory around a particle whose cell is
// gc, local frame with the particle's cell at 2; nodes outside the grid
// (absorbing x) read 0 and raise the flag.
template <int DIM>
struct LoadGlobal {
    const Geo* g;
    const float* F[6];
    int gc[3];
    bool* outside;
    __device__ inline float operator()(int comp, int x, int y, int z) const {
        const long long m = fidx(*g, gc[0] + x - 2, gc[1] + y - 2, DIM == 3 ? gc[2] + z - 2 : 0);
        if (m < 0) { *outside = true; return 0.0f; }
        return F[comp][m];
    }
};

// ----------------------------------------------------------- the tile kernel
// Shared memory: 6 field boxes (T+4 per dimension, halo 2 below and 2 above),
// an int64 total box and an int32 round box for J (T+5 per dimension), then in
// 3D the deposit staging and in 2D the particle prefetch buffers.
// Blocks per SM the register allocation targets (2D: the kernel fits 80
// registers with negligible spills; 3D: 128 registers, a few spills, measured
// 1.57x faster than one block per SM at 255 registers).
#ifndef LPIC_GPD2D_MINB
#define LPIC_GPD2D_MINB 4
#endif
#ifndef LPIC_GPD3D_MINB
#define LPIC_GPD3D_MINB 2
#endif

// Threads per block of the tile kernel, and the 3D deposit staging in shared
// memory (words per slot: packed start cell, packed end-cell carries, start
// offsets, end offsets, charge): 256 slots for a round's same-stencil moves
// and a ring of 512 for the other moves, deposited 256 at a time.
constexpr int kGpdThreads = 256;
constexpr int kStageWords = 9;
constexpr int kRing = 2 * kGpdThreads;
constexpr int kStageBytes = (kStageWords * (kGpdThreads + kRing) + 4) * 4;
// 2D: the next round's particles (cell, 2 offsets, 3 momenta, weight) are
// copied into shared memory asynchronously while the current round runs, two
// buffers of one word per thread and array.
constexpr int kPrefWords = 7;
constexpr int kPrefBytes = 2 * kPrefWords * kGpdThreads * 4;

__device__ inline void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// One staged move: write / read kStageWords words at slot stride `stride`.
__device__ inline void stage_move(int* w, int stride, const int* lc, const int* ce, const float* f0,
                                  const float* f1, float s) {
    w[0] = lc[0] | (lc[1] << 16);
    w[stride] = lc[2] | (((ce[0] - lc[0] + 1) | ((ce[1] - lc[1] + 1) << 2) | ((ce[2] - lc[2] + 1) << 4)) << 16);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        w[(2 + d) * stride] = __float_as_int(f0[d]);
        w[(5 + d) * stride] = __float_as_int(f1[d]);
    }
    w[8 * stride] = __float_as_int(s);
}

template <int ORDER, bool SAME, class Acc>
__device__ inline void deposit_staged3d(const Acc& acc, int jsz, int H0, int H1, const int* w, int stride) {
    const int w0 = w[0], w1 = w[stride];
    const int lc[3] = {w0 & 0xffff, (int)((unsigned)w0 >> 16), w1 & 0xffff};
    const int cc = (int)((unsigned)w1 >> 16);
    const int ce[3] = {lc[0] + (cc & 3) - 1, lc[1] + ((cc >> 2) & 3) - 1, lc[2] + ((cc >> 4) & 3) - 1};
    const float f[3] = {__int_as_float(w[2 * stride]), __int_as_float(w[3 * stride]),
                        __int_as_float(w[4 * stride])};
    const float fe[3] = {__int_as_float(w[5 * stride]), __int_as_float(w[6 * stride]),
                         __int_as_float(w[7 * stride])};
    const float s = __int_as_float(w[8 * stride]);
    if (SAME) deposit3d_same<ORDER>(acc, jsz, H0, H1, lc, f, ce, fe, s);
    else      deposit3d<ORDER>(acc, jsz, H0, H1, lc, f, ce, fe, s);
}

// Everything the fused kernel needs for one species of one grid.
struct GpdArgs {
    Geo g;
    Ptr3<const float> E, B;
    Ptr3<unsigned long long> J;
    P32 p;
    Tiles t;
    CellDecode dec;
    float k, sq, dth0, dth1, dth2;
    unsigned* st;
    float* fields;       // unfused stages: per-particle E_x..B_z, [6][fcap]
    long long fcap;
};

// Forms of the tile kernel: the fused gather/push/deposit, and the two
// stages of the unfused path (the gather alone, writing each particle's
// fields; the push and deposit with fields read back).  Between them the
// caller may change the fields (an external field, a diagnostic).
enum { kGpdFused = 0, kGpdGather = 1, kGpdFieldsIn = 2 };

// One work item (a tile, or a chunk of a crowded tile) of one species.
template <int DIM, int ORDER, int MODE = kGpdFused>
__device__ __forceinline__ void gpd_item(const GpdArgs& A, int item_index, float4* smem4) {
    const Geo& g = A.g;
    const Ptr3<const float>& E = A.E;
    const Ptr3<const float>& B = A.B;
    const Ptr3<unsigned long long>& J = A.J;
    const P32& p = A.p;
    const Tiles& t = A.t;
    const CellDecode& dec = A.dec;
    const float k = A.k, sq = A.sq, dth0 = A.dth0, dth1 = A.dth1, dth2 = A.dth2;
    unsigned* st = A.st;

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
    const int G0 = Te[0] + 4, G1 = Te[1] + 4, G2 = (DIM == 3) ? Te[2] + 4 : 1;
    const int H0 = Te[0] + 5, H1 = Te[1] + 5, H2 = (DIM == 3) ? Te[2] + 5 : 1;
    const int fsz = G0 * G1 * G2, jsz = H0 * H1 * H2;
    const int n4 = (3 * jsz + 3) >> 2;     // the J boxes in groups of 4 nodes
    float* sF = reinterpret_cast<float*>(smem4);
    long long* sJ = reinterpret_cast<long long*>(sF + ((6 * fsz + 3) & ~3));
    int* sR = reinterpret_cast<int*>(sJ + 4 * n4);
    longlong2* sJ2 = reinterpret_cast<longlong2*>(sJ);
    int4* sR4 = reinterpret_cast<int4*>(sR);
    // 3D deposit staging: same-stencil slots, the ring, then the counters:
    // [round & 1] same-stencil moves of the round, [2] moves ever queued
    int* sSt = sR + 4 * n4;
    int* sRing = sSt + kStageWords * kGpdThreads;
    int* sCnt = sRing + kStageWords * kRing;

    for (int idx = threadIdx.x; MODE != kGpdFieldsIn && idx < 6 * fsz; idx += blockDim.x) {
        const int c = fdiv(idx, t.fF), r = idx - c * fsz;
        const int q = fdiv(r, t.fG0), lx = r - q * G0;
        const int lz = (DIM == 3) ? fdiv(q, t.fG1) : 0, ly = q - lz * G1;
        const long long m = fidx_near(g, t0[0] - 2 + lx, t0[1] - 2 + ly, DIM == 3 ? t0[2] - 2 + lz : 0);
        const float* src = c == 0 ? E.p[0] : c == 1 ? E.p[1] : c == 2 ? E.p[2]
                         : c == 3 ? B.p[0] : c == 4 ? B.p[1] : B.p[2];
        sF[idx] = (m < 0) ? 0.0f : src[m];
    }
    for (int q = threadIdx.x; q < n4; q += blockDim.x) {
        sJ2[2 * q] = make_longlong2(0, 0);
        sJ2[2 * q + 1] = make_longlong2(0, 0);
        sR4[q] = make_int4(0, 0, 0, 0);
    }
    if (DIM == 3 && threadIdx.x < 4) sCnt[threadIdx.x] = 0;
    __syncthreads();

    const float dth[3] = {dth0, dth1, dth2};
    const Acc32<DIM == 2> acc{sR};
    // adds the int32 box into the int64 box, four nodes at a time, and clears
    // it (callers place the barriers)
    auto fold = [&]() {
        for (int q = threadIdx.x; q < n4; q += kGpdThreads) {
            const int4 v = sR4[q];
            if ((v.x | v.y | v.z | v.w) != 0) {
                longlong2 a = sJ2[2 * q], b = sJ2[2 * q + 1];
                a.x += v.x; a.y += v.y; b.x += v.z; b.y += v.w;
                sJ2[2 * q] = a; sJ2[2 * q + 1] = b;
                sR4[q] = make_int4(0, 0, 0, 0);
            }
        }
    };
    // 3D (block-uniform): moves deposited since the last fold, moves queued in
    // and taken from the ring
    int moves = 0, queued = 0, consumed = 0;
    const int nround = (end - beg + kGpdThreads - 1) / kGpdThreads;
    // 2D: this thread's particle of round r, prefetched into buffer r & 1
    int* sPf = sR + 4 * n4;
    auto prefetch = [&](int r) {
        const int ii = beg + r * kGpdThreads + threadIdx.x;
        if (r < nround && ii < end) {
            int* b = sPf + (r & 1) * kPrefWords * kGpdThreads + threadIdx.x;
            cp_async4(b, p.cell + ii);
            cp_async4(b + 1 * kGpdThreads, p.off[0] + ii);
            cp_async4(b + 2 * kGpdThreads, p.off[1] + ii);
            cp_async4(b + 3 * kGpdThreads, p.u[0] + ii);
            cp_async4(b + 4 * kGpdThreads, p.u[1] + ii);
            cp_async4(b + 5 * kGpdThreads, p.u[2] + ii);
            cp_async4(b + 6 * kGpdThreads, p.w + ii);
        }
        cp_async_commit();
    };
    if constexpr (DIM == 2) prefetch(0);
    for (int rnd = 0; rnd < nround; ++rnd) {
        const int i = beg + rnd * kGpdThreads + threadIdx.x;
        int cell = -1;
        // off0, off1, u0, u1, u2, then 2D: w / 3D: off2 (3D weight in pf3w)
        float pf[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, pf3w = 0.0f;
        if constexpr (DIM == 2) {
            cp_async_wait_all();
            const int* b = sPf + (rnd & 1) * kPrefWords * kGpdThreads + threadIdx.x;
            if (i < end) {
                cell = b[0];
#pragma unroll
                for (int k2 = 0; k2 < 6; ++k2) pf[k2] = __int_as_float(b[(1 + k2) * kGpdThreads]);
            }
            prefetch(rnd + 1);
        } else {
            // 3D: all of the particle's loads in flight together
            if (i < end) {
                cell = p.cell[i];
                pf[0] = p.off[0][i]; pf[1] = p.off[1][i]; pf[5] = p.off[2][i];
                pf[2] = p.u[0][i]; pf[3] = p.u[1][i]; pf[4] = p.u[2][i];
                pf3w = p.w[i];
            }
        }
        int cell_out = cell;      // the particle's cell after this round (-1: removed)
        // 3D: the move this particle deposits (if dep), staged below
        bool dep = false, same = false;
        int mlc[3] = {0, 0, 0}, mce[3] = {0, 0, 0};
        float mf0[3] = {0.0f, 0.0f, 0.0f}, mf1[3] = {0.0f, 0.0f, 0.0f}, ms = 0.0f;
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
                if (MODE == kGpdFused) {
                    // beyond the tile's drift margin: queued for the global-memory
                    // path, which also counts its new tile key
                    t.esc[atomicAdd(t.nesc, 1)] = i;
                } else {
                    // the unfused stages run on freshly sorted particles only
                    set_status(st, LPIC_ST_HALO);
                }
                cell_out = -1;
            } else {
                float f[3], ux, uy, uz, w;
                if constexpr (DIM == 2) {
                    f[0] = pf[0]; f[1] = pf[1]; f[2] = 0.0f;
                    ux = pf[2]; uy = pf[3]; uz = pf[4]; w = pf[5];
                } else {
                    f[0] = pf[0]; f[1] = pf[1]; f[2] = pf[5];
                    ux = pf[2]; uy = pf[3]; uz = pf[4]; w = pf3w;
                }

                // gather at x^{n+1/2} from the shared-memory halo
                const NodeW<ORDER> nx_(lc[0], f[0]), ny_(lc[1], f[1]), nz_(lc[2], f[2]);
                const HalfW<ORDER> hx_(lc[0], f[0]), hy_(lc[1], f[1]), hz_(lc[2], f[2]);
                float fld[6];
                if constexpr (MODE == kGpdFieldsIn) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) fld[c] = A.fields[c * A.fcap + i];
                } else {
                    gather32<DIM, ORDER>(LoadShared<DIM>{sF, fsz, G0, G1}, nx_, ny_, nz_, hx_, hy_, hz_, fld);
                }
                if constexpr (MODE == kGpdGather) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) A.fields[c * A.fcap + i] = fld[c];
                } else {
                boris_f32(ux, uy, uz, k, fld[0], fld[1], fld[2], fld[3], fld[4], fld[5]);
                if (!isfinite(ux) || !isfinite(uy) || !isfinite(uz)) {
                    set_status(st, LPIC_ST_NAN);
                    p.cell[i] = -1;
                    cell_out = -1;
                } else {
                    const float ig = rsqrtf(1.0f + ux * ux + uy * uy + uz * uz);
                    const float uu[3] = {ux, uy, uz};
                    int ce[3] = {0, 0, 0};
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
                        cell_out = -1;
                    } else {
                        same = same_stencils<DIM, ORDER>(lc, f, ce, fe);
                        if constexpr (DIM == 2) {
                            // the stencil-sized window when every converged lane allows it
                            if (__all_sync(__activemask(), same))
                                deposit2d_same<ORDER>(acc, jsz, H0, lc, f, ce, fe, sq * w, uz * ig);
                            else
                                deposit2d<ORDER>(acc, jsz, H0, lc, f, ce, fe, sq * w, uz * ig);
                        } else {
                            dep = true;
#pragma unroll
                            for (int d = 0; d < 3; ++d) { mlc[d] = lc[d]; mce[d] = ce[d]; mf0[d] = f[d]; mf1[d] = fe[d]; }
                            ms = sq * w;
                        }
                        // store x^{n+3/2} and u^{n+1}
                        int ng[3];
#pragma unroll
                        for (int d = 0; d < 3; ++d) ng[d] = (d < DIM) ? t0[d] + ce[d] : 0;
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
            if (key >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
                atomicAdd(t.next_count + key, __popc(peers));
        }
        if constexpr (DIM == 3) {
            // 3D: same-stencil moves go to this round's slots; the others to
            // the ring, deposited 256 at a time, so that each warp runs one
            // form of the deposit with full lanes (most particles keep their
            // stencil, but few warps are uniform; the order of the integer
            // sums does not matter)
            int* cf = sCnt + (rnd & 1);
            const unsigned lane = threadIdx.x & 31u;
            const unsigned mfast = __ballot_sync(0xffffffffu, dep && same);
            const unsigned mgen = __ballot_sync(0xffffffffu, dep && !same);
            int bf = 0, bg = 0;
            if (lane == 0) {
                if (mfast) bf = atomicAdd(cf, __popc(mfast));
                if (mgen) bg = atomicAdd(sCnt + 2, __popc(mgen));
            }
            bf = __shfl_sync(0xffffffffu, bf, 0);
            bg = __shfl_sync(0xffffffffu, bg, 0);
            if (dep) {
                const unsigned below = (1u << lane) - 1u;
                if (same) stage_move(sSt + bf + __popc(mfast & below), kGpdThreads, mlc, mce, mf0, mf1, ms);
                else      stage_move(sRing + ((bg + __popc(mgen & below)) & (kRing - 1)), kRing, mlc, mce, mf0,
                                     mf1, ms);
            }
            __syncthreads();
            const int nf = *cf;
            queued = sCnt[2];
            // the other parity's counter was last read before this barrier
            if (threadIdx.x == 0) sCnt[(rnd + 1) & 1] = 0;
            if (moves + nf > kGpdThreads * t.R) { fold(); moves = 0; __syncthreads(); }
            if ((int)threadIdx.x < nf)
                deposit_staged3d<ORDER, true>(acc, jsz, H0, H1, sSt + threadIdx.x, kGpdThreads);
            moves += nf;
            if (queued - consumed >= kGpdThreads) {
                if (moves + kGpdThreads > kGpdThreads * t.R) {
                    __syncthreads(); fold(); moves = 0; __syncthreads();
                }
                deposit_staged3d<ORDER, false>(acc, jsz, H0, H1,
                                               sRing + ((consumed + threadIdx.x) & (kRing - 1)), kRing);
                consumed += kGpdThreads;
                moves += kGpdThreads;
            }
            // the staging slots are rewritten by the next round
            __syncthreads();
        } else {
            // 2D: every R rounds (and at the end) fold the int32 box into the
            // int64 box (block-uniform condition)
            if ((rnd + 1) % t.R == 0 || rnd + 1 == nround) { __syncthreads(); fold(); __syncthreads(); }
        }
    }
    if constexpr (DIM == 3) {
        // the moves still in the ring, then the last fold
        const int rest = queued - consumed;
        if (rest > 0) {
            if (moves + rest > kGpdThreads * t.R) { fold(); __syncthreads(); }
            if ((int)threadIdx.x < rest)
                deposit_staged3d<ORDER, false>(acc, jsz, H0, H1,
                                               sRing + ((consumed + threadIdx.x) & (kRing - 1)), kRing);
            __syncthreads();
        }
        fold();
        __syncthreads();
    }

    // one flush of the item's current to the global int64 arrays
    bool outside = false;
    for (int idx = threadIdx.x; idx < 3 * jsz; idx += blockDim.x) {
        const long long v = sJ[idx];
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
    __device__ inline void operator()(int idx, int v) const {
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
                                     {gc[0], gc[1], gc[2]}, &outside};
            gather32<DIM, ORDER>(ld, nx_, ny_, nz_, hx_, hy_, hz_, fld);
            if (outside) set_status(st, LPIC_ST_OUTSIDE);
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
