// lpic_fp32.cuh -- FP32 particle path with an int64 fixed-point current.
//
// Particles: int32 linear cell + FP32 in-cell offsets (f in [0, 1)), FP32 u
// and w, stored leapfrog-style (x^{n+1/2}, u^n).  They are sorted by cell tile
// before the push, so one thread block owns one tile: it stages the tile's
// E/B halo in shared memory, pushes the tile's particles (gather, Boris,
// straight path x^{n+1/2} -> x^{n+3/2}, Sec. 3.1) and accumulates their
// Esirkepov current in an int64 shared-memory tile that is flushed once to
// the global int64 J with integer atomics.  Integer sums do not depend on
// the order of the additions, so the result is bitwise deterministic.
//
// Exact charge conservation in integers.  The unit of charge is 2^-F.  A
// particle of charge s = 2^F q w carries the integer charge S = rint(s); on
// its stencil node (a, b[, c]) it puts Q = rint(s Sx Sy [Sz]) and the node
// at index 1 of its own stencil takes the remainder S - sum Q, so every
// particle's integer charge is the same at every position.  Weights are
// computed from the stored (cell, offset) pair with explicitly rounded
// arithmetic, so the charge at the end of one step's path is bit-identical
// to the charge at the start of the next step's path.  The Esirkepov weights
// W_d (Sec. 3.1) are quantised with closures that make the integer current
// a valid flow for the integer charge change dQ = Q1 - Q0:
//   2D: W_x = rint(s DS_x A_y) except the last column (b), fixed so that
//       sum_b W_x(a, .) = sum_b dQ(a, .), and the last row (a), fixed so that
//       sum_a W_x(., b) = 0; W_y = dQ - W_x.
//   3D: the same construction on the column sums over c (targets X, Y for
//       sum_c W_x, sum_c W_y), then W_x, W_y per node with closures along c
//       (to X, Y) and along a / b (to 0); W_z = dQ - W_x - W_y.
// J_d is then the running sum of -W_d along d and satisfies, node by node,
// J_d(i+1/2) - J_d(i-1/2) summed over d = -(Q1 - Q0) exactly.  Per-particle
// integers stay below 2^31 (F is chosen so that S <= 2^29).
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
    const int* start;    // ntiles + 1 prefix offsets (after the sort)
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

__device__ inline void sj_add(long long* sJ, int idx, int v) {
    if (v != 0) atomicAdd(reinterpret_cast<unsigned long long*>(sJ + idx),
                          static_cast<unsigned long long>(static_cast<long long>(v)));
}

// ----------------------------------------------------------- 2D deposit
// lc/f: start (cell relative to the J box origin minus 2, offset); ce/fe: end.
// sJ holds three components of H0 x H1 int64, node (a, b) of component c at
// c * jsz + (b + 2) * H0 + (a + 2) with a, b relative to the tile origin.
template <int ORDER>
__device__ inline void deposit2d(long long* sJ, int jsz, int H0, const int* lc, const float* f,
                                 const int* ce, const float* fe, float s, float vz) {
    constexpr int WN = ORDER + 2;
    const NodeW<ORDER> ax(lc[0], f[0]), ay(lc[1], f[1]), bx(ce[0], fe[0]), by(ce[1], fe[1]);
    const int basex = min(ax.base, bx.base), basey = min(ay.base, by.base);
    const int o0x = ax.base - basex, o1x = bx.base - basex;
    const int o0y = ay.base - basey, o1y = by.base - basey;
    float S0x[WN], S1x[WN], S0y[WN], S1y[WN];
    place32<ORDER>(S0x, ax, o0x); place32<ORDER>(S1x, bx, o1x);
    place32<ORDER>(S0y, ay, o0y); place32<ORDER>(S1y, by, o1y);
    const int sint = __float2int_rn(s);
    int dQ[WN][WN];
    int sum0 = 0, sum1 = 0;
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        const float x0 = __fmul_rn(s, S0x[a]), x1 = __fmul_rn(s, S1x[a]);
#pragma unroll
        for (int b = 0; b < WN; ++b) {
            const int q0 = __float2int_rn(__fmul_rn(x0, S0y[b]));
            const int q1 = __float2int_rn(__fmul_rn(x1, S1y[b]));
            dQ[a][b] = q1 - q0; sum0 += q0; sum1 += q1;
        }
    }
    const int d0 = sint - sum0, d1 = sint - sum1;
#pragma unroll
    for (int a = 0; a < WN; ++a)
#pragma unroll
        for (int b = 0; b < WN; ++b)
            dQ[a][b] += ((a == o1x + 1 && b == o1y + 1) ? d1 : 0) - ((a == o0x + 1 && b == o0y + 1) ? d0 : 0);

    float DSx[WN], DSy[WN], Ax[WN], Ay[WN];
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        DSx[a] = S1x[a] - S0x[a]; DSy[a] = S1y[a] - S0y[a];
        Ax[a] = 0.5f * (S0x[a] + S1x[a]); Ay[a] = 0.5f * (S0y[a] + S1y[a]);
    }
    // W_x with closures; W_y = dQ - W_x
    int Wx[WN][WN];
#pragma unroll
    for (int a = 0; a < WN - 1; ++a) {
        int row = 0, M = 0;
#pragma unroll
        for (int b = 0; b < WN; ++b) M += dQ[a][b];
        const float sdx = s * DSx[a];
#pragma unroll
        for (int b = 0; b < WN - 1; ++b) { Wx[a][b] = __float2int_rn(sdx * Ay[b]); row += Wx[a][b]; }
        Wx[a][WN - 1] = M - row;
    }
#pragma unroll
    for (int b = 0; b < WN; ++b) {
        int col = 0;
#pragma unroll
        for (int a = 0; a < WN - 1; ++a) col += Wx[a][b];
        Wx[WN - 1][b] = -col;
    }
    // J_x: running sum along a; J_y: running sum along b
#pragma unroll
    for (int b = 0; b < WN; ++b) {
        int run = 0;
#pragma unroll
        for (int a = 0; a < WN - 1; ++a) {
            run -= Wx[a][b];
            sj_add(sJ, (basey + b + 2) * H0 + (basex + a + 2), run);
        }
    }
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        int run = 0;
#pragma unroll
        for (int b = 0; b < WN - 1; ++b) {
            run -= dQ[a][b] - Wx[a][b];
            sj_add(sJ, jsz + (basey + b + 2) * H0 + (basex + a + 2), run);
        }
    }
    // J_z: s v_z W_z, W_z = A_x A_y + DS_x DS_y / 12 (needs no closure in 2D)
    const float svz = s * vz;
#pragma unroll
    for (int a = 0; a < WN; ++a)
#pragma unroll
        for (int b = 0; b < WN; ++b) {
            const float wz = Ax[a] * Ay[b] + DSx[a] * DSy[b] * (1.0f / 12.0f);
            sj_add(sJ, 2 * jsz + (basey + b + 2) * H0 + (basex + a + 2), __float2int_rn(svz * wz));
        }
}

// ----------------------------------------------------------- 3D deposit
template <int ORDER>
__device__ inline void deposit3d(long long* sJ, int jsz, int H0, int H1, const int* lc,
                                 const float* f, const int* ce, const float* fe, float s) {
    constexpr int WN = ORDER + 2;
    constexpr int L = WN - 1;
    const NodeW<ORDER> a0(lc[0], f[0]), a1(lc[1], f[1]), a2(lc[2], f[2]);
    const NodeW<ORDER> b0(ce[0], fe[0]), b1(ce[1], fe[1]), b2(ce[2], fe[2]);
    const int bs0 = min(a0.base, b0.base), bs1 = min(a1.base, b1.base), bs2 = min(a2.base, b2.base);
    float S0x[WN], S1x[WN], S0y[WN], S1y[WN], S0z[WN], S1z[WN];
    place32<ORDER>(S0x, a0, a0.base - bs0); place32<ORDER>(S1x, b0, b0.base - bs0);
    place32<ORDER>(S0y, a1, a1.base - bs1); place32<ORDER>(S1y, b1, b1.base - bs1);
    place32<ORDER>(S0z, a2, a2.base - bs2); place32<ORDER>(S1z, b2, b2.base - bs2);
    const int c0x = a0.base - bs0 + 1, c0y = a1.base - bs1 + 1, c0z = a2.base - bs2 + 1;
    const int c1x = b0.base - bs0 + 1, c1y = b1.base - bs1 + 1, c1z = b2.base - bs2 + 1;
    const int sint = __float2int_rn(s);

    // integer charge change dQ with canonical remainders
    int R[WN][WN][WN];
    int sum0 = 0, sum1 = 0;
    float sx0[WN], sx1[WN];
#pragma unroll
    for (int a = 0; a < WN; ++a) { sx0[a] = __fmul_rn(s, S0x[a]); sx1[a] = __fmul_rn(s, S1x[a]); }
#pragma unroll
    for (int b = 0; b < WN; ++b)
#pragma unroll
        for (int c = 0; c < WN; ++c) {
            const float yz0 = __fmul_rn(S0y[b], S0z[c]), yz1 = __fmul_rn(S1y[b], S1z[c]);
#pragma unroll
            for (int a = 0; a < WN; ++a) {
                const int q0 = __float2int_rn(__fmul_rn(sx0[a], yz0));
                const int q1 = __float2int_rn(__fmul_rn(sx1[a], yz1));
                R[a][b][c] = q1 - q0; sum0 += q0; sum1 += q1;
            }
        }
    const int d0 = sint - sum0, d1 = sint - sum1;
#pragma unroll
    for (int a = 0; a < WN; ++a)
#pragma unroll
        for (int b = 0; b < WN; ++b)
#pragma unroll
            for (int c = 0; c < WN; ++c)
                R[a][b][c] += ((a == c1x && b == c1y && c == c1z) ? d1 : 0)
                            - ((a == c0x && b == c0y && c == c0z) ? d0 : 0);

    float DSx[WN], DSy[WN], DSz[WN], Ay[WN], Az[WN], Ax[WN];
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        DSx[a] = S1x[a] - S0x[a]; DSy[a] = S1y[a] - S0y[a]; DSz[a] = S1z[a] - S0z[a];
        Ax[a] = 0.5f * (S0x[a] + S1x[a]); Ay[a] = 0.5f * (S0y[a] + S1y[a]);
        Az[a] = 0.5f * (S0z[a] + S1z[a]);
    }
    // column sums over c: Z(a, b); x-marginal M(a)
    int Z[WN][WN], M[WN];
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        M[a] = 0;
#pragma unroll
        for (int b = 0; b < WN; ++b) {
            int z = 0;
#pragma unroll
            for (int c = 0; c < WN; ++c) z += R[a][b][c];
            Z[a][b] = z; M[a] += z;
        }
    }
    // level 2: X(a, b) = target of sum_c W_x; Y = Z - X
    int X[WN][WN];
#pragma unroll
    for (int a = 0; a < L; ++a) {
        int row = 0;
        const float sdx = s * DSx[a];
#pragma unroll
        for (int b = 0; b < L; ++b) { X[a][b] = __float2int_rn(sdx * Ay[b]); row += X[a][b]; }
        X[a][L] = M[a] - row;
    }
#pragma unroll
    for (int b = 0; b < WN; ++b) {
        int col = 0;
#pragma unroll
        for (int a = 0; a < L; ++a) col += X[a][b];
        X[L][b] = -col;
    }
    // level 3, x: W_x(a, b, c) = s DS_x(a) (A_y A_z + DS_y DS_z / 12)
#pragma unroll
    for (int b = 0; b < WN; ++b) {
        int cs[WN];
#pragma unroll
        for (int a = 0; a < WN; ++a) cs[a] = 0;
#pragma unroll
        for (int c = 0; c < WN; ++c) {
            const float kyz = Ay[b] * Az[c] + DSy[b] * DSz[c] * (1.0f / 12.0f);
            int colsum = 0, run = 0;
#pragma unroll
            for (int a = 0; a < L; ++a) {
                const int v = (c < L) ? __float2int_rn(s * DSx[a] * kyz) : X[a][b] - cs[a];
                cs[a] += v; colsum += v;
                R[a][b][c] -= v;
                run -= v;
                sj_add(sJ, ((bs2 + c + 2) * H1 + (bs1 + b + 2)) * H0 + (bs0 + a + 2), run);
            }
            R[L][b][c] += colsum;      // W_x(L, b, c) = -colsum
        }
    }
    // level 3, y: W_y(a, b, c) = s DS_y(b) (A_x A_z + DS_x DS_z / 12), sum_c -> Y = Z - X
#pragma unroll
    for (int a = 0; a < WN; ++a) {
        int cs[WN];
#pragma unroll
        for (int b = 0; b < WN; ++b) cs[b] = 0;
#pragma unroll
        for (int c = 0; c < WN; ++c) {
            const float kxz = Ax[a] * Az[c] + DSx[a] * DSz[c] * (1.0f / 12.0f);
            int colsum = 0, run = 0;
#pragma unroll
            for (int b = 0; b < L; ++b) {
                const int v = (c < L) ? __float2int_rn(s * DSy[b] * kxz) : (Z[a][b] - X[a][b]) - cs[b];
                cs[b] += v; colsum += v;
                R[a][b][c] -= v;
                run -= v;
                sj_add(sJ, jsz + ((bs2 + c + 2) * H1 + (bs1 + b + 2)) * H0 + (bs0 + a + 2), run);
            }
            R[a][L][c] += colsum;
        }
    }
    // z: W_z = dQ - W_x - W_y (what is left in R); J_z is its running sum along c
#pragma unroll
    for (int a = 0; a < WN; ++a)
#pragma unroll
        for (int b = 0; b < WN; ++b) {
            int run = 0;
#pragma unroll
            for (int c = 0; c < L; ++c) {
                run -= R[a][b][c];
                sj_add(sJ, 2 * jsz + ((bs2 + c + 2) * H1 + (bs1 + b + 2)) * H0 + (bs0 + a + 2), run);
            }
        }
}

// Integer charge of one particle (the Q of the deposit) added to rho_int.
template <int DIM, int ORDER>
__device__ inline void charge_int(unsigned long long* rho, const Geo& g, const int* gc,
                                  const float* f, float s) {
    const NodeW<ORDER> wx(gc[0], f[0]), wy(gc[1], f[1]), wz(DIM == 3 ? gc[2] : 0, DIM == 3 ? f[2] : 0.0f);
    const int sint = __float2int_rn(s);
    int sum = 0;
    int q[ORDER + 1][ORDER + 1][ORDER + 1];
#pragma unroll
    for (int a = 0; a <= ORDER; ++a) {
        const float sx = __fmul_rn(s, wx.w[a]);
#pragma unroll
        for (int b = 0; b <= ORDER; ++b)
#pragma unroll
            for (int c = 0; c <= ORDER; ++c) {
                int v = 0;
                if (DIM == 3) v = __float2int_rn(__fmul_rn(sx, __fmul_rn(wy.w[b], wz.w[c])));
                else if (c == 0) v = __float2int_rn(__fmul_rn(sx, wy.w[b]));
                q[a][b][c] = v; sum += v;
            }
    }
    q[1][1][DIM == 3 ? 1 : 0] += sint - sum;
#pragma unroll
    for (int a = 0; a <= ORDER; ++a)
#pragma unroll
        for (int b = 0; b <= ORDER; ++b)
#pragma unroll
            for (int c = 0; c <= (DIM == 3 ? ORDER : 0); ++c) {
                const long long m = fidx(g, wx.base + a, wy.base + b, DIM == 3 ? wz.base + c : 0);
                if (m >= 0 && q[a][b][c] != 0)
                    atomicAdd(rho + m, static_cast<unsigned long long>(static_cast<long long>(q[a][b][c])));
            }
}

// ----------------------------------------------------------- the tile kernel
template <int DIM, int ORDER>
__global__ void __launch_bounds__(256) k_gpd32(Geo g, Ptr3<const float> E, Ptr3<const float> B,
                                               Ptr3<unsigned long long> J, P32 p, Tiles t,
                                               float k, float sq, float dth0, float dth1,
                                               float dth2, unsigned* st) {
    const int tile = blockIdx.x;
    const int beg = t.start[tile], end = t.start[tile + 1];
    if (beg == end) return;
    const int t0[3] = {(tile % t.nt[0]) * t.T[0], ((tile / t.nt[0]) % t.nt[1]) * t.T[1],
                       DIM == 3 ? (tile / (t.nt[0] * t.nt[1])) * t.T[2] : 0};
    const int G0 = t.T[0] + 4, G1 = t.T[1] + 4, G2 = (DIM == 3) ? t.T[2] + 4 : 1;
    const int H0 = t.T[0] + 5, H1 = t.T[1] + 5, H2 = (DIM == 3) ? t.T[2] + 5 : 1;
    const int fsz = G0 * G1 * G2, jsz = H0 * H1 * H2;
    extern __shared__ float4 smem4[];
    float* sF = reinterpret_cast<float*>(smem4);
    long long* sJ = reinterpret_cast<long long*>(sF + ((6 * fsz + 3) & ~3));

    for (int idx = threadIdx.x; idx < 6 * fsz; idx += blockDim.x) {
        const int c = idx / fsz, r = idx - c * fsz;
        const int lx = r % G0, ly = (r / G0) % G1, lz = r / (G0 * G1);
        const long long m = fidx(g, t0[0] - 2 + lx, t0[1] - 2 + ly, DIM == 3 ? t0[2] - 2 + lz : 0);
        sF[idx] = (m < 0) ? 0.0f : (c < 3 ? E.p[c][m] : B.p[c - 3][m]);
    }
    for (int idx = threadIdx.x; idx < 3 * jsz; idx += blockDim.x) sJ[idx] = 0;
    __syncthreads();

    const float dth[3] = {dth0, dth1, dth2};
    for (int i = beg + threadIdx.x; i < end; i += blockDim.x) {
        const int cell = p.cell[i];
        if (cell < 0) continue;
        int gc[3];
        gc[0] = cell % g.nx;
        const int rr = cell / g.nx;
        gc[1] = rr % g.ny;
        gc[2] = (DIM == 3) ? rr / g.ny : 0;
        int lc[3] = {gc[0] - t0[0], gc[1] - t0[1], DIM == 3 ? gc[2] - t0[2] : 0};
        bool inside = true;
#pragma unroll
        for (int d = 0; d < DIM; ++d) inside &= (lc[d] >= 0 && lc[d] < t.T[d]);
        if (!inside) { set_status(st, LPIC_ST_HALO); continue; }
        float f[3] = {p.off[0][i], p.off[1][i], DIM == 3 ? p.off[2][i] : 0.0f};
        float ux = p.u[0][i], uy = p.u[1][i], uz = p.u[2][i];
        const float w = p.w[i];

        // gather at x^{n+1/2} from the shared-memory halo
        const NodeW<ORDER> nx_(lc[0], f[0]), ny_(lc[1], f[1]), nz_(lc[2], f[2]);
        const HalfW<ORDER> hx_(lc[0], f[0]), hy_(lc[1], f[1]), hz_(lc[2], f[2]);
        float fld[6];
#pragma unroll
        for (int comp = 0; comp < 6; ++comp) {
            // staggering: E_x (h,n,n) E_y (n,h,n) E_z (n,n,h) B_x (n,h,h) B_y (h,n,h) B_z (h,h,n)
            const bool hx = (comp == 0 || comp == 4 || comp == 5);
            const bool hy = (comp == 1 || comp == 3 || comp == 5);
            const bool hz = (comp == 2 || comp == 3 || comp == 4);
            const int bx = hx ? hx_.base : nx_.base, by = hy ? hy_.base : ny_.base;
            const int bz = (DIM == 3) ? (hz ? hz_.base : nz_.base) : -2;
            const float* F = sF + comp * fsz;
            float acc = 0.0f;
#pragma unroll
            for (int c = 0; c < (DIM == 3 ? ORDER + 1 : 1); ++c) {
                const float wzv = (DIM == 3) ? (hz ? hz_.w[c] : nz_.w[c]) : 1.0f;
#pragma unroll
                for (int b = 0; b <= ORDER; ++b) {
                    const float wyz = (hy ? hy_.w[b] : ny_.w[b]) * wzv;
                    const float* row = F + ((bz + c + 2) * G1 + (by + b + 2)) * G0 + (bx + 2);
#pragma unroll
                    for (int a = 0; a <= ORDER; ++a) acc += row[a] * ((hx ? hx_.w[a] : nx_.w[a]) * wyz);
                }
            }
            fld[comp] = acc;
        }
        boris<float>(ux, uy, uz, k, fld[0], fld[1], fld[2], fld[3], fld[4], fld[5]);
        if (!isfinite(ux) || !isfinite(uy) || !isfinite(uz)) {
            set_status(st, LPIC_ST_NAN); p.cell[i] = -1; continue;
        }
        const float ig = 1.0f / sqrtf(1.0f + ux * ux + uy * uy + uz * uz);
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
        if (cfl) { set_status(st, LPIC_ST_CFL); p.cell[i] = -1; continue; }

        const float s = sq * w;
        if (DIM == 3) deposit3d<ORDER>(sJ, jsz, H0, H1, lc, f, ce, fe, s);
        else          deposit2d<ORDER>(sJ, jsz, H0, lc, f, ce, fe, s, uz * ig);

        // store x^{n+3/2} and u^{n+1}
        int ng[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) ng[d] = (d < DIM) ? t0[d] + ce[d] : 0;
        bool dead = false;
        if (g.absorb) dead = (ng[0] < 2 || ng[0] >= g.nx - 2);
        else ng[0] = wrapi(ng[0], g.nx);
        ng[1] = wrapi(ng[1], g.ny);
        if (DIM == 3) ng[2] = wrapi(ng[2], g.nz);
        p.cell[i] = dead ? -1 : (ng[2] * g.ny + ng[1]) * g.nx + ng[0];
#pragma unroll
        for (int d = 0; d < DIM; ++d) p.off[d][i] = fe[d];
        p.u[0][i] = ux; p.u[1][i] = uy; p.u[2][i] = uz;
    }
    __syncthreads();

    // one flush of the tile's current to the global int64 arrays
    bool outside = false;
    for (int idx = threadIdx.x; idx < 3 * jsz; idx += blockDim.x) {
        const long long v = sJ[idx];
        if (v == 0) continue;
        const int c = idx / jsz, r = idx - c * jsz;
        const int lx = r % H0, ly = (r / H0) % H1, lz = r / (H0 * H1);
        const long long m = fidx(g, t0[0] - 2 + lx, t0[1] - 2 + ly, DIM == 3 ? t0[2] - 2 + lz : 0);
        if (m < 0) { outside = true; continue; }
        atomicAdd(J.p[c] + m, static_cast<unsigned long long>(v));
    }
    if (outside) set_status(st, LPIC_ST_OUTSIDE);
}

// x^0 -> x^{1/2}: offsets advance by (dt/2) v / h with carries into the cell.
template <int DIM>
__global__ void k_advance32(Geo g, P32 p, float frac, float dth0, float dth1, float dth2) {
    const int n = *p.n;
    const float dth[3] = {dth0, dth1, dth2};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int cell = p.cell[i];
        if (cell < 0) continue;
        int gc[3];
        gc[0] = cell % g.nx;
        const int rr = cell / g.nx;
        gc[1] = rr % g.ny;
        gc[2] = (DIM == 3) ? rr / g.ny : 0;
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
        p.cell[i] = (gc[0] < 0 || gc[0] >= g.nx) ? -1 : (gc[2] * g.ny + gc[1]) * g.nx + gc[0];
    }
}

template <int DIM, int ORDER>
__global__ void k_charge32(Geo g, P32 p, float sq, unsigned long long* rho) {
    const int n = *p.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int cell = p.cell[i];
        if (cell < 0) continue;
        int gc[3];
        gc[0] = cell % g.nx;
        const int rr = cell / g.nx;
        gc[1] = rr % g.ny;
        gc[2] = (DIM == 3) ? rr / g.ny : 0;
        const float f[3] = {p.off[0][i], p.off[1][i], DIM == 3 ? p.off[2][i] : 0.0f};
        charge_int<DIM, ORDER>(rho, g, gc, f, sq * p.w[i]);
    }
}

}  // namespace lpic
