// lpic_fp64.cuh -- plain FP64 particle path: one thread per particle, field
// gather from the global Yee arrays, relativistic Boris, Esirkepov deposit
// with double-precision atomics (Sec. 3.1, Algorithm 1 particle loop).
//
// Stored state at the loop boundary t_n: x^{n+1/2} and u^n.  The kernel
// gathers at x^{n+1/2}, pushes u^n -> u^{n+1}, moves the particle to
// x^{n+3/2} = x^{n+1/2} + dt v^{n+1} and deposits the current of that path.
#pragma once
#include "lpic_common.cuh"

namespace lpic {

struct P64 {
    double* x[3];
    double* u[3];
    double* w;
    int* id;
    const int* n;        // device count
};

// Sum of F over the (ORDER+1)^DIM nodes of one component's stencil.
template <int DIM, int ORDER, class WX, class WY, class WZ>
__device__ inline double gather64(const double* __restrict__ F, const Geo& g, const WX& wx,
                                  const WY& wy, const WZ& wz, bool& outside) {
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < (DIM == 3 ? ORDER + 1 : 1); ++c)
#pragma unroll
        for (int b = 0; b <= ORDER; ++b)
#pragma unroll
            for (int a = 0; a <= ORDER; ++a) {
                const long long n = fidx(g, wx.base + a, wy.base + b, DIM == 3 ? wz.base + c : 0);
                if (n < 0) { outside = true; continue; }
                double v = F[n] * wx.w[a] * wy.w[b];
                if (DIM == 3) v *= wz.w[c];
                acc += v;
            }
    return acc;
}

// Window of WN = ORDER + 2 nodes starting at `base` holding the weights of a
// stencil starting at base + off (off = 0 or 1).
template <int ORDER, typename T, class W>
__device__ inline void place(T (&S)[ORDER + 2], const W& w, int off) {
#pragma unroll
    for (int a = 0; a < ORDER + 2; ++a) {
        const T lo = (a <= ORDER) ? w.w[a < ORDER + 1 ? a : 0] : T(0);
        const T hi = (a >= 1) ? w.w[a >= 1 ? a - 1 : 0] : T(0);
        S[a] = off ? hi : lo;
    }
}

template <int DIM, int ORDER>
__global__ void __launch_bounds__(256) k_gpd64(Geo g, Ptr3<const double> E, Ptr3<const double> B,
                                               Ptr3<double> J, P64 p, double k, double q,
                                               unsigned* st) {
    constexpr int WN = ORDER + 2;
    const int n = *p.n;
    const double h[3] = {g.dx, g.dy, g.dz};
    const double L[3] = {g.nx * g.dx, g.ny * g.dy, g.nz * g.dz};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double w = p.w[i];
        if (w == 0.0) continue;
        double x[3] = {0, 0, 0}, xi[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < DIM; ++d) { x[d] = p.x[d][i]; xi[d] = x[d] / h[d]; }
        double ux = p.u[0][i], uy = p.u[1][i], uz = p.u[2][i];

        // gather at x^{n+1/2}: each component from its own staggered nodes
        const NodeWd<ORDER> ix(xi[0]), iy(xi[1]), iz(xi[2]);
        const NodeWd<ORDER> hx(xi[0] - 0.5), hy(xi[1] - 0.5), hz(xi[2] - 0.5);
        bool outside = false;
        const double ex = gather64<DIM, ORDER>(E.p[0], g, hx, iy, iz, outside);
        const double ey = gather64<DIM, ORDER>(E.p[1], g, ix, hy, iz, outside);
        const double ez = gather64<DIM, ORDER>(E.p[2], g, ix, iy, hz, outside);
        const double bx = gather64<DIM, ORDER>(B.p[0], g, ix, hy, hz, outside);
        const double by = gather64<DIM, ORDER>(B.p[1], g, hx, iy, hz, outside);
        const double bz = gather64<DIM, ORDER>(B.p[2], g, hx, hy, iz, outside);
        if (outside) set_status(st, LPIC_ST_OUTSIDE);

        boris<double>(ux, uy, uz, k, ex, ey, ez, bx, by, bz);
        if (!isfinite(ux) || !isfinite(uy) || !isfinite(uz)) { set_status(st, LPIC_ST_NAN); continue; }
        const double g1 = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        const double v[3] = {ux / g1, uy / g1, uz / g1};

        // path x^{n+1/2} -> x^{n+3/2}
        double xe[3] = {0, 0, 0}, xie[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            xe[d] = x[d] + g.dt * v[d];
            xie[d] = xe[d] / h[d];
            if (fabs(g.dt * v[d]) >= h[d]) set_status(st, LPIC_ST_CFL);
        }

        // Esirkepov weights on a WN-node window per dimension
        double S0[3][WN], DS[3][WN];
        int base[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d >= DIM) {
#pragma unroll
                for (int a = 0; a < WN; ++a) { S0[d][a] = 0.0; DS[d][a] = 0.0; }
                continue;
            }
            const NodeWd<ORDER> w0(xi[d]), w1(xie[d]);
            base[d] = min(w0.base, w1.base);
            double s0[WN], s1[WN];
            place<ORDER>(s0, w0, w0.base - base[d]);
            place<ORDER>(s1, w1, w1.base - base[d]);
#pragma unroll
            for (int a = 0; a < WN; ++a) { S0[d][a] = s0[a]; DS[d][a] = s1[a] - s0[a]; }
        }
        const double qw = q * w;
        bool out2 = false;
        if (DIM == 3) {
            const double cx = -qw / (g.dt * g.dy * g.dz);
            const double cy = -qw / (g.dt * g.dx * g.dz);
            const double cz = -qw / (g.dt * g.dx * g.dy);
#pragma unroll
            for (int b = 0; b < WN; ++b)
#pragma unroll
                for (int c = 0; c < WN; ++c) {
                    double run = 0.0;
#pragma unroll
                    for (int a = 0; a < WN - 1; ++a) {
                        run += cx * (DS[0][a] * (S0[1][b] * S0[2][c] + 0.5 * DS[1][b] * S0[2][c]
                                                 + 0.5 * S0[1][b] * DS[2][c] + DS[1][b] * DS[2][c] / 3.0));
                        if (run != 0.0) {
                            const long long m = fidx(g, base[0] + a, base[1] + b, base[2] + c);
                            if (m < 0) out2 = true; else atomicAdd(&J.p[0][m], run);
                        }
                    }
                }
#pragma unroll
            for (int a = 0; a < WN; ++a)
#pragma unroll
                for (int c = 0; c < WN; ++c) {
                    double run = 0.0;
#pragma unroll
                    for (int b = 0; b < WN - 1; ++b) {
                        run += cy * (DS[1][b] * (S0[0][a] * S0[2][c] + 0.5 * DS[0][a] * S0[2][c]
                                                 + 0.5 * S0[0][a] * DS[2][c] + DS[0][a] * DS[2][c] / 3.0));
                        if (run != 0.0) {
                            const long long m = fidx(g, base[0] + a, base[1] + b, base[2] + c);
                            if (m < 0) out2 = true; else atomicAdd(&J.p[1][m], run);
                        }
                    }
                }
#pragma unroll
            for (int a = 0; a < WN; ++a)
#pragma unroll
                for (int b = 0; b < WN; ++b) {
                    double run = 0.0;
#pragma unroll
                    for (int c = 0; c < WN - 1; ++c) {
                        run += cz * (DS[2][c] * (S0[0][a] * S0[1][b] + 0.5 * DS[0][a] * S0[1][b]
                                                 + 0.5 * S0[0][a] * DS[1][b] + DS[0][a] * DS[1][b] / 3.0));
                        if (run != 0.0) {
                            const long long m = fidx(g, base[0] + a, base[1] + b, base[2] + c);
                            if (m < 0) out2 = true; else atomicAdd(&J.p[2][m], run);
                        }
                    }
                }
        } else {
            const double cx = -qw / (g.dt * g.dy);
            const double cy = -qw / (g.dt * g.dx);
            const double cz = qw * v[2] / (g.dx * g.dy);
#pragma unroll
            for (int b = 0; b < WN; ++b) {
                double run = 0.0;
#pragma unroll
                for (int a = 0; a < WN - 1; ++a) {
                    run += cx * DS[0][a] * (S0[1][b] + 0.5 * DS[1][b]);
                    if (run != 0.0) {
                        const long long m = fidx(g, base[0] + a, base[1] + b, 0);
                        if (m < 0) out2 = true; else atomicAdd(&J.p[0][m], run);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < WN; ++a) {
                double run = 0.0;
#pragma unroll
                for (int b = 0; b < WN - 1; ++b) {
                    run += cy * DS[1][b] * (S0[0][a] + 0.5 * DS[0][a]);
                    if (run != 0.0) {
                        const long long m = fidx(g, base[0] + a, base[1] + b, 0);
                        if (m < 0) out2 = true; else atomicAdd(&J.p[1][m], run);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < WN; ++a)
#pragma unroll
                for (int b = 0; b < WN; ++b) {
                    const double Wz = S0[0][a] * S0[1][b] + 0.5 * DS[0][a] * S0[1][b]
                                    + 0.5 * S0[0][a] * DS[1][b] + DS[0][a] * DS[1][b] / 3.0;
                    if (Wz != 0.0) {
                        const long long m = fidx(g, base[0] + a, base[1] + b, 0);
                        if (m < 0) out2 = true; else atomicAdd(&J.p[2][m], cz * Wz);
                    }
                }
        }
        if (out2) set_status(st, LPIC_ST_OUTSIDE);

        // store x^{n+3/2} (wrapped) and u^{n+1}; absorbing x removes the particle
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            if (d == 0 && g.absorb) continue;
            if (xe[d] >= L[d]) xe[d] -= L[d];
            else if (xe[d] < 0.0) xe[d] += L[d];
        }
        if (g.absorb && (xe[0] < 2.0 * g.dx || xe[0] >= (g.nx - 2) * g.dx)) p.w[i] = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) p.x[d][i] = xe[d];
        p.u[0][i] = ux; p.u[1][i] = uy; p.u[2][i] = uz;
    }
}

// x += frac * dt * v (used once at add time to stagger positions by dt/2).
template <int DIM>
__global__ void k_advance64(Geo g, P64 p, double frac) {
    const int n = *p.n;
    const double L[3] = {g.nx * g.dx, g.ny * g.dy, g.nz * g.dz};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (p.w[i] == 0.0) continue;
        const double ux = p.u[0][i], uy = p.u[1][i], uz = p.u[2][i];
        const double gm = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        const double u[3] = {ux, uy, uz};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            double x = p.x[d][i] + frac * g.dt * u[d] / gm;
            if (!(d == 0 && g.absorb)) {
                if (x >= L[d]) x -= L[d]; else if (x < 0.0) x += L[d];
            }
            p.x[d][i] = x;
        }
    }
}

}  // namespace lpic
