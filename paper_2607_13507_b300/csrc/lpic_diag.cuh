// lpic_diag.cuh -- FP64 diagnostics (Sec. 4.1 energy history): kinetic and
// field energy, total charge, charge density, and integer-time positions.
#pragma once
#include "lpic_common.cuh"
#include "lpic_fp32.cuh"
#include "lpic_fp64.cuh"

namespace lpic {

// acc[0] += sum w m (gamma - 1), acc[1] += sum q w, cnt += alive
__device__ inline void block_add3(double a, double b, long long c, double* acc, unsigned long long* cnt) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc + 0, a);
        atomicAdd(acc + 1, b);
        atomicAdd(cnt, (unsigned long long)c);
    }
}

__global__ void k_diag_p32(P32 p, double q, double m, double* acc, unsigned long long* cnt) {
    const int n = *p.n;
    double ek = 0.0, qt = 0.0;
    long long c = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (p.cell[i] < 0) continue;
        const double ux = p.u[0][i], uy = p.u[1][i], uz = p.u[2][i], w = p.w[i];
        // a massless particle carries energy |u| (m c^2 units of the unit mass)
        ek += m == 0.0 ? w * sqrt(ux * ux + uy * uy + uz * uz)
                       : w * m * (sqrt(1.0 + ux * ux + uy * uy + uz * uz) - 1.0);
        qt += q * w;
        ++c;
    }
    block_add3(ek, qt, c, acc, cnt);
}

__global__ void k_diag_p64(P64 p, double q, double m, double* acc, unsigned long long* cnt) {
    const int n = *p.n;
    double ek = 0.0, qt = 0.0;
    long long c = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double w = p.w[i];
        if (w == 0.0) continue;
        const double ux = p.u[0][i], uy = p.u[1][i], uz = p.u[2][i];
        ek += w * m * (sqrt(1.0 + ux * ux + uy * uy + uz * uz) - 1.0);
        qt += q * w;
        ++c;
    }
    block_add3(ek, qt, c, acc, cnt);
}

template <typename R>
__global__ void k_diag_field(Ptr3<const R> E, Ptr3<const R> B, long long total, double dV, double* acc) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double e = E.p[c][i], b = B.p[c][i];
            s += e * e + b * b;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc + 2, 0.5 * dV * s);
}

template <int DIM, int ORDER>
__global__ void k_charge64(Geo g, P64 p, double q, double* rho) {
    const int n = *p.n;
    const double dV = g.dx * g.dy * (DIM == 3 ? g.dz : 1.0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double w = p.w[i];
        if (w == 0.0) continue;
        const NodeWd<ORDER> wx(p.x[0][i] / g.dx), wy(p.x[1][i] / g.dy),
            wz(DIM == 3 ? p.x[2][i] / g.dz : 0.0);
        const double c0 = q * w / dV;
#pragma unroll
        for (int c = 0; c < (DIM == 3 ? ORDER + 1 : 1); ++c)
#pragma unroll
            for (int b = 0; b <= ORDER; ++b)
#pragma unroll
                for (int a = 0; a <= ORDER; ++a) {
                    const long long m = fidx(g, wx.base + a, wy.base + b, DIM == 3 ? wz.base + c : 0);
                    double v = c0 * wx.w[a] * wy.w[b];
                    if (DIM == 3) v *= wz.w[c];
                    if (m >= 0) atomicAdd(rho + m, v);
                }
    }
}

// x^n = x^{n+1/2} - (dt/2) v^n, as physical doubles out[d * cap + i].
template <int DIM>
__global__ void k_positions32(Geo g, P32 p, CellDecode dec, double* out, long long cap, bool massless) {
    const int n = *p.n;
    const double h[3] = {g.dx, g.dy, g.dz};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)cap; i += gridDim.x * blockDim.x) {
        const int cell = (i < n) ? p.cell[i] : -1;
        if (cell < 0) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) out[d * cap + i] = __longlong_as_double(0x7ff8000000000000LL);
            continue;
        }
        int gc[3];
        dec(cell, gc);
        const double ux = p.u[0][i], uy = p.u[1][i], uz = p.u[2][i];
        // gamma for a massive particle, |u| for a massless one (v = u / |u|)
        const double um2 = ux * ux + uy * uy + uz * uz;
        const double gm = massless ? (um2 > 0.0 ? sqrt(um2) : 1.0) : sqrt(1.0 + um2);
        const double u[3] = {ux, uy, uz};
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            out[d * cap + i] = ((double)gc[d] + (double)p.off[d][i]) * h[d] - 0.5 * g.dt * u[d] / gm;
    }
}

template <int DIM>
__global__ void k_positions64(Geo g, P64 p, double* out, long long cap) {
    const int n = *p.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)cap; i += gridDim.x * blockDim.x) {
        const double w = (i < n) ? p.w[i] : 0.0;
        if (w == 0.0) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) out[d * cap + i] = __longlong_as_double(0x7ff8000000000000LL);
            continue;
        }
        const double ux = p.u[0][i], uy = p.u[1][i], uz = p.u[2][i];
        const double gm = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        const double u[3] = {ux, uy, uz};
#pragma unroll
        for (int d = 0; d < DIM; ++d) out[d * cap + i] = p.x[d][i] - 0.5 * g.dt * u[d] / gm;
    }
}

// Discrete divergence of E at the integer nodes (Gauss's law, Sec. 3.2):
// sum_d (E_d(i+1/2) - E_d(i-1/2)) / h_d, periodic wrap; an absorbing x edge
// takes E_x = 0 below node 0.  out[nz][ny][fx] is overwritten.
template <typename R>
__global__ void k_div_e(Geo g, Ptr3<const R> E, double* out, FastDiv dfx, FastDiv dny) {
    const int total = g.fx * g.ny * (g.dim == 3 ? g.nz : 1);
    const double rdx = 1.0 / g.dx, rdy = 1.0 / g.dy, rdz = g.dim == 3 ? 1.0 / g.dz : 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < total; n += gridDim.x * blockDim.x) {
        const int r = fdiv(n, dfx), i = n - r * g.fx;
        const int k = fdiv(r, dny), j = r - k * g.ny;
        const int im = g.absorb ? i - 1 : (i == 0 ? g.nx - 1 : i - 1);
        const int jm = j == 0 ? g.ny - 1 : j - 1;
        const double exm = im < 0 ? 0.0 : (double)E.p[0][n - i + im];
        double v = ((double)E.p[0][n] - exm) * rdx + ((double)E.p[1][n] - (double)E.p[1][n + (jm - j) * g.fx]) * rdy;
        if (g.dim == 3) {
            const int km = k == 0 ? g.nz - 1 : k - 1;
            v += ((double)E.p[2][n] - (double)E.p[2][n + (km - k) * g.ny * g.fx]) * rdz;
        }
        out[n] = v;
    }
}

}  // namespace lpic
