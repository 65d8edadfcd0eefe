// lpic_field.cuh -- Yee FDTD half-step kernels (Sec. 3.2 Eq. 1-4, split in
// two dt/2 halves as in Algorithm 1) with periodic or absorbing x edges.
//
// E and B are updated in place, one thread per grid node, all three
// components: the E update reads only B (and J), the B update only E, so no
// thread reads a value another thread of the same launch writes.
// Absorbing x edges: E_y and E_z on the edge planes i = 0 and i = nx follow
// the first-order Mur condition for an outgoing wave (Mur 1981), written with
// tau = dt/2 for each half-step; at x-min the incoming laser is added to the
// wave that the condition lets through.
#pragma once
#include "lpic_common.cuh"

namespace lpic {

template <typename R, typename JT>
struct FieldArgs {
    R* E[3];
    R* B[3];
    const JT* J[3];
    R rdx, rdy, rdz;      // 1 / h
    R tau;                // dt / 2
    double jfac[3];       // tau * (J units -> field units)
    FastDiv dfx, dny;     // division by the stored x extent and by ny
};

// tau J in field units: FP64 fields convert exactly in double; FP32 fields
// (J int64 fixed point) convert in single precision (one rounding of J and
// one of the product, well inside the FP32 path's tolerance).
template <typename R, typename JT>
__device__ inline R jterm(JT v, double f) {
    if constexpr (sizeof(R) == 4 && sizeof(JT) == 8) return __ll2float_rn((long long)v) * (float)f;
    else return (R)((double)v * f);
}

// Node n = (k ny + j) fx + i of a field array (fewer than 2^31 nodes).
__device__ inline void node_ijk(int n, const FastDiv& dfx, const FastDiv& dny, int& i, int& j, int& k) {
    const int r = fdiv(n, dfx);
    i = n - r * (int)dfx.d;
    k = fdiv(r, dny);
    j = r - k * (int)dny.d;
}

template <int DIM, typename R, typename JT>
__device__ inline void update_E_range(const Geo& g, const FieldArgs<R, JT>& a, long long n0, long long step) {
    const long long total = (long long)g.fx * g.ny * (DIM == 3 ? g.nz : 1);
    for (long long n = n0; n < total; n += step) {
        int i, j, k;
        node_ijk((int)n, a.dfx, a.dny, i, j, k);
        const long long nj = (j == 0) ? n + (long long)(g.ny - 1) * g.fx : n - g.fx;
        long long nk = n;
        if (DIM == 3) nk = (k == 0) ? n + (long long)(g.nz - 1) * g.ny * g.fx : n - (long long)g.ny * g.fx;
        long long ni;
        bool edge = false;
        if (g.absorb) { ni = n - 1; edge = (i == 0 || i == g.nx); }
        else          { ni = (i == 0) ? n + (g.nx - 1) : n - 1; }
        // E_x at (i+1/2, j, k)
        if (!(g.absorb && i == g.nx)) {
            R cb = (a.B[2][n] - a.B[2][nj]) * a.rdy;
            if (DIM == 3) cb -= (a.B[1][n] - a.B[1][nk]) * a.rdz;
            a.E[0][n] += a.tau * cb - jterm<R>(a.J[0][n], a.jfac[0]);
        }
        if (!edge) {
            // E_y at (i, j+1/2, k)
            R cb = -(a.B[2][n] - a.B[2][ni]) * a.rdx;
            if (DIM == 3) cb += (a.B[0][n] - a.B[0][nk]) * a.rdz;
            a.E[1][n] += a.tau * cb - jterm<R>(a.J[1][n], a.jfac[1]);
            // E_z at (i, j, k+1/2)
            const R cz = (a.B[1][n] - a.B[1][ni]) * a.rdx - (a.B[0][n] - a.B[0][nj]) * a.rdy;
            a.E[2][n] += a.tau * cz - jterm<R>(a.J[2][n], a.jfac[2]);
        }
    }
}

template <int DIM, typename R, typename JT>
__device__ inline void update_B_range(const Geo& g, const FieldArgs<R, JT>& a, long long n0, long long step) {
    const long long total = (long long)g.fx * g.ny * (DIM == 3 ? g.nz : 1);
    for (long long n = n0; n < total; n += step) {
        int i, j, k;
        node_ijk((int)n, a.dfx, a.dny, i, j, k);
        const long long nj = (j == g.ny - 1) ? n - (long long)(g.ny - 1) * g.fx : n + g.fx;
        long long nk = n;
        if (DIM == 3)
            nk = (k == g.nz - 1) ? n - (long long)(g.nz - 1) * g.ny * g.fx : n + (long long)g.ny * g.fx;
        const bool last = g.absorb && i == g.nx;
        const long long ni = (!g.absorb && i == g.nx - 1) ? n - (g.nx - 1) : n + 1;
        // B_x at (i, j+1/2, k+1/2)
        {
            R ce = (a.E[2][nj] - a.E[2][n]) * a.rdy;
            if (DIM == 3) ce -= (a.E[1][nk] - a.E[1][n]) * a.rdz;
            a.B[0][n] -= a.tau * ce;
        }
        if (!last) {
            // B_y at (i+1/2, j, k+1/2)
            R ce = -(a.E[2][ni] - a.E[2][n]) * a.rdx;
            if (DIM == 3) ce += (a.E[0][nk] - a.E[0][n]) * a.rdz;
            a.B[1][n] -= a.tau * ce;
            // B_z at (i+1/2, j+1/2, k)
            const R cz = (a.E[1][ni] - a.E[1][n]) * a.rdx - (a.E[0][nj] - a.E[0][n]) * a.rdy;
            a.B[2][n] -= a.tau * cz;
        }
    }
}

template <int DIM, typename R, typename JT>
__global__ void k_update_E(Geo g, FieldArgs<R, JT> a) {
    update_E_range<DIM>(g, a, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

template <int DIM, typename R, typename JT>
__global__ void k_update_B(Geo g, FieldArgs<R, JT> a) {
    update_B_range<DIM>(g, a, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// Save E_y, E_z on planes i = 0, 1, nx-1, nx before the E update:
// old[((c - 1) * 4 + p) * plane + q], q = k * ny + j.
template <typename R>
__global__ void k_mur_save(Geo g, Ptr3<R> E, R* old) {
    const int plane = g.ny * (g.dim == 3 ? g.nz : 1);
    const int planes[4] = {0, 1, g.nx - 1, g.nx};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * 4 * plane; t += gridDim.x * blockDim.x) {
        const int q = t % plane;
        const int p = (t / plane) % 4;
        const int c = 1 + t / (4 * plane);
        old[t] = E.p[c][(long long)q * g.fx + planes[p]];
    }
}

// Transverse laser profile of each row (j, k) of the x-min plane; E_y sits
// at y = (j + 1/2) dy, z = k dz.
__global__ void k_laser_profile(Geo g, Laser L, double* prof) {
    const int plane = g.ny * (g.dim == 3 ? g.nz : 1);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < plane; q += gridDim.x * blockDim.x) {
        const int j = q % g.ny, k = q / g.ny;
        prof[q] = laser_profile(L, g.dim, (j + 0.5) * g.dy, k * g.dz);
    }
}

// t_old = *clock + t_arg when a device clock is given (graph replay), else t_arg.
// The laser's time factors at x = 0 and x = dx, old and new time, are the same
// for every row: four threads of each block evaluate them once.
template <typename R>
__global__ void k_mur_apply(Geo g, Ptr3<R> E, const R* old, Laser L, const double* prof, double t_arg,
                            const double* clock, double tau) {
    __shared__ double s_tf[4][2];
    const int plane = g.ny * (g.dim == 3 ? g.nz : 1);
    const double c1 = (tau - g.dx) / (tau + g.dx);
    const double t_old = clock ? *clock + t_arg : t_arg;
    const double t_new = t_old + tau;
    if (threadIdx.x < 4) {
        const double tt = (threadIdx.x < 2) ? t_old : t_new;
        laser_time(L, tt - ((threadIdx.x & 1) ? g.dx : 0.0), s_tf[threadIdx.x][0], s_tf[threadIdx.x][1]);
    }
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * plane; t += gridDim.x * blockDim.x) {
        const int q = t % plane;
        const int c = 1 + t / plane;
        const R* o = old + (c - 1) * 4 * plane;
        const long long row = (long long)q * g.fx;
        double i0o = 0, i1o = 0, i0n = 0, i1n = 0;
        if (L.on && c == 1) {
            const double pr = prof[q];
            i0o = s_tf[0][0] * pr * s_tf[0][1];
            i1o = s_tf[1][0] * pr * s_tf[1][1];
            i0n = s_tf[2][0] * pr * s_tf[2][1];
            i1n = s_tf[3][0] * pr * s_tf[3][1];
        }
        const double e1n = (double)E.p[c][row + 1];
        E.p[c][row] = (R)(i0n + ((double)o[1 * plane + q] - i1o)
                        + c1 * ((e1n - i1n) - ((double)o[0 * plane + q] - i0o)));
        const double eMn = (double)E.p[c][row + g.nx - 1];
        E.p[c][row + g.nx] = (R)((double)o[2 * plane + q] + c1 * (eMn - (double)o[3 * plane + q]));
    }
}

// ----------------------------------------------------------------- CPML
// Layers of L cells at both x ends (layer slots 0..L: nodes 0..L; slots
// L+1..2L+1: nodes nx-L..nx).  After the interior update has applied the
// plain x derivative, these kernels add the difference to the CPML form
// (1/kappa) d/dx + psi, updating psi first (psi <- b psi + a d/dx).  Node
// coefficients serve E_y, E_z (at x = i dx), half-node ones B_y, B_z (at
// x = (i + 1/2) dx); E_y, E_z stay zero on the outer faces i = 0, nx.
template <typename R>
struct CpmlArgs {
    R* psi[4];                    // E_y, E_z, B_y, B_z memory: [plane][2 L + 2]
    const R* kinv[2];             // 1 / kappa: [0] nodes, [1] half nodes, fx entries
    const R* a[2];
    const R* b[2];
    int L;
};

__device__ inline int cpml_node(const Geo& g, int L, int slot) {
    return slot <= L ? slot : g.nx - L + (slot - (L + 1));
}

template <typename R>
__global__ void k_cpml_E(Geo g, Ptr3<R> E, Ptr3<const R> B, CpmlArgs<R> c, R tau) {
    const int plane = g.ny * (g.dim == 3 ? g.nz : 1);
    const int W = 2 * c.L + 2;
    const R rdx = (R)(1.0 / g.dx);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < plane * W; t += gridDim.x * blockDim.x) {
        const int q = t / W, slot = t - q * W;
        const int i = cpml_node(g, c.L, slot);
        if (i <= 0 || i >= g.nx) continue;
        const long long n = (long long)q * g.fx + i;
        const R ki = c.kinv[0][i], a = c.a[0][i], b = c.b[0][i];
        const R dbz = (B.p[2][n] - B.p[2][n - 1]) * rdx;
        const R p0 = b * c.psi[0][t] + a * dbz;
        c.psi[0][t] = p0;
        E.p[1][n] += tau * (((R)1 - ki) * dbz - p0);
        const R dby = (B.p[1][n] - B.p[1][n - 1]) * rdx;
        const R p1 = b * c.psi[1][t] + a * dby;
        c.psi[1][t] = p1;
        E.p[2][n] += tau * ((ki - (R)1) * dby + p1);
    }
}

template <typename R>
__global__ void k_cpml_B(Geo g, Ptr3<const R> E, Ptr3<R> B, CpmlArgs<R> c, R tau) {
    const int plane = g.ny * (g.dim == 3 ? g.nz : 1);
    const int W = 2 * c.L + 2;
    const R rdx = (R)(1.0 / g.dx);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < plane * W; t += gridDim.x * blockDim.x) {
        const int q = t / W, slot = t - q * W;
        const int i = cpml_node(g, c.L, slot);
        if (i < 0 || i >= g.nx) continue;
        const long long n = (long long)q * g.fx + i;
        const R ki = c.kinv[1][i], a = c.a[1][i], b = c.b[1][i];
        const R dez = (E.p[2][n + 1] - E.p[2][n]) * rdx;
        const R p2 = b * c.psi[2][t] + a * dez;
        c.psi[2][t] = p2;
        B.p[1][n] -= tau * (((R)1 - ki) * dez - p2);
        const R dey = (E.p[1][n + 1] - E.p[1][n]) * rdx;
        const R p3 = b * c.psi[3][t] + a * dey;
        c.psi[3][t] = p3;
        B.p[2][n] -= tau * ((ki - (R)1) * dey + p3);
    }
}

// The laser with CPML: a surface current K_y = -2 E_inc on node plane `is`
// radiates E_inc into +x (and into -x, where the layer absorbs it); added to
// E_y there as tau K_y / dx with the laser at the half step's centre time
// t_old + tau / 2 (t_old = *clock + t_arg under graph replay).
template <typename R>
__global__ void k_laser_sheet(Geo g, R* Ey, Laser L, const double* prof, int is, double t_arg,
                              const double* clock, double tau) {
    __shared__ double s_tf[2];
    const int plane = g.ny * (g.dim == 3 ? g.nz : 1);
    if (threadIdx.x == 0) {
        const double t_old = clock ? *clock + t_arg : t_arg;
        laser_time(L, t_old + 0.5 * tau, s_tf[0], s_tf[1]);
    }
    __syncthreads();
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < plane; q += gridDim.x * blockDim.x) {
        const double einc = s_tf[0] * prof[q] * s_tf[1];
        const long long n = (long long)q * g.fx + is;
        Ey[n] = (R)((double)Ey[n] + tau * (2.0 * einc / g.dx));
    }
}

// Device clock of the captured step: advanced by dt at the end of each replay.
__global__ void k_clock_add(double* clock, double dt) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *clock += dt;
}

__global__ void k_clock_set(double* clock, double t) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *clock = t;
}

// Step counter of the fused emission: advanced at the end of each full step.
__global__ void k_add_uint(unsigned* p, unsigned v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p += v;
}

__global__ void k_set_uint(unsigned* p, unsigned v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

}  // namespace lpic
