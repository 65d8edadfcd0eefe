// lpic_common.cuh -- device helpers shared by the liblpic kernels:
// index wrapping, particle shapes (Sec. 3.1), the relativistic Boris push
// (Sec. 3.1), the incoming laser (Sec. 4.2) and the status word.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "lpic.h"

namespace lpic {

// ------------------------------------------------------------ geometry
struct Geo {
    int dim, nx, ny, nz, fx;      // cells; stored x extent of field arrays
    int absorb;                    // absorbing x edges
    double dx, dy, dz, dt;
};

// Wrap an index that is off by less than one period.
__host__ __device__ inline int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
// Wrap any index into [0, n).
__host__ __device__ inline int wrapm(int i, int n) { i %= n; return i < 0 ? i + n : i; }

// wrapm with a cheap path for indices off by less than one period.
__host__ __device__ inline int wrapn(int i, int n) {
    if (i < 0) { i += n; if (i < 0) i = wrapm(i, n); }
    else if (i >= n) { i -= n; if (i >= n) i = wrapm(i, n); }
    return i;
}

// Linear field index of node (i, j, k); periodic dimensions wrap, an
// absorbing x index outside [0, fx) yields -1.
__device__ inline long long fidx(const Geo& g, int i, int j, int k) {
    if (g.absorb) {
        if (i < 0 || i >= g.fx) return -1;
    } else {
        i = wrapm(i, g.nx);
    }
    j = wrapm(j, g.ny);
    k = (g.dim == 3) ? wrapm(k, g.nz) : 0;
    return ((long long)k * g.ny + j) * g.fx + i;
}

// fidx for the loops over a tile's boxes, whose indices are mostly within
// one period of the grid.
__device__ inline long long fidx_near(const Geo& g, int i, int j, int k) {
    if (g.absorb) {
        if (i < 0 || i >= g.fx) return -1;
    } else {
        i = wrapn(i, g.nx);
    }
    j = wrapn(j, g.ny);
    k = (g.dim == 3) ? wrapn(k, g.nz) : 0;
    return ((long long)k * g.ny + j) * g.fx + i;
}

template <typename T> struct Ptr3 { T* p[3]; };

// Division by a runtime constant d >= 1 with a multiply-high (Granlund and
// Montgomery 1994): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (umulhi(n, m) + n) >> l for 0 <= n < 2^31.
struct FastDiv { unsigned d, m, l; };

inline FastDiv make_fastdiv(unsigned d) {
    unsigned l = 0;
    while ((1ull << l) < d) ++l;
    const unsigned long long m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
    return FastDiv{d, (unsigned)m, l};
}

__device__ inline int fdiv(int n, const FastDiv& f) {
    return (int)((__umulhi((unsigned)n, f.m) + (unsigned)n) >> f.l);
}

// Cell coordinates of a linear cell index (k * ny + j) * nx + i.
struct CellDecode {
    FastDiv nx, ny;
    __device__ inline void operator()(int cell, int* gc) const {
        const int r = fdiv(cell, nx);
        gc[0] = cell - r * (int)nx.d;
        gc[2] = fdiv(r, ny);
        gc[1] = r - gc[2] * (int)ny.d;
    }
};

// Round to the nearest integer (ties to even) for |x| < 2^22: adding
// 1.5 * 2^23 leaves the rounded value in the low mantissa bits.
__device__ inline int rint22(float x) {
    return __float_as_int(__fadd_rn(x, 12582912.0f)) - 0x4B400000;
}
// rint(a * b) with one rounding: the product is formed exactly inside the
// fused multiply-add, so this is the nearest integer to the exact a * b.
__device__ inline int rint22_mul(float a, float b) {
    return __float_as_int(__fmaf_rn(a, b, 12582912.0f)) - 0x4B400000;
}

__device__ inline void set_status(unsigned* st, unsigned bit) { atomicOr(st, bit); }

// ------------------------------------------------------------ shapes (Sec. 3.1)
// Weights of a particle on the integer nodes of one dimension, from its cell
// lc and in-cell offset f in [0, 1).  Order 1 (cloud-in-cell): nodes lc, lc+1.
// Order 2 (quadratic spline): the three nodes around the nearest one.  The
// arithmetic uses explicitly rounded intrinsics (no contraction), so the same
// (cell, offset) pair always gives bit-identical weights -- the fixed-point
// deposit relies on this to chain charge exactly from one step to the next.
template <int ORDER> struct NodeW;

template <> struct NodeW<1> {
    int base; float w[2];
    __device__ __forceinline__ static int base_of(int lc, float) { return lc; }
    __device__ __forceinline__ NodeW(int lc, float f) {
        base = lc; w[0] = __fsub_rn(1.0f, f); w[1] = f;
    }
};

template <> struct NodeW<2> {
    int base; float w[3];
    __device__ __forceinline__ static int base_of(int lc, float f) { return f < 0.5f ? lc - 1 : lc; }
    __device__ __forceinline__ NodeW(int lc, float f) {
        float d;
        if (f < 0.5f) { base = lc - 1; d = f; }
        else          { base = lc;     d = __fsub_rn(f, 1.0f); }   // exact for f in [0.5, 1)
        const float a = __fsub_rn(0.5f, d), b = __fadd_rn(0.5f, d);
        w[0] = __fmul_rn(0.5f, __fmul_rn(a, a));
        w[1] = __fsub_rn(0.75f, __fmul_rn(d, d));
        w[2] = __fmul_rn(0.5f, __fmul_rn(b, b));
    }
};

// Weights on the half-integer nodes (index i stands for position i + 1/2).
template <int ORDER> struct HalfW;

template <> struct HalfW<1> {
    int base; float w[2];
    __device__ __forceinline__ HalfW(int lc, float f) {
        float t;
        if (f >= 0.5f) { base = lc; t = f - 0.5f; } else { base = lc - 1; t = f + 0.5f; }
        w[0] = 1.0f - t; w[1] = t;
    }
};

template <> struct HalfW<2> {
    int base; float w[3];
    __device__ __forceinline__ HalfW(int lc, float f) {
        const float d = f - 0.5f;           // distance to half node lc (position lc + 1/2)
        base = lc - 1;
        const float a = 0.5f - d, b = 0.5f + d;
        w[0] = 0.5f * a * a; w[1] = 0.75f - d * d; w[2] = 0.5f * b * b;
    }
};

// Double-precision weights at an arbitrary coordinate xi (cell units).
template <int ORDER> struct NodeWd;
template <> struct NodeWd<1> {
    int base; double w[2];
    __device__ inline NodeWd(double xi) {
        const double fl = floor(xi); base = (int)fl; const double f = xi - fl;
        w[0] = 1.0 - f; w[1] = f;
    }
};
template <> struct NodeWd<2> {
    int base; double w[3];
    __device__ inline NodeWd(double xi) {
        const double n = floor(xi + 0.5); const double d = xi - n; base = (int)n - 1;
        const double a = 0.5 - d, b = 0.5 + d;
        w[0] = 0.5 * a * a; w[1] = 0.75 - d * d; w[2] = 0.5 * b * b;
    }
};

// ------------------------------------------------------------ Boris (Sec. 3.1)
// u = gamma v (c = 1); k = q dt / (2 m).  Half electric kick, rotation about
// B with gamma taken after the first kick, half electric kick.
template <typename R>
__device__ inline void boris(R& ux, R& uy, R& uz, R k, R ex, R ey, R ez, R bx, R by, R bz) {
    const R mx = ux + k * ex, my = uy + k * ey, mz = uz + k * ez;
    const R g = sqrt(R(1) + mx * mx + my * my + mz * mz);
    const R tx = k * bx / g, ty = k * by / g, tz = k * bz / g;
    const R t2 = tx * tx + ty * ty + tz * tz;
    const R f = R(2) / (R(1) + t2);
    const R sx = f * tx, sy = f * ty, sz = f * tz;
    const R px = mx + (my * tz - mz * ty);
    const R py = my + (mz * tx - mx * tz);
    const R pz = mz + (mx * ty - my * tx);
    ux = mx + (py * sz - pz * sy) + k * ex;
    uy = my + (pz * sx - px * sz) + k * ey;
    uz = mz + (px * sy - py * sx) + k * ez;
}

// FP32 Boris with hardware reciprocal square root and fast division (a few
// ulp, within the FP32 path's error budget).
__device__ __forceinline__ void boris_f32(float& ux, float& uy, float& uz, float k, float ex, float ey,
                                 float ez, float bx, float by, float bz) {
    const float mx = ux + k * ex, my = uy + k * ey, mz = uz + k * ez;
    const float kg = k * rsqrtf(1.0f + mx * mx + my * my + mz * mz);
    const float tx = kg * bx, ty = kg * by, tz = kg * bz;
    const float f = __fdividef(2.0f, 1.0f + tx * tx + ty * ty + tz * tz);
    const float sx = f * tx, sy = f * ty, sz = f * tz;
    const float px = mx + (my * tz - mz * ty);
    const float py = my + (mz * tx - mx * tz);
    const float pz = mz + (mx * ty - my * tx);
    ux = mx + (py * sz - pz * sy) + k * ex;
    uy = my + (pz * sx - px * sz) + k * ey;
    uz = mz + (px * sy - py * sx) + k * ez;
}

// ------------------------------------------------------------ laser (Sec. 4.2)
struct Laser {
    int on; double a0, w0, tau, omega, yc, zc;
};

// The laser's E_y = a0 env(s) exp(-r^2 / w0^2) sin(omega s), s = t - x, split
// into its time factors (a0 env, sin) and its transverse profile.
__device__ inline void laser_time(const Laser& L, double s, double& a0env, double& sn) {
    if (!L.on || s <= 0.0 || s >= L.tau) { a0env = 0.0; sn = 0.0; return; }
    double env = sin(3.14159265358979323846 * s / L.tau);
    env *= env;
    a0env = L.a0 * env;
    sn = sin(L.omega * s);
}
__device__ inline double laser_profile(const Laser& L, int dim, double y, double z) {
    double r2 = (y - L.yc) * (y - L.yc);
    if (dim == 3) r2 += (z - L.zc) * (z - L.zc);
    return exp(-r2 / (L.w0 * L.w0));
}

}  // namespace lpic
