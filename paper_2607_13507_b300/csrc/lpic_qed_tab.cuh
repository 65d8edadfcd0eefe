// lpic_qed_tab.cuh -- device pieces of the nonlinear Compton module (Sec.
// 3.4) shared by the emission pass and the fused particle kernel: the
// Philox4x32-10 counter-based generator and the lookups of the photon rate
// and spectrum tables (built on the host at lpic_qed_init).
#pragma once
#include <cstdint>
#include "lpic_common.cuh"

namespace lpic {

// ------------------------------------------------------------ Philox4x32-10
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ inline void mulhilo32(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

// Ten rounds of the Philox-4x32 bijection (multipliers 0xD2511F53 and
// 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85).
__host__ __device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        uint32_t h0, l0, h1, l1;
        mulhilo32(0xD2511F53u, c.x, h0, l0);
        mulhilo32(0xCD9E8D57u, c.z, h1, l1);
        c = U4{h1 ^ c.y ^ k0, l1, h0 ^ c.w ^ k1, l0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// uniform in (0, 1) from 32 bits: (x + 1/2) 2^-32
// (x + 1/2) 2^-32 in single precision, kept below 1
__device__ __forceinline__ float u01f(uint32_t x) { return fminf(((float)x + 0.5f) * 0x1p-32f, 0.99999994f); }

// -ln u for u = (x + 1/2) 2^-32, in single precision (the FP64 units of this
// part are slow): below 1/2 from u itself, above it as -log1p(-(1 - u)) with
// 1 - u = ((2^32 - 1 - x) + 1/2) 2^-32 formed without cancellation, so the
// relative error stays at float rounding for every x
__device__ __forceinline__ float neg_log_u01(uint32_t x) {
    if (x < 0x80000000u) return -logf(((float)x + 0.5f) * 0x1p-32f);
    return -log1pf(-(((float)(0xFFFFFFFFu - x) + 0.5f) * 0x1p-32f));
}

// --------------------------------------------------------------- the tables
struct QedTab {
    const float* logh;     // [nchi]
    const float* cdf;      // [nchi][ny]
    const float* top;      // [nchi]
    int nchi, ny;
    float lchi0, inv_dl;   // ln chi_0, 1 / dl
    float chi0;
    float pref;            // alpha / (eps_ref sqrt(3) pi): W = pref h(chi) / gamma
    float eps_ref;
};

// h(chi): piecewise linear in (ln chi, ln h); linear extrapolation in the
// log-log plane past the last node (h grows like chi^{2/3} there).
__device__ inline float qed_h(const QedTab& T, float chi) {
    if (chi <= T.chi0) return __expf(T.logh[0]) * (chi / T.chi0);
    const float u = (logf(chi) - T.lchi0) * T.inv_dl;
    const int i = min((int)u, T.nchi - 2);
    const float f = u - (float)i;
    return expf(T.logh[i] + f * (T.logh[i + 1] - T.logh[i]));
}

__device__ inline float qed_map(float y, float top) {
    const float y3 = y * y * y;
    return top < 1.0f ? top * y3 : y3 * (10.0f + y * (-15.0f + 6.0f * y));
}

// xi of cumulative probability r in table row i, given the interval
// [lo, hi] of the row's cumulative that holds r: xi^{1/3} linear in the
// probability (the cumulative grows like xi^{1/3} at small xi).
__device__ __forceinline__ float qed_row_xi_at(const QedTab& T, int i, int lo, int hi, float r) {
    const float* P = T.cdf + (long long)i * T.ny;
    const float pa = P[lo], pb = P[hi];
    const float f = pb > pa ? fminf((r - pa) / (pb - pa), 1.0f) : 0.0f;
    const float dy = 1.0f / (float)(T.ny - 1);
    const float za = cbrtf(qed_map((float)lo * dy, T.top[i]));
    const float zb = cbrtf(qed_map((float)hi * dy, T.top[i]));
    const float z = za + f * (zb - za);
    return z * z * z;
}

// The intervals holding r in rows i0 and i1, by bisections of both rows in
// one loop (their loads are independent, so the two chains of dependent
// loads overlap).
__device__ __forceinline__ void qed_bisect2(const QedTab& T, int i0, int i1, float r, int& lo0, int& hi0,
                                            int& lo1, int& hi1) {
    const float* P0 = T.cdf + (long long)i0 * T.ny;
    const float* P1 = T.cdf + (long long)i1 * T.ny;
    lo0 = 0; hi0 = T.ny - 1; lo1 = 0; hi1 = T.ny - 1;
    while (hi0 - lo0 > 1 || hi1 - lo1 > 1) {
        const int m0 = (lo0 + hi0) >> 1, m1 = (lo1 + hi1) >> 1;
        const float p0 = P0[m0], p1 = P1[m1];
        if (hi0 - lo0 > 1) { if (p0 <= r) lo0 = m0; else hi0 = m0; }
        if (hi1 - lo1 > 1) { if (p1 <= r) lo1 = m1; else hi1 = m1; }
    }
}

// xi(chi, r): rows interpolated in (ln chi, ln xi) (exact in the classical
// limit, where xi is proportional to chi); clamped to the last row.
__device__ inline float qed_xi(const QedTab& T, float chi, float r) {
    int lo0, hi0, lo1, hi1;
    if (chi <= T.chi0) {
        qed_bisect2(T, 0, 0, r, lo0, hi0, lo1, hi1);
        return qed_row_xi_at(T, 0, lo0, hi0, r) * (chi / T.chi0);
    }
    float u = (logf(chi) - T.lchi0) * T.inv_dl;
    u = fminf(u, (float)(T.nchi - 1));
    const int i = min((int)u, T.nchi - 2);
    const float f = u - (float)i;
    qed_bisect2(T, i, i + 1, r, lo0, hi0, lo1, hi1);
    const float a = qed_row_xi_at(T, i, lo0, hi0, r), b = qed_row_xi_at(T, i + 1, lo1, hi1, r);
    if (!(a > 0.0f) || !(b > 0.0f)) return a + f * (b - a);
    return expf(logf(a) + f * (logf(b) - logf(a)));
}

}  // namespace lpic
