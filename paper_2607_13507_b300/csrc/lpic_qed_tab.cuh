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
__device__ inline double u01d(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386963e-10; }

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

// xi of cumulative probability r in table row i: bisection for the interval
// of the cumulative holding r, then xi^{1/3} linear in the probability (the
// cumulative grows like xi^{1/3} at small xi).
__device__ inline float qed_row_xi(const QedTab& T, int i, float r) {
    const float* P = T.cdf + (long long)i * T.ny;
    int lo = 0, hi = T.ny - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (P[mid] <= r) lo = mid; else hi = mid;
    }
    const float pa = P[lo], pb = P[hi];
    const float f = pb > pa ? fminf((r - pa) / (pb - pa), 1.0f) : 0.0f;
    const float dy = 1.0f / (float)(T.ny - 1);
    const float za = cbrtf(qed_map((float)lo * dy, T.top[i]));
    const float zb = cbrtf(qed_map((float)hi * dy, T.top[i]));
    const float z = za + f * (zb - za);
    return z * z * z;
}

// xi(chi, r): rows interpolated in (ln chi, ln xi) (exact in the classical
// limit, where xi is proportional to chi); clamped to the last row.
__device__ inline float qed_xi(const QedTab& T, float chi, float r) {
    if (chi <= T.chi0) return qed_row_xi(T, 0, r) * (chi / T.chi0);
    float u = (logf(chi) - T.lchi0) * T.inv_dl;
    u = fminf(u, (float)(T.nchi - 1));
    const int i = min((int)u, T.nchi - 2);
    const float f = u - (float)i;
    const float a = qed_row_xi(T, i, r), b = qed_row_xi(T, i + 1, r);
    if (!(a > 0.0f) || !(b > 0.0f)) return a + f * (b - a);
    return expf(logf(a) + f * (logf(b) - logf(a)));
}

}  // namespace lpic
