// Hamiltonian matrix elements <I|H|J> between determinants (alpha string,
// beta string) by the Slater–Condon rules on the occupation bit masks, for
// H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps)
// (no constant): zero beyond double excitations; for a single excitation
// j -> a (spin s) the sign is the parity of the orbitals occupied strictly
// between a and j; a same-spin double is two such excitations applied in
// turn; an opposite-spin double is the product of the two single signs.
#pragma once
#include "common.cuh"

namespace ifci {

// Jacobi rotation (c, s) that zeroes A_pq of a symmetric matrix.  The angle
// is taken in FP32 (its FP64 divides and square roots would cost ~40 FP64
// operations, on a part whose FP64 rate is a small fraction of its FP32
// rate), then (c, s) is scaled to c^2 + s^2 = 1 to FP64 rounding by two
// Newton steps on 1 / sqrt(c^2 + s^2), so the rotation stays orthogonal and
// the eigenvalues exact; the ~1e-7 error of the angle leaves A_pq at ~1e-7
// of its size, which the next sweep removes.
__device__ __forceinline__ void jacobi_rotation(double app, double aqq, double apq, double &c, double &s) {
    if (fabs(apq) < 1e-30) {   // below FP32's normal range: FP64 throughout
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        c = 1.0 / sqrt(1.0 + t * t);
        s = t * c;
        return;
    }
    const float tau = (float)(aqq - app) / (2.0f * (float)apq);
    const float tf = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
    const float cf = rsqrtf(1.0f + tf * tf);
    double cc = cf, ss = (double)tf * (double)cf;
#pragma unroll
    for (int it = 0; it < 2; it++) {
        const double k = 1.5 - 0.5 * (cc * cc + ss * ss);
        cc *= k;
        ss *= k;
    }
    c = cc;
    s = ss;
}

__device__ __forceinline__ int between_parity(uint32_t m, int p, int q) {
    const int lo = min(p, q), hi = max(p, q);
    const uint32_t mask = ((1u << hi) - 1u) & ~((2u << lo) - 1u);
    return __popc(m & mask) & 1;
}

__device__ __forceinline__ double eri4(const double *eri, int np, int p, int q, int r, int s) {
    return eri[(long long)pair_of(p, q) * np + pair_of(r, s)];
}

// <ia ib | H | ja jb> for alpha/beta occupation masks of n orbitals.
__device__ inline double h_element(int n, const double *__restrict__ h1, const double *__restrict__ eri, uint32_t ia,
                            uint32_t ib, uint32_t ja, uint32_t jb) {
    const int np = n * (n + 1) / 2;
    const uint32_t da = ia ^ ja, db = ib ^ jb;
    const int na = __popc(da) / 2, nb = __popc(db) / 2;
    if (na + nb > 2) return 0.0;
    if (na + nb == 0) {
        double e = 0.0, two = 0.0;
        for (uint32_t x = ia; x; x &= x - 1) e += h1[(__ffs(x) - 1) * (n + 1)];
        for (uint32_t x = ib; x; x &= x - 1) e += h1[(__ffs(x) - 1) * (n + 1)];
        for (uint32_t x = ia; x; x &= x - 1) {
            const int p = __ffs(x) - 1;
            for (uint32_t y = ia; y; y &= y - 1) {
                const int q = __ffs(y) - 1;
                two += eri4(eri, np, p, p, q, q) - eri4(eri, np, p, q, q, p);
            }
            for (uint32_t y = ib; y; y &= y - 1) two += 2.0 * eri4(eri, np, p, p, __ffs(y) - 1, __ffs(y) - 1);
        }
        for (uint32_t x = ib; x; x &= x - 1) {
            const int p = __ffs(x) - 1;
            for (uint32_t y = ib; y; y &= y - 1) {
                const int q = __ffs(y) - 1;
                two += eri4(eri, np, p, p, q, q) - eri4(eri, np, p, q, q, p);
            }
        }
        return e + 0.5 * two;
    }
    if (na + nb == 1) {
        // one electron j -> a of spin s; "same" = the other electrons of spin s, "other" = the other spin
        const bool alpha = na == 1;
        const uint32_t bra = alpha ? ia : ib, ket = alpha ? ja : jb, other = alpha ? ib : ia;
        const int a = __ffs(bra & ~ket) - 1, j = __ffs(ket & ~bra) - 1;
        double v = h1[a * n + j];
        for (uint32_t x = bra & ket; x; x &= x - 1) {
            const int k = __ffs(x) - 1;
            v += eri4(eri, np, a, j, k, k) - eri4(eri, np, a, k, k, j);
        }
        for (uint32_t x = other; x; x &= x - 1) {
            const int k = __ffs(x) - 1;
            v += eri4(eri, np, a, j, k, k);
        }
        return between_parity(ket, a, j) ? -v : v;
    }
    if (na == 1 && nb == 1) {
        const int a = __ffs(ia & ~ja) - 1, j = __ffs(ja & ~ia) - 1;
        const int b = __ffs(ib & ~jb) - 1, l = __ffs(jb & ~ib) - 1;
        const double v = eri4(eri, np, a, j, b, l);
        return (between_parity(ja, a, j) ^ between_parity(jb, b, l)) ? -v : v;
    }
    // two electrons of one spin: j1 -> a1, then j2 -> a2
    const bool alpha = na == 2;
    const uint32_t bra = alpha ? ia : ib, ket = alpha ? ja : jb;
    uint32_t up = bra & ~ket, dn = ket & ~bra;
    const int a1 = __ffs(up) - 1;
    up &= up - 1;
    const int a2 = __ffs(up) - 1;
    const int j1 = __ffs(dn) - 1;
    dn &= dn - 1;
    const int j2 = __ffs(dn) - 1;
    const int s1 = between_parity(ket, a1, j1);
    const uint32_t mid = ket ^ (1u << j1) ^ (1u << a1);
    const int s2 = between_parity(mid, a2, j2);
    const double v = eri4(eri, np, a1, j1, a2, j2) - eri4(eri, np, a1, j2, a2, j1);
    return (s1 ^ s2) ? -v : v;
}

}  // namespace ifci
