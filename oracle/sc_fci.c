/*
 * Oracle (test infrastructure only): Slater–Condon matrix elements of the
 * electronic Hamiltonian between spin-orbital determinants, a dense builder,
 * a matrix-free matvec, and brute-force reduced density matrices.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this code.  It shares nothing with the CUDA library.
 *
 * What it computes (the paper, Methods, "Incremental Full Configuration
 * Interaction": each E_c(X) is a correlation energy from a CI in the orbitals
 * of body set X; here the CI is exact FCI in that space):
 *
 *   H = sum_{PQ} h_PQ a+_P a_Q + 1/2 sum_{PQRS} <PR|QS> a+_P a+_R a_S a_Q,
 *   <PR|QS> = (pq|rs) delta(sP,sQ) delta(sR,sS)   (chemist (pq|rs), real orbitals)
 *
 * Determinants: two bit masks over the local orbitals (bit p = orbital p),
 * alpha mask a and beta mask b, |a,b> = A+(a) B+(b)|0>, where A+(a) creates
 * the occupied alpha spin-orbitals in ascending orbital order and B+(b) the
 * beta ones; canonical spin-orbital order is all alpha, then all beta.
 * The phase of an operator acting on spin-orbital X is (-1)^(number of
 * occupied spin-orbitals that precede X in that order).
 *
 * Integrals: h is norb*norb row-major, eri is norb^4 row-major
 * eri[((p*norb+q)*norb+r)*norb+s] = (pq|rs).  norb <= 64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { uint64_t a, b; } det_t;

static inline int popc(uint64_t x) { return __builtin_popcountll(x); }
static inline uint64_t below(int p) { return p >= 64 ? ~0ull : ((1ull << p) - 1ull); }

/* Annihilate spin-orbital (p, spin) in *d.  Returns the phase (+1/-1) or 0 if empty. */
static int annihilate(det_t *d, int p, int spin) {
    if (spin == 0) {
        if (!((d->a >> p) & 1ull)) return 0;
        int n = popc(d->a & below(p));
        d->a &= ~(1ull << p);
        return (n & 1) ? -1 : 1;
    } else {
        if (!((d->b >> p) & 1ull)) return 0;
        int n = popc(d->a) + popc(d->b & below(p));
        d->b &= ~(1ull << p);
        return (n & 1) ? -1 : 1;
    }
}

/* Create spin-orbital (p, spin) in *d.  Returns the phase or 0 if occupied. */
static int create(det_t *d, int p, int spin) {
    if (spin == 0) {
        if ((d->a >> p) & 1ull) return 0;
        int n = popc(d->a & below(p));
        d->a |= (1ull << p);
        return (n & 1) ? -1 : 1;
    } else {
        if ((d->b >> p) & 1ull) return 0;
        int n = popc(d->a) + popc(d->b & below(p));
        d->b |= (1ull << p);
        return (n & 1) ? -1 : 1;
    }
}

#define ERI(n, p, q, r, s) eri[(((size_t)(p) * (n) + (q)) * (n) + (r)) * (n) + (s)]

/* Physicist <PR|QS> with spin deltas, P=(p,sp) etc. */
static inline double phys(int n, const double *eri, int p, int sp, int r, int sr,
                          int q, int sq, int s, int ss) {
    if (sp != sq || sr != ss) return 0.0;
    return ERI(n, p, q, r, s);
}

/* Lowest set bit index of a mask, and a list of set bits. */
static int bits(uint64_t m, int *out) {
    int k = 0;
    while (m) { out[k++] = __builtin_ctzll(m); m &= m - 1; }
    return k;
}

/* <I|H|J> by the Slater–Condon rules. */
double oracle_h_element(int n, const double *h, const double *eri,
                        uint64_t ia, uint64_t ib, uint64_t ja, uint64_t jb) {
    uint64_t da = ia ^ ja, db = ib ^ jb;
    int ndiff = popc(da) + popc(db);
    if (popc(ia) != popc(ja) || popc(ib) != popc(jb)) return 0.0;   /* spin conservation */
    if (ndiff == 0) {
        int oa[64], ob[64];
        int na = bits(ia, oa), nb = bits(ib, ob);
        double e = 0.0;
        for (int i = 0; i < na; i++) e += h[oa[i] * n + oa[i]];
        for (int i = 0; i < nb; i++) e += h[ob[i] * n + ob[i]];
        /* 1/2 sum over ordered pairs of occupied spin-orbitals of <PQ||PQ> */
        double two = 0.0;
        for (int i = 0; i < na; i++)
            for (int j = 0; j < na; j++)
                two += ERI(n, oa[i], oa[i], oa[j], oa[j]) - ERI(n, oa[i], oa[j], oa[j], oa[i]);
        for (int i = 0; i < nb; i++)
            for (int j = 0; j < nb; j++)
                two += ERI(n, ob[i], ob[i], ob[j], ob[j]) - ERI(n, ob[i], ob[j], ob[j], ob[i]);
        for (int i = 0; i < na; i++)
            for (int j = 0; j < nb; j++)
                two += 2.0 * ERI(n, oa[i], oa[i], ob[j], ob[j]);
        return e + 0.5 * two;
    }
    if (ndiff == 2) {
        /* single excitation: Q (occupied in J, not I) -> P (occupied in I, not J) */
        int spin = popc(da) ? 0 : 1;
        uint64_t jm = spin ? jb : ja, im = spin ? ib : ia;
        int q = __builtin_ctzll(jm & ~im), p = __builtin_ctzll(im & ~jm);
        det_t d = {ja, jb};
        int ph = annihilate(&d, q, spin);
        ph *= create(&d, p, spin);
        double v = h[p * n + q];
        int oa[64], ob[64];
        int na = bits(ja, oa), nb = bits(jb, ob);
        for (int i = 0; i < na; i++) {
            int r = oa[i];
            v += ERI(n, p, q, r, r) - (spin == 0 ? ERI(n, p, r, r, q) : 0.0);
        }
        for (int i = 0; i < nb; i++) {
            int r = ob[i];
            v += ERI(n, p, q, r, r) - (spin == 1 ? ERI(n, p, r, r, q) : 0.0);
        }
        return ph * v;
    }
    if (ndiff == 4) {
        /* double excitation: holes Q,S in J; particles P,R in I. */
        int hs[2], hsp[2], ps[2], psp[2], nh = 0, np = 0;
        uint64_t x;
        x = ja & ~ia; while (x) { hs[nh] = __builtin_ctzll(x); hsp[nh++] = 0; x &= x - 1; }
        x = jb & ~ib; while (x) { hs[nh] = __builtin_ctzll(x); hsp[nh++] = 1; x &= x - 1; }
        x = ia & ~ja; while (x) { ps[np] = __builtin_ctzll(x); psp[np++] = 0; x &= x - 1; }
        x = ib & ~jb; while (x) { ps[np] = __builtin_ctzll(x); psp[np++] = 1; x &= x - 1; }
        if (nh != 2 || np != 2) return 0.0;
        int Q = hs[0], sQ = hsp[0], S = hs[1], sS = hsp[1];
        int P = ps[0], sP = psp[0], R = ps[1], sR = psp[1];
        /* phase of a+_P a+_R a_S a_Q |J> (rightmost acts first) */
        det_t d = {ja, jb};
        int ph = annihilate(&d, Q, sQ);
        ph *= annihilate(&d, S, sS);
        ph *= create(&d, R, sR);
        ph *= create(&d, P, sP);
        double v = phys(n, eri, P, sP, R, sR, Q, sQ, S, sS) - phys(n, eri, P, sP, R, sR, S, sS, Q, sQ);
        return ph * v;
    }
    return 0.0;
}

/* Dense H over an explicit determinant list (row-major ndet x ndet). */
void oracle_h_dense(int n, const double *h, const double *eri, int ndet,
                    const uint64_t *da, const uint64_t *db, double *H) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < ndet; i++)
        for (int j = 0; j < ndet; j++)
            H[(size_t)i * ndet + j] = oracle_h_element(n, h, eri, da[i], db[i], da[j], db[j]);
}

/*
 * Matrix-free y = H x over the determinant space
 *   { core | alpha string, core | beta string },
 * where the core orbitals are local orbitals [0, ncore) (doubly occupied in
 * every determinant) and the active strings are masks over local orbitals
 * [ncore, ncore + nact).  Determinant (ia, ib) has index ia * nstr + ib.
 * rank_of[m >> ncore] gives the position of active mask m in ``strings``.
 * Row I is formed from every determinant J that differs from I by at most a
 * double excitation inside the active orbitals; H_IJ comes from
 * oracle_h_element.
 */
void oracle_matvec(int n, const double *h, const double *eri, int ncore, int nact,
                   int nstr, const uint64_t *strings, const int32_t *rank_of,
                   const double *x, double *y) {
    uint64_t core = below(ncore);
    int64_t ndet = (int64_t)nstr * nstr;
    #pragma omp parallel
    {
        /* per-thread lists of connected strings: singles <= nact^2/4 and
           doubles <= (nact^2/8)^2 for any occupation of nact orbitals */
        int cap = 1 + nact * nact + (nact * nact / 2) * (nact * nact / 2) + 8;
        uint64_t *SA = (uint64_t *)malloc(sizeof(uint64_t) * cap);
        uint64_t *SB = (uint64_t *)malloc(sizeof(uint64_t) * cap);
        #pragma omp for schedule(dynamic, 64)
        for (int64_t I = 0; I < ndet; I++) {
            int ia = (int)(I / nstr), ib = (int)(I % nstr);
            uint64_t A = strings[ia], B = strings[ib];
            uint64_t IA = core | A, IB = core | B;
            double acc = oracle_h_element(n, h, eri, IA, IB, IA, IB) * x[I];
            int occA[64], virA[64], occB[64], virB[64];
            int noa = 0, nva = 0, nob = 0, nvb = 0;
            for (int p = ncore; p < ncore + nact; p++) {
                if ((A >> p) & 1ull) occA[noa++] = p; else virA[nva++] = p;
                if ((B >> p) & 1ull) occB[nob++] = p; else virB[nvb++] = p;
            }
            /* alpha strings connected to A: [0, sa1) singles, [sa1, sa2) doubles */
            int ns = 0, nt = 0;
            for (int i = 0; i < noa; i++)
                for (int a = 0; a < nva; a++) SA[ns++] = (A & ~(1ull << occA[i])) | (1ull << virA[a]);
            int sa1 = ns;
            for (int i = 0; i < noa; i++) for (int j = i + 1; j < noa; j++)
                for (int a = 0; a < nva; a++) for (int b = a + 1; b < nva; b++)
                    SA[ns++] = (A & ~(1ull << occA[i]) & ~(1ull << occA[j])) | (1ull << virA[a]) | (1ull << virA[b]);
            for (int i = 0; i < nob; i++)
                for (int a = 0; a < nvb; a++) SB[nt++] = (B & ~(1ull << occB[i])) | (1ull << virB[a]);
            int sb1 = nt;
            for (int i = 0; i < nob; i++) for (int j = i + 1; j < nob; j++)
                for (int a = 0; a < nvb; a++) for (int b = a + 1; b < nvb; b++)
                    SB[nt++] = (B & ~(1ull << occB[i]) & ~(1ull << occB[j])) | (1ull << virB[a]) | (1ull << virB[b]);
            int rb = rank_of[B >> ncore], ra = rank_of[A >> ncore];
            /* alpha single or double, beta unchanged */
            for (int s = 0; s < ns; s++) {
                double hij = oracle_h_element(n, h, eri, IA, IB, core | SA[s], IB);
                acc += hij * x[(int64_t)rank_of[SA[s] >> ncore] * nstr + rb];
            }
            /* beta single or double, alpha unchanged */
            for (int t = 0; t < nt; t++) {
                double hij = oracle_h_element(n, h, eri, IA, IB, IA, core | SB[t]);
                acc += hij * x[(int64_t)ra * nstr + rank_of[SB[t] >> ncore]];
            }
            /* alpha single and beta single */
            for (int s = 0; s < sa1; s++) {
                int ja = rank_of[SA[s] >> ncore];
                for (int t = 0; t < sb1; t++) {
                    double hij = oracle_h_element(n, h, eri, IA, IB, core | SA[s], core | SB[t]);
                    acc += hij * x[(int64_t)ja * nstr + rank_of[SB[t] >> ncore]];
                }
            }
            y[I] = acc;
        }
        free(SA); free(SB);
    }
}

/* Rows of H x for a list of determinant indices only (sampled parity at large sizes). */
void oracle_matvec_rows(int n, const double *h, const double *eri, int ncore, int nact,
                        int nstr, const uint64_t *strings, const int32_t *rank_of,
                        const double *x, int nrows, const int64_t *rows, double *y) {
    uint64_t core = below(ncore);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nrows; k++) {
        int64_t I = rows[k];
        int ia = (int)(I / nstr), ib = (int)(I % nstr);
        uint64_t IA = core | strings[ia], IB = core | strings[ib];
        double acc = 0.0;
        for (int ja = 0; ja < nstr; ja++) {
            uint64_t JA = core | strings[ja];
            int ea = popc(JA ^ IA) / 2;
            if (ea > 2) continue;
            for (int jb = 0; jb < nstr; jb++) {
                uint64_t JB = core | strings[jb];
                if (ea + popc(JB ^ IB) / 2 > 2) continue;
                acc += oracle_h_element(n, h, eri, IA, IB, JA, JB) * x[(int64_t)ja * nstr + jb];
            }
        }
        y[k] = acc;
    }
}

/* ---- brute-force expectation values over an explicit, sorted determinant list ---- */

static int64_t find_det(int64_t ndet, const uint64_t *da, const uint64_t *db, uint64_t a, uint64_t b) {
    int64_t lo = 0, hi = ndet - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (da[mid] < a || (da[mid] == a && db[mid] < b)) lo = mid + 1;
        else if (da[mid] == a && db[mid] == b) return mid;
        else hi = mid - 1;
    }
    return -1;
}

/*
 * Spin-summed one- and two-particle density matrices of the real vector c:
 *   gamma[p,q]     = sum_s <c| a+_ps a_qs |c>
 *   Gamma[p,q,r,s] = sum_{s1,s2} <c| a+_{p s1} a+_{r s2} a_{s s2} a_{q s1} |c>
 * The determinant list must be sorted by (alpha mask, beta mask) ascending and
 * closed under the operators' action within its particle/spin sector.
 */
void oracle_rdm12(int n, int64_t ndet, const uint64_t *da, const uint64_t *db,
                  const double *c, double *gamma, double *Gamma) {
    memset(gamma, 0, sizeof(double) * n * n);
    memset(Gamma, 0, sizeof(double) * (size_t)n * n * n * n);
    for (int64_t J = 0; J < ndet; J++) {
        if (c[J] == 0.0) continue;
        for (int q = 0; q < n; q++) for (int sq = 0; sq < 2; sq++) {
            det_t d1 = {da[J], db[J]};
            int ph1 = annihilate(&d1, q, sq);
            if (!ph1) continue;
            for (int p = 0; p < n; p++) {
                det_t d2 = d1;
                int ph2 = create(&d2, p, sq);
                if (!ph2) continue;
                int64_t I = find_det(ndet, da, db, d2.a, d2.b);
                if (I >= 0) gamma[p * n + q] += c[I] * c[J] * ph1 * ph2;
            }
            for (int s = 0; s < n; s++) for (int ss = 0; ss < 2; ss++) {
                det_t d2 = d1;
                int ph2 = annihilate(&d2, s, ss);
                if (!ph2) continue;
                for (int r = 0; r < n; r++) {
                    det_t d3 = d2;
                    int ph3 = create(&d3, r, ss);
                    if (!ph3) continue;
                    for (int p = 0; p < n; p++) {
                        det_t d4 = d3;
                        int ph4 = create(&d4, p, sq);
                        if (!ph4) continue;
                        int64_t I = find_det(ndet, da, db, d4.a, d4.b);
                        if (I >= 0)
                            Gamma[(((size_t)p * n + q) * n + r) * n + s] += c[I] * c[J] * ph1 * ph2 * ph3 * ph4;
                    }
                }
            }
        }
    }
}

/* <c| S- S+ |c> with S+ = sum_p a+_{p alpha} a_{p beta}; list sorted as above. */
double oracle_s_minus_s_plus(int n, int64_t ndet, const uint64_t *da, const uint64_t *db,
                             const double *c) {
    double acc = 0.0;
    for (int64_t J = 0; J < ndet; J++) {
        if (c[J] == 0.0) continue;
        for (int q = 0; q < n; q++) {
            det_t d1 = {da[J], db[J]};
            int ph = annihilate(&d1, q, 1);
            if (!ph) continue;
            ph *= create(&d1, q, 0);
            if (!ph) continue;
            for (int p = 0; p < n; p++) {
                det_t d2 = d1;
                int ph2 = annihilate(&d2, p, 0);
                if (!ph2) continue;
                ph2 *= create(&d2, p, 1);
                if (!ph2) continue;
                int64_t I = find_det(ndet, da, db, d2.a, d2.b);
                if (I >= 0) acc += c[I] * c[J] * ph * ph2;
            }
        }
    }
    return acc;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
