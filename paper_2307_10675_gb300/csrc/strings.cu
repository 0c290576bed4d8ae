// Occupation strings and the single-excitation table (integer kernels).
//
// A determinant of the CI of body set X is a pair of occupation strings of
// nelec_spin electrons in the norb active orbitals.  Strings are ranked by
// the combinatorial number system, rank(I) = sum_k C(p_k, k+1) over the
// occupied orbitals p_0 < p_1 < ..., which orders them by increasing integer
// value of the bit mask.
#include "common.cuh"

namespace ifci {

struct Binom {
    int c[32][32];
};

__device__ __forceinline__ int string_rank(uint32_t mask, const Binom &B) {
    int r = 0, k = 1;
    while (mask) {
        int p = __ffs(mask) - 1;
        r += B.c[p][k];
        k++;
        mask &= mask - 1;
    }
    return r;
}

__device__ __forceinline__ uint32_t string_unrank(int rank, int n, int m, const Binom &B) {
    uint32_t mask = 0;
    int rem = rank;
    for (int k = m; k >= 1; k--) {
        int p = k - 1;
        while (p + 1 < n && B.c[p + 1][k] <= rem) p++;
        rem -= B.c[p][k];
        mask |= 1u << p;
    }
    return mask;
}

// One thread per string I: its mask and its nexc excitation entries in
// ascending pair order.
__global__ void build_strings_kernel(int n, int m, int nstr, int nexc, Binom B,
                                     uint64_t *__restrict__ strings, int32_t *__restrict__ exc) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nstr) return;
    uint32_t mask = string_unrank(I, n, m, B);
    strings[I] = mask;
    int32_t *row = exc + (size_t)I * nexc;
    int k = 0;
    for (int P = 0; P < n; P++) {
        bool oP = (mask >> P) & 1u;
        for (int Q = 0; Q <= P; Q++) {
            int A = P * (P + 1) / 2 + Q;
            bool oQ = (mask >> Q) & 1u;
            if (P == Q) {
                if (oP && k < nexc) row[k++] = (I << 10) | (A << 1);
            } else if (oP != oQ) {
                // E_PQ (Q occupied) or E_QP (P occupied): move the electron
                // across the orbitals strictly between Q and P
                uint32_t J = mask ^ (1u << P) ^ (1u << Q);
                uint32_t between = ((1u << P) - 1u) & ~((2u << Q) - 1u);
                int neg = __popc(mask & between) & 1;
                if (k < nexc) row[k++] = (string_rank(J, B) << 10) | (A << 1) | neg;
            }
        }
    }
}

// blk[I][b] = index of the first entry of string I's excitation list whose
// pair is >= 16 b, for b = 0 .. kBlk16Stride - 1 (lists are sorted by pair, so the
// entries of the 16-pair block b are [blk[I][b], blk[I][b + 1])).
__global__ void exc_blocks_kernel(int nstr, int nexc, const int32_t *__restrict__ exc, uint8_t *__restrict__ blk) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nstr) return;
    const int32_t *row = exc + (size_t)I * nexc;
    uint8_t *out = blk + (size_t)I * kBlk16Stride;
    int e = 0;
    for (int b = 0; b < kBlk16Stride; b++) {   // 19 blocks + the end: npair up to 304
        while (e < nexc && exc_pair(row[e]) < 16 * b) e++;
        out[b] = (uint8_t)e;
    }
}

// Dense pair map of a string table for spin-flip-symmetric vectors:
// pmap[I][A] = J nstr + neg ndet for the entry (J, A, neg) of string I, -1 where
// I has no excitation on pair A (rows padded to pmap_ld(np) with -1).  The
// value is the element offset of +-c[J][0] in the pair [c | -c] of quantised
// copies, so the tensor-core gathers pick the sign by address.
__global__ void pair_map_kernel(int nstr, int nexc, int np, long long ndet, const int32_t *__restrict__ exc,
                                int32_t *__restrict__ pmap) {
    const int I = blockIdx.x;
    const int ld = pmap_ld(np);
    int32_t *row = pmap + (size_t)I * ld;
    for (int A = threadIdx.x; A < ld; A += blockDim.x) row[A] = -1;
    __syncthreads();
    for (int e = threadIdx.x; e < nexc; e += blockDim.x) {
        const int32_t x = exc[(size_t)I * nexc + e];
        row[exc_pair(x)] = (int32_t)((long long)exc_J(x) * nstr + ((x & 1) ? ndet : 0));
    }
}

int launch_pair_map(ifci_handle_t h, int nstr, int nexc, int np, const int32_t *exc, int32_t *pmap, cudaStream_t s) {
    const long long ndet = (long long)nstr * nstr;
    if (2 * ndet >= (1ll << 31)) return set_error(h, IFCI_ERR_INVALID_ARG, "pair map: %lld determinants", ndet);
    pair_map_kernel<<<nstr, 128, 0, s>>>(nstr, nexc, np, ndet, exc, pmap);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_exc_blocks(ifci_handle_t h, int nstr, int nexc, const int32_t *exc, uint8_t *blk, cudaStream_t s) {
    exc_blocks_kernel<<<(nstr + 127) / 128, 128, 0, s>>>(nstr, nexc, exc, blk);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

}  // namespace ifci

extern "C" {

int ifci_string_counts(int norb, int nelec_spin, int *nstr, int *nexc) {
    if (norb < 1 || norb > ifci::kMaxNorb || nelec_spin < 0 || nelec_spin > norb)
        return IFCI_ERR_INVALID_ARG;
    long long ns = ifci::binom(norb, nelec_spin);
    if (ns >= ifci::kMaxStr) return IFCI_ERR_INVALID_ARG;
    if (nstr) *nstr = (int)ns;
    if (nexc) *nexc = nelec_spin * (norb - nelec_spin + 1);
    return IFCI_OK;
}

int ifci_build_strings(ifci_handle_t h, int norb, int nelec_spin, uint64_t *strings, int32_t *exc,
                       ifci_stream_t stream) {
    if (!h) return IFCI_ERR_INVALID_ARG;
    int nstr = 0, nexc = 0;
    if (ifci_string_counts(norb, nelec_spin, &nstr, &nexc) != IFCI_OK)
        return ifci::set_error(h, IFCI_ERR_INVALID_ARG, "build_strings: norb=%d nelec_spin=%d out of range",
                               norb, nelec_spin);
    if (!strings || !exc) return ifci::set_error(h, IFCI_ERR_INVALID_ARG, "build_strings: null output");
    ifci::Binom B;
    for (int i = 0; i < 32; i++)
        for (int j = 0; j < 32; j++) B.c[i][j] = (int)ifci::binom(i, j);
    IFCI_CUDA_TRY(h, cudaSetDevice(h->device));
    int threads = 128, blocks = (nstr + threads - 1) / threads;
    ifci::build_strings_kernel<<<blocks, threads, 0, ifci::as_cuda(stream)>>>(norb, nelec_spin, nstr, nexc, B,
                                                                             strings, exc);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

}  // extern "C"
