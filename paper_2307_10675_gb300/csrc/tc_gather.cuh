// Fused gather D^T = (E+ c)^T for the tensor-core contractions: tile geometry
// and the two independent passes that fill the A operand in shared memory.
//
// A tile holds whole alpha-string rows of the CI vector: R rows x Cw columns
// (R = 1 and Cw <= 128 when nstr >= 128; else R = min(16, 128 / nstr) rows of
// all nstr columns).  Thread t owns determinant (ka0 + t / Cw, kb0 + t % Cw).
// Four threads share a determinant row; each owns 16-pair blocks of it and
// finds the alpha and beta excitations that land in its block through the
// per-string table of list offsets per 16-pair block (lists are sorted by
// pair).  The alpha part reads c[J_alpha][kb] with consecutive kb across a
// warp (coalesced), the beta part c[ka][J_beta] from one row; both parts of
// an element are summed in registers before its single conversion, and the
// block is written to shared memory as whole 16-byte chunks.
#pragma once
#include "sigma.cuh"

namespace ifci {
namespace tcg {

constexpr int kRows = 16;       // at most this many alpha rows per tile
constexpr int kTileDets = 128;

struct TileGeom {
    int ka0, kb0, R, Cw;
};

__host__ __device__ inline TileGeom tile_geom(long long start, int nstr) {
    TileGeom g;
    g.ka0 = (int)(start / nstr);
    g.kb0 = (int)(start % nstr);
    if (nstr >= kTileDets) {
        g.R = 1;
        g.Cw = nstr - g.kb0 < kTileDets ? nstr - g.kb0 : kTileDets;
    } else {
        int rmax = kTileDets / nstr;
        if (rmax > kRows) rmax = kRows;
        g.R = nstr - g.ka0 < rmax ? nstr - g.ka0 : rmax;
        g.Cw = nstr;
    }
    return g;
}

// Alpha rows one tile covers when a row is shorter than a tile (else 1).
inline int rows_per_tile(int nstr) {
    if (nstr >= kTileDets) return 1;
    const int rmax = kTileDets / nstr;
    return rmax > kRows ? kRows : rmax;
}

// Host: the row-aligned tiles of alpha rows [r0, r1) of one problem (all rows
// when r1 < 0), in order; r0 and r1 are multiples of rows_per_tile(nstr)
// (r1 may be nstr).
inline void append_row_tiles(std::vector<WorkItem> &out, int prob, int sub, int nstr, int r0 = 0, int r1 = -1) {
    if (r1 < 0) r1 = nstr;
    if (nstr >= kTileDets) {
        for (int ka = r0; ka < r1; ka++)
            for (int kb0 = 0; kb0 < nstr; kb0 += kTileDets)
                out.push_back(WorkItem{prob, sub, (long long)ka * nstr + kb0});
    } else {
        const int rmax = rows_per_tile(nstr);
        for (int ka0 = r0; ka0 < r1; ka0 += rmax) out.push_back(WorkItem{prob, sub, (long long)ka0 * nstr});
    }
}

// Dynamic tile scheduling of the persistent tensor-core kernels: the next tile
// whose problem is still active, from a global counter (ntile when none is
// left).  Called by one thread.
__device__ __forceinline__ int claim_tile(int *counter, const SigmaProb *probs, const WorkItem *tiles, int ntile) {
    while (true) {
        const int t = atomicAdd(counter, 1);
        if (t >= ntile) return ntile;
        const SigmaProb &p = probs[tiles[t].prob];
        if (!(p.active && !*p.active)) return t;
    }
}

inline long long row_tile_count(int nstr) {
    if (nstr >= kTileDets) return (long long)nstr * ((nstr + kTileDets - 1) / kTileDets);
    int rmax = kTileDets / nstr;
    if (rmax > kRows) rmax = kRows;
    return (nstr + rmax - 1) / rmax;
}

}  // namespace tcg
}  // namespace ifci

namespace ifci {
namespace tcg {

// Sum of the alpha and beta contributions of determinant (ka, kb) to the 16
// pairs [16 b, 16 b + 16): x[i] += sign * c.  T = float or long long.
template <typename T>
__device__ __forceinline__ void gather_block16(const SigmaProb &p, const T *__restrict__ c, int ka, int kb, int b,
                                               T (&x)[16]) {
    // padding block of the last atom (its pairs are beyond np): nothing to add,
    // and its end offset lies past the string's row of block offsets
    if (16 * b >= p.np) return;
    const int nstr = p.nstr, nexc = p.nexc;
    const uint8_t *ba = p.blk + (size_t)ka * kBlk16Stride, *bb = p.blk + (size_t)kb * kBlk16Stride;
    const int a0 = ba[b], a1 = ba[b + 1], b0 = bb[b], b1 = bb[b + 1];
    const int32_t *ea = p.exc + (size_t)ka * nexc, *eb = p.exc + (size_t)kb * nexc;
    const T *crow = c + (long long)ka * nstr;
    const int base = 16 * b;
    for (int e0 = a0; e0 < a1; e0 += 4) {
        int32_t xe[4];
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) xe[u] = e0 + u < a1 ? ea[e0 + u] : 0;
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = e0 + u < a1 ? c[(long long)exc_J(xe[u]) * nstr + kb] : T(0);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int i = exc_pair(xe[u]) - base;
            const T sv = (xe[u] & 1) ? -v[u] : v[u];
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] += (e0 + u < a1 && i == k) ? sv : T(0);
        }
    }
    for (int e0 = b0; e0 < b1; e0 += 4) {
        int32_t ye[4];
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) ye[u] = e0 + u < b1 ? eb[e0 + u] : 0;
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = e0 + u < b1 ? crow[exc_J(ye[u])] : T(0);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int i = exc_pair(ye[u]) - base;
            const T sv = (ye[u] & 1) ? -v[u] : v[u];
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] += (e0 + u < b1 && i == k) ? sv : T(0);
        }
    }
}

// Alpha part of the 16 pairs [16 b, 16 b + 16) of determinant (ka, kb) for a
// spin-flip-symmetric vector: each pair has at most one alpha excitation of
// ka, read from the dense pair map as the offset of +-c[J][0] in the quantised
// pair [c | -c] (C2), so an element is one predicated load and no arithmetic.
// Every thread of a tile row reads the same map row (a broadcast).  Split in
// two so that a kernel can fetch the map row of its next block early.
__device__ __forceinline__ void pmap_load16(const int32_t *__restrict__ pmap, int np, int ka, int b, int4 (&pm)[4]) {
    if (16 * b >= np) {   // padding block of the last atom: the map row ends before it
#pragma unroll
        for (int g = 0; g < 4; g++) pm[g] = make_int4(-1, -1, -1, -1);
        return;
    }
    const int4 *src = reinterpret_cast<const int4 *>(pmap + ((size_t)ka * pmap_ld(np) + 16 * b));
#pragma unroll
    for (int g = 0; g < 4; g++) pm[g] = src[g];
}

template <typename T>
__device__ __forceinline__ void gather_pm16(const T *__restrict__ C2, int kb, const int4 (&pm)[4], T (&x)[16]) {
#pragma unroll
    for (int g = 0; g < 4; g++) {
        const int e[4] = {pm[g].x, pm[g].y, pm[g].z, pm[g].w};
#pragma unroll
        for (int u = 0; u < 4; u++) x[4 * g + u] = e[u] >= 0 ? C2[(long long)e[u] + kb] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void gather_alpha16(const SigmaProb &p, const T *__restrict__ C2, int ka, int kb, int b,
                                               T (&x)[16]) {
    int4 pm[4];
    pmap_load16(p.pmap, p.np, ka, b, pm);
    gather_pm16<T>(C2, kb, pm, x);
}

}  // namespace tcg
}  // namespace ifci
