// FP64-accurate contraction G = W D on the FP16 tensor cores (tcgen05).
//
// GB300 runs FP64 at ~1/1800 of its 16-bit tensor rate, so the sigma builds
// that must be exact to FP64 level (Davidson restart vectors, final Rayleigh
// quotients) are emulated with integer slices (an Ozaki-style splitting):
//
//   W[A][B] = Wscale 2^-7 (w1 + 2^-8 w2 + ... + 2^-32 w5)    Wscale >= max|W|
//   D[B][K] = dscale  2^-6 (d1 + 2^-8 d2 + ... + 2^-32 d5)    dscale >= max|D|
//
// with every slice an integer in [-128, 128], exact in FP16.  D comes from the
// fixed-point copy round(c 2^38 / dscale) of the input vector (quantise_kernel),
// so the gather adds integers and the slices are the base-256 digits of
// X + 128 (1 + 2^8 + ... + 2^32) minus 128, turned into FP16 by a byte permute
// and one packed FP16 subtraction: no FP64 arithmetic in this kernel.
// The product of two slices over K <= 204 terms stays below 2^24 even when the (up to five)
// slice pairs of one scale level L = i + j share an accumulator, so each level
// is summed exactly by the tensor cores in FP32; a problem with more pairs is
// split into K chunks of 192 pairs, each its own tile, whose int64 partial
// sums are added into G (exact, in any order).  The 15 slice pairs with
// i + j <= 4 (0-based) are kept; the epilogue combines the five levels exactly
// in int64, G = 2^-45 Wscale dscale sum_L 2^{8 (4 - L)} acc_L, and stores the
// integer; the scatter sums those integers and converts once per determinant
// (no FP64 arithmetic in the hot loop).  The dropped terms and the slice
// truncation leave a relative error of order 2^-38 of max|W| max|D|.
//
// Tile: 128 determinants (TMEM lanes) x 96 output pairs; five accumulators
// of 96 FP32 columns (480 of the 512 TMEM columns).  K runs in 64-pair atoms:
// the W slices of the next atom (5 x 96 x 64 FP16, pre-swizzled image) arrive
// by bulk async copy into the second stage buffer while 512 threads (four per
// determinant) build the five D slices of the current atom, then one thread
// issues the 15 x 4 MMAs.  For spin-flip-symmetric vectors the gather reads
// the alpha excitations only (see sigma.cu): one pair-map lookup and one
// predicated load per element.
#include <cuda_fp16.h>

#include "sigma.cuh"
#include "tc_gather.cuh"
#include "tcgen05.cuh"

namespace ifci {

namespace {

using namespace tc;

constexpr int kS = 5;                       // slices per operand
constexpr int kNT = 96;                     // output pairs per tile
constexpr int kThreads = 512;               // 4 threads per determinant row
constexpr int kOzTmemCols = 512;
constexpr int kMaxNpExact = 204;            // exact level sums need at most 204 pairs per K chunk
constexpr int kMaxNpTable = 304;            // 16-pair block offsets per string (kBlk16Stride) cover 304 pairs
constexpr size_t kWStage = (size_t)kS * kNT * kAtomBytes;     // 61,440 B
constexpr size_t kAStage = (size_t)kS * kTM * kAtomBytes;     // 81,920 B
constexpr long long kDigitBias = 128ll * 0x0101010101ll;      // 128 in each of the five digits

__host__ __device__ inline int n_tiles(int np) { return (np + kNT - 1) / kNT; }

// slice a value in [-1, 1] into kS integers in [-128, 128]: x = 2^-7 sum_i 2^{-8i} s_i
__device__ __forceinline__ void slice5(double x, float (&sl)[kS]) {
    double r = x * 128.0;
#pragma unroll
    for (int i = 0; i < kS; i++) {
        double q = rint(r);
        sl[i] = (float)q;
        r = (r - q) * 256.0;
    }
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __half a = __float2half_rn(lo), b = __float2half_rn(hi);   // exact: |lo|, |hi| <= 128, integers
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// FP16 pair (u0 - 128, u1 - 128) of byte D of a and of b: the byte permute
// puts u into the low mantissa bits of the FP16 number 1024 (0x6400), which
// then reads 1024 + u exactly, and one packed subtraction of 1152 leaves
// u - 128 in [-128, 127] (exact).
__device__ __forceinline__ uint32_t digit_pair_f16(uint32_t a, uint32_t b, int D) {
    const uint32_t sel = D | (D << 4) | ((D + 4) << 8) | ((D + 4) << 12);   // a compile-time constant once unrolled
    const uint32_t t = (__byte_perm(a, b, sel) & 0x00FF00FFu) | 0x64006400u;
    __half2 v = *reinterpret_cast<const __half2 *>(&t);
    const __half2 off = __halves2half2(__ushort_as_half((unsigned short)0x6480), __ushort_as_half((unsigned short)0x6480));
    v = __hsub2(v, off);
    return *reinterpret_cast<uint32_t *>(&v);
}

// A tile's sub field: its first output pair (low 16 bits) and its K chunk (the
// atoms [kChunkAtoms kc, kChunkAtoms (kc + 1)), so that every level sum of a
// chunk stays an exact integer below 2^24 whatever npair is)
constexpr int kChunkAtoms = 3;   // 192 pairs per chunk
static_assert(kChunkAtoms * 64 <= kMaxNpExact, "a K chunk must keep its level sums exact");
__host__ __device__ inline int tile_n0(int sub) { return sub & 0xFFFF; }
__host__ __device__ inline int tile_kc(int sub) { return sub >> 16; }

// W stage of local atom la of tile t
__device__ __forceinline__ const uint8_t *stage_src(const SigmaProb *probs, const WorkItem *tiles, int t, int la) {
    const WorkItem tile = tiles[t];
    const SigmaProb &p = probs[tile.prob];
    const int KA = k_atoms(p.act ? p.npc : p.np), nt = tile_n0(tile.sub) / kNT;
    return (const uint8_t *)p.Woz + ((size_t)nt * KA + kChunkAtoms * tile_kc(tile.sub) + la) * kWStage;
}

// G[A][K] (int64, fixed point 2^-45 Wscale dscale) for one tile of 128 determinants x 96 pairs;
// for a row slab (kn > 0) G[A][K - k0] with row stride kn.
__global__ void __launch_bounds__(kThreads, 1)
oz_contract_kernel(const SigmaProb *__restrict__ probs, const WorkItem *__restrict__ tiles, int ntile,
                   const long long *__restrict__ Q, long long *__restrict__ G, int *__restrict__ err,
                   int *__restrict__ counter, long long k0, long long kn) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_w[2], bar_mma;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_tile, s_next;
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *Wsm0 = base;                   // two W stages: [slice i][kNT rows][128 B]
    uint8_t *Asm = base + 2 * kWStage;      // [slice j][128 rows][128 B]
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (kTM - 1), q = tid >> 7;   // determinant row of the tile, quarter
    const uint32_t bw0 = smem_u32(&bar_w[0]), bw1 = smem_u32(&bar_w[1]), bm = smem_u32(&bar_mma);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kOzTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bw0, 1);
        mbar_init(bw1, 1);
        mbar_init(bm, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // tiles are handed out by a global counter (dynamic load balance); the tile
    // after the current one is claimed early so that its first W stage can be
    // prefetched during the current tile's last atom
    uint32_t ph_m = 0;
    uint32_t g = 0;            // W stages consumed so far: buffer g & 1, phase (g >> 1) & 1
    bool ok = true;
    if (tid == 0) {
        const int t = tcg::claim_tile(counter, probs, tiles, ntile);
        s_tile = t;
        if (t < ntile) bulk_load(smem_u32(Wsm0), stage_src(probs, tiles, t, 0), (uint32_t)kWStage, bw0);
    }
    __syncthreads();
    for (int t = s_tile; t < ntile && ok;) {
        if (tid == 0) s_next = tcg::claim_tile(counter, probs, tiles, ntile);
        const WorkItem tile = tiles[t];
        // descriptor fields in registers (the asm memory clobbers below would
        // otherwise make the compiler reload them from global memory)
        const SigmaProb &pg = probs[tile.prob];
        // np: the pairs contracted (a sectored space: its active pairs, in compact order)
        const int np = pg.act ? pg.npc : pg.np, nstr = pg.nstr, sym = pg.sym;
        // G row stride: the problem's determinants, or those of its row slab [k0, k0 + kn)
        const long long gld = kn ? kn : pg.ndet, doff = pg.doff;
        const int32_t *pmap = pg.act ? pg.pmapc : pg.pmap;
        const int32_t *act = pg.act;
        const long long *C = Q + pg.qoff;   // round(c 2^38 / dscale) (and its negation when sym)
        const int KA = k_atoms(np), n0 = tile_n0(tile.sub);
        const int a0 = kChunkAtoms * tile_kc(tile.sub), a1 = min(KA, a0 + kChunkAtoms);
        const bool chunked = KA > kChunkAtoms;   // partial sums: added to G (zeroed before the launch)
        const int Nt = round_up(min(kNT, np - n0), 16);
        const tcg::TileGeom geo = tcg::tile_geom(tile.start, nstr);
        const bool live = row < geo.R * geo.Cw;
        const int r = live ? row / geo.Cw : 0;
        const int ka = geo.ka0 + r, kb = geo.kb0 + (live ? row % geo.Cw : 0);
        const long long K = (long long)ka * nstr + kb;
        int4 pmn[4];               // pair-map row of this thread's next block
        if (sym && live) tcg::pmap_load16(pmap, np, ka, 4 * a0 + q, pmn);
        for (int a = a0; a < a1; a++, g++) {
            // ---- loads of this atom's block (pairs 64a + 16q .. + 16): they overlap
            // the MMAs of the previous atom, which are still running
            const int b = 4 * a + q;
            long long x[16];
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = 0;
            if (live) {
                if (sym) {
                    int4 pmc[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) pmc[u] = pmn[u];
                    if (a + 1 < a1) tcg::pmap_load16(pmap, np, ka, b + 4, pmn);
                    tcg::gather_pm16<long long>(C, kb, pmc, x);
                } else {
                    tcg::gather_block16<long long>(probs[tile.prob], C, ka, kb, b, x);
                }
            }
            // MMAs of the previous atom done: A and W buffer (g + 1) & 1 are free
            // (thread 0 polls, the others wait at the barrier)
            if (a > a0) {
                if (!__syncthreads_and(tid == 0 ? (ok && mbar_wait(bm, ph_m)) : 1)) { ok = false; break; }
                ph_m ^= 1;
            }
            // prefetch the next W stage (thread 0 wrote s_next itself: no barrier needed to read it)
            if (tid == 0) {
                const int nt2 = a + 1 < a1 ? t : s_next, na = a + 1 < a1 ? a + 1 - a0 : 0;
                if (nt2 < ntile)
                    bulk_load(smem_u32(Wsm0 + ((g + 1) & 1) * kWStage), stage_src(probs, tiles, nt2, na),
                              (uint32_t)kWStage, ((g + 1) & 1) ? bw1 : bw0);
            }
            // ---- five digit slices of the block, two 16-byte chunks per slice
#pragma unroll
            for (int half = 0; half < 2; half++) {
                uint32_t lo[8], hi[8];
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    const unsigned long long Xb = (unsigned long long)(x[8 * half + e] + kDigitBias);
                    lo[e] = (uint32_t)Xb;
                    hi[e] = (uint32_t)(Xb >> 32);
                }
                const int ch = 2 * q + half;
                uint8_t *dst = Asm + row * kAtomBytes + ((ch ^ (row & 7)) << 4);
#pragma unroll
                for (int j = 0; j < kS; j++) {
                    const int d = kS - 1 - j;          // slice j = digit d (j = 0 most significant)
                    uint32_t w4[4];
#pragma unroll
                    for (int e = 0; e < 8; e += 2)
                        w4[e / 2] = d == 4 ? digit_pair_f16(hi[e], hi[e + 1], 0) : digit_pair_f16(lo[e], lo[e + 1], d);
                    *(uint4 *)(dst + (size_t)j * kTM * kAtomBytes) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            // ---- one thread: wait for this stage's W, issue the 15 x (up to 4) MMAs
            if (tid == 0) {
                ok = ok && mbar_wait((g & 1) ? bw1 : bw0, (g >> 1) & 1);
                if (ok) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t idesc = idesc_f16(kTM, Nt);
                    // descriptors of the stage bases; an offset below 256 KB adds (offset >> 4)
                    const uint64_t ad0 = smem_desc(smem_u32(Asm));
                    const uint64_t wd0 = smem_desc(smem_u32(Wsm0 + (g & 1) * kWStage));
                    const int kst = min(4, (round_up(np, 16) - a * 64) / 16);
#pragma unroll
                    for (int j = 0; j < kS; j++)
#pragma unroll
                        for (int i = 0; i + j < kS; i++)
#pragma unroll
                            for (int ks = 0; ks < 4; ks++)
                                if (ks < kst)
                                    mma_f16(tmem + (uint32_t)((i + j) * kNT),
                                            ad0 + (uint64_t)((j * kTM * kAtomBytes + ks * 32) >> 4),
                                            wd0 + (uint64_t)((i * kNT * kAtomBytes + ks * 32) >> 4), idesc,
                                            (a > a0 || j > 0 || ks > 0) ? 1u : 0u);
                    mma_commit(bm);
                }
            }
            __syncwarp();
        }
        // the MMAs of the tile's last atom (every thread reaches this barrier: a
        // failed vote above made all of them leave the atom loop together, and
        // thread 0 alone may hold ok = false from its W wait)
        if (!__syncthreads_and(tid == 0 ? (ok && mbar_wait(bm, ph_m)) : ok)) ok = false;
        ph_m ^= 1;
        if (!ok) break;
        // read before the closing barrier: thread 0 overwrites s_next after it
        const int t_next = s_next;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---- epilogue: the levels are exact integers below 2^24; combine them
        // in int64, G = sum_L acc_L 2^{8 (4 - L)}  (no FP64 arithmetic)
        long long *Gp = G + doff;
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        for (int c0 = 16 * (warp >> 2); c0 < Nt; c0 += 64) {
            long long gi[16];
#pragma unroll
            for (int j = 0; j < 16; j++) gi[j] = 0;
#pragma unroll
            for (int L = 0; L < kS; L++) {
                float v[16];
                tmem_ld16(tmem + lane_base + (uint32_t)(L * kNT + c0), v);
#pragma unroll
                for (int j = 0; j < 16; j++) gi[j] += (long long)__float2int_rn(v[j]) << (8 * (kS - 1 - L));
            }
            if (live) {
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int A = n0 + c0 + j;
                    if (c0 + j < Nt && A < np) {
                        long long *dst = Gp + (long long)(act ? act[A] : A) * gld + (K - k0);
                        if (chunked) atomicAdd(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)gi[j]);
                        else *dst = gi[j];
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        t = t_next;
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    // a prefetch may still be in flight after a timeout: wait for it (bounded)
    if (!ok) __syncthreads_and(mbar_wait((g & 1) ? bw1 : bw0, (g >> 1) & 1));
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzTmemCols)
                     : "memory");
}

// Sliced image of W: [tile nt][atom a][slice i][kNT rows][128 B], W scaled by
// 2^-e with one exponent per problem (max |W| <= 2^e, stored in Wexp[0]), the
// 16-byte chunk c of a row at c ^ (row % 8), zeros beyond npair.
__global__ void oz_pack_w_kernel(const SigmaProb *__restrict__ probs) {
    const SigmaProb &p = probs[blockIdx.x];
    // a sectored space packs only its active pairs, in compact order
    const int np = p.act ? p.npc : p.np, KA = k_atoms(np), NTl = n_tiles(np);
    const int32_t *act = p.act;
    uint8_t *img = (uint8_t *)const_cast<void *>(p.Woz);
    __shared__ double red[256];
    double mx = 0.0;
    for (long long i = threadIdx.x; i < (long long)np * np; i += blockDim.x) {
        const long long r = i / np, c = i % np;
        mx = fmax(mx, fabs(p.W[(act ? act[r] : r) * (long long)p.ld + (act ? act[c] : c)]));
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    int e = 0;
    if (red[0] > 0.0) frexp(red[0], &e);          // max = f 2^e, f in [0.5, 1)
    const double scale = ldexp(1.0, e);
    if (threadIdx.x == 0) p.Wexp[0] = scale;
    const int rows = NTl * kNT;
    for (int t = threadIdx.x; t < rows * KA * 8; t += blockDim.x) {
        const int n = t / (KA * 8), rest = t % (KA * 8), a = rest / 8, ch = rest % 8;
        const int nt = n / kNT, r = n % kNT;
        float sl[8][kS];
        for (int e2 = 0; e2 < 8; e2++) {
            const int k = a * 64 + ch * 8 + e2;
            double x = (n < np && k < np) ? p.W[(long long)(act ? act[n] : n) * p.ld + (act ? act[k] : k)] / scale
                                          : 0.0;
            slice5(x, sl[e2]);
        }
        for (int i = 0; i < kS; i++) {
            uint4 qv = make_uint4(pack2(sl[0][i], sl[1][i]), pack2(sl[2][i], sl[3][i]), pack2(sl[4][i], sl[5][i]),
                                  pack2(sl[6][i], sl[7][i]));
            size_t off = (((size_t)nt * KA + a) * kS + i) * (kNT * kAtomBytes) + (size_t)r * kAtomBytes +
                         ((ch ^ (r & 7)) << 4);
            *(uint4 *)(img + off) = qv;
        }
    }
}

// dscale = smallest power of two >= 2 max|c| (|D| <= 2 max|c|)
__global__ void oz_absmax_kernel(const double *__restrict__ c, long long n, unsigned long long *__restrict__ out) {
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(c[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void oz_set_dscale_kernel(SigmaProb *__restrict__ p, const unsigned long long *__restrict__ mx) {
    double m = __longlong_as_double((long long)*mx);
    int e = 0;
    if (m > 0.0) frexp(2.0 * m, &e);
    p->dscale = m > 0.0 ? ldexp(1.0, e) : 1.0;
}

}  // namespace

int oz_tile_n() { return kNT; }

int oz_operand_bytes(int np) {
    return (int)((size_t)n_tiles(np) * k_atoms(np) * kWStage + (size_t)np * 8 + 256);
}

int launch_oz_pack_w(ifci_handle_t h, int nprob, const SigmaProb *d_probs, cudaStream_t s) {
    if (nprob <= 0) return IFCI_OK;
    oz_pack_w_kernel<<<nprob, 256, 0, s>>>(d_probs);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_oz_dscale(ifci_handle_t h, SigmaProb *d_prob, const double *c, long long n, cudaStream_t s) {
    unsigned long long *mx = ws_take<unsigned long long>(h, 1);
    if (!mx) return set_error(h, IFCI_ERR_OOM, "FP64E: workspace (scale)");
    IFCI_CUDA_TRY(h, cudaMemsetAsync(mx, 0, sizeof(*mx), s));
    int blocks = (int)std::min<long long>(1024, (n + 255) / 256);
    oz_absmax_kernel<<<std::max(blocks, 1), 256, 0, s>>>(c, n, mx);
    IFCI_LAUNCH_CHECK(h);
    oz_set_dscale_kernel<<<1, 1, 0, s>>>(d_prob, mx);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_oz_contract(ifci_handle_t h, const SigmaPlan &plan, const SigmaWave &w, const void *Q, void *G,
                       cudaStream_t s) {
    if (w.ntc == 0) return IFCI_OK;
    for (const SigmaProb &p : plan.probs)
        if (p.np > kMaxNpTable)
            return set_error(h, IFCI_ERR_UNSUPPORTED, "FP64E: npair %d > %d", p.np, kMaxNpTable);
    // K chunks add their partial sums: zero those problems' G first
    for (int i = w.prob0; i < w.prob0 + w.nprob; i++) {
        const SigmaProb &p = plan.probs[i];
        if (k_atoms(p.act ? p.npc : p.np) > kChunkAtoms)
            IFCI_CUDA_TRY(h, cudaMemsetAsync(static_cast<long long *>(G) + p.doff, 0,
                                             (size_t)p.np * (w.kn ? w.kn : p.ndet) * 8, s));
    }
    if (!h->d_err || !h->d_counter) return set_error(h, IFCI_ERR_INVALID_ARG, "FP64E: no error flag / counter");
    const size_t smem = 1024 + 2 * kWStage + kAStage;   // 205,824 B
    static SmemOptIn opt;
    IFCI_CUDA_TRY(h, ensure_smem(opt, h->device, oz_contract_kernel, (int)smem));
    const int grid = std::min(w.ntc, device_sm_count(h->device));
    IFCI_CUDA_TRY(h, cudaMemsetAsync(h->d_counter, 0, sizeof(int), s));
    ProfScope ps(h, s, PK_CONTRACT_HI);
    oz_contract_kernel<<<grid, kThreads, smem, s>>>(plan.d_probs, plan.d_tctiles + w.tc0, w.ntc,
                                                    (const long long *)Q, (long long *)G, h->d_err, h->d_counter,
                                                    w.k0, w.kn);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

}  // namespace ifci
