// FP64-accurate contraction G = W D on BF16 tensor cores (tcgen05).
//
// GB300 runs FP64 at ~1/1800 of its BF16 tensor rate, so the sigma builds
// that must be exact to FP64 level (Davidson restart vectors, final Rayleigh
// quotients) are emulated with integer slices (an Ozaki-style splitting):
//
//   W[A][B] = 2^{e_A} 2^-7 (w1 + 2^-8 w2 + ... + 2^-32 w5)    per output row A
//   D[B][K] = dscale  2^-7 (d1 + 2^-8 d2 + ... + 2^-32 d5)    dscale >= max|D|
//
// with every slice an integer in [-128, 128], exact in BF16.  The product of
// two slices over K <= 204 terms stays below 2^24 even when the (up to five)
// slice pairs of one scale level L = i + j share an accumulator, so each level
// is summed exactly by the tensor cores in FP32.  The 15 slice pairs with
// i + j <= 4 (0-based) are kept; the epilogue combines the five levels in
// FP64: G = 2^{e_A} dscale 2^-14 sum_L 2^{-8L} acc_L.  The dropped terms and
// the slice truncation leave a relative error of order 2^-38 of max|W| max|D|.
//
// Tile: 128 determinants (TMEM lanes) x 96 output pairs; five accumulators
// of 96 FP32 columns (480 of the 512 TMEM columns).  K runs in 64-pair atoms:
// for each atom the W slices (5 x 96 x 64 BF16, pre-swizzled image) arrive by
// one bulk async copy while the 128 threads build the five D slices of their
// determinants (fused gather), then one thread issues the 15 x 4 MMAs.
#include "sigma.cuh"
#include "tcgen05.cuh"

namespace ifci {

namespace {

using namespace tc;

constexpr int kS = 5;                       // slices per operand
constexpr int kNT = 96;                     // output pairs per tile
constexpr int kOzTmemCols = 512;
constexpr int kMaxNpExact = 204;            // exact level sums need npair <= 204
constexpr size_t kWStage = (size_t)kS * kNT * kAtomBytes;     // 61,440 B
constexpr size_t kAStage = (size_t)kS * kTM * kAtomBytes;     // 81,920 B

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
    __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);   // exact: |lo|, |hi| <= 128, integers
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__global__ void __launch_bounds__(kTM, 1)
oz_contract_kernel(const SigmaProb *__restrict__ probs, const WorkItem *__restrict__ tiles, int ntile,
                   double *__restrict__ G, int *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_w, bar_mma;
    __shared__ uint32_t tmem_slot;
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *Wsm = base;                    // [slice i][kNT rows][128 B]
    uint8_t *Asm = base + kWStage;          // [slice j][128 rows][128 B]
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t bw = smem_u32(&bar_w), bm = smem_u32(&bar_mma);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kOzTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bw, 1);
        mbar_init(bm, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    const int per = (ntile + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * per, t1 = min(ntile, t0 + per);
    uint32_t ph_w = 0, ph_m = 0;
    bool ok = true;
    for (int t = t0; t < t1 && ok; t++) {
        const WorkItem tile = tiles[t];
        const SigmaProb &p = probs[tile.prob];
        if (p.active && !*p.active) continue;
        const int np = p.np, KA = k_atoms(np), n0 = tile.sub, nt = n0 / kNT;
        const int Nt = round_up(min(kNT, np - n0), 16);
        const long long ndet = p.ndet;
        const long long K = tile.start + tid;
        const bool live = K < ndet;
        const int nstr = p.nstr, nexc = p.nexc;
        const int ka = live ? (int)(K / nstr) : 0, kb = live ? (int)(K % nstr) : 0;
        const double *c = p.cbase + (p.cslot ? (long long)*p.cslot : 0ll) * p.stride;
        const int32_t *ea = p.exc + (size_t)ka * nexc;
        const int32_t *eb = p.exc + (size_t)kb * nexc;
        const double *crow = c + (long long)ka * nstr;
        const double inv_ds = 1.0 / p.dscale;
        int ia = 0, ib = 0;
        int32_t xa = live ? ea[0] : 0, xb = live ? eb[0] : 0;
        int pa = live ? exc_pair(xa) : -1, pb = live ? exc_pair(xb) : -1;
        uint32_t started = 0;   // accumulator levels already written in this tile
        const uint8_t *wimg = (const uint8_t *)p.Woz + (size_t)nt * KA * kWStage;
        for (int a = 0; a < KA && ok; a++) {
            if (tid == 0) bulk_load(smem_u32(Wsm), wimg + (size_t)a * kWStage, (uint32_t)kWStage, bw);
            // ---- fused gather of pairs [64a, 64a + 64) and slicing into kS BF16 atoms
            uint8_t *row = Asm + tid * kAtomBytes;
            for (int ch = 0; ch < 8; ch++) {
                float sl[8][kS];
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    const int A = a * 64 + ch * 8 + e;
                    double v = 0.0;
                    if (pa == A) {
                        v += exc_sign(xa) * c[(long long)exc_J(xa) * nstr + kb];
                        if (++ia < nexc) { xa = ea[ia]; pa = exc_pair(xa); } else pa = -1;
                    }
                    if (pb == A) {
                        v += exc_sign(xb) * crow[exc_J(xb)];
                        if (++ib < nexc) { xb = eb[ib]; pb = exc_pair(xb); } else pb = -1;
                    }
                    slice5(v * inv_ds, sl[e]);
                }
                const int sw = (ch ^ (tid & 7)) << 4;
#pragma unroll
                for (int j = 0; j < kS; j++) {
                    uint4 q = make_uint4(pack2(sl[0][j], sl[1][j]), pack2(sl[2][j], sl[3][j]),
                                         pack2(sl[4][j], sl[5][j]), pack2(sl[6][j], sl[7][j]));
                    *(uint4 *)(row + (size_t)j * kTM * kAtomBytes + sw) = q;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (!__syncthreads_and(mbar_wait(bw, ph_w))) { ok = false; break; }
            ph_w ^= 1;
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t idesc = idesc_bf16(kTM, Nt);
                const uint32_t a0 = smem_u32(Asm), w0 = smem_u32(Wsm);
                const int kst = min(4, (round_up(np, 16) - a * 64) / 16);
                for (int j = 0; j < kS; j++) {
                    for (int i = 0; i + j < kS; i++) {
                        const int L = i + j;
                        for (int ks = 0; ks < kst; ks++) {
                            const uint32_t acc = (started >> L) & 1u;
                            mma_bf16(tmem + (uint32_t)(L * kNT),
                                     smem_desc(a0 + (uint32_t)(j * kTM * kAtomBytes + ks * 32)),
                                     smem_desc(w0 + (uint32_t)(i * kNT * kAtomBytes + ks * 32)), idesc, acc);
                            started |= 1u << L;
                        }
                    }
                }
                mma_commit(bm);
            }
            __syncwarp();
            if (!__syncthreads_and(mbar_wait(bm, ph_m))) { ok = false; break; }
            ph_m ^= 1;
        }
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---- epilogue: combine the levels in FP64, scale, store G[A][K]
        double *Gp = G + p.doff;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        const double ds = p.dscale * (1.0 / 16384.0);
        for (int c0 = 0; c0 < Nt; c0 += 16) {
            double g[16];
#pragma unroll
            for (int j = 0; j < 16; j++) g[j] = 0.0;
            double wL = 1.0;
#pragma unroll
            for (int L = 0; L < kS; L++) {
                float v[16];
                tmem_ld16(tmem + lane_base + (uint32_t)(L * kNT + c0), v);
#pragma unroll
                for (int j = 0; j < 16; j++) g[j] += wL * (double)v[j];
                wL *= 1.0 / 256.0;
            }
            if (live) {
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int A = n0 + c0 + j;
                    if (c0 + j < Nt && A < np && A < n0 + kNT) Gp[(long long)A * ndet + K] = g[j] * ds * p.Wexp[A];
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzTmemCols)
                     : "memory");
}

// Sliced image of W: [tile nt][atom a][slice i][kNT rows][128 B], rows n0 + r
// of W scaled by 2^-e (e: smallest power with max_k |W[n][k]| <= 2^e), the
// 16-byte chunk c of a row at c ^ (row % 8), zeros beyond npair.
__global__ void oz_pack_w_kernel(const SigmaProb *__restrict__ probs) {
    const SigmaProb &p = probs[blockIdx.x];
    const int np = p.np, KA = k_atoms(np), NTl = n_tiles(np);
    uint8_t *img = (uint8_t *)const_cast<void *>(p.Woz);
    for (int n = threadIdx.x; n < np; n += blockDim.x) {
        double mx = 0.0;
        for (int k = 0; k < np; k++) mx = fmax(mx, fabs(p.W[(long long)n * p.ld + k]));
        int e = 0;
        if (mx > 0.0) frexp(mx, &e);          // mx = f 2^e, f in [0.5, 1)
        p.Wexp[n] = ldexp(1.0, e);
    }
    __syncthreads();
    const int rows = NTl * kNT;
    for (int t = threadIdx.x; t < rows * KA * 8; t += blockDim.x) {
        const int n = t / (KA * 8), rest = t % (KA * 8), a = rest / 8, ch = rest % 8;
        const int nt = n / kNT, r = n % kNT;
        float sl[8][kS];
        for (int e = 0; e < 8; e++) {
            const int k = a * 64 + ch * 8 + e;
            double x = (n < np && k < np) ? p.W[(long long)n * p.ld + k] / p.Wexp[n] : 0.0;
            slice5(x, sl[e]);
        }
        for (int i = 0; i < kS; i++) {
            uint4 q = make_uint4(pack2(sl[0][i], sl[1][i]), pack2(sl[2][i], sl[3][i]), pack2(sl[4][i], sl[5][i]),
                                 pack2(sl[6][i], sl[7][i]));
            size_t off = (((size_t)nt * KA + a) * kS + i) * (kNT * kAtomBytes) + (size_t)r * kAtomBytes +
                         ((ch ^ (r & 7)) << 4);
            *(uint4 *)(img + off) = q;
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

int launch_oz_contract(ifci_handle_t h, const SigmaPlan &plan, const SigmaWave &w, void *G, cudaStream_t s) {
    if (w.ntc == 0) return IFCI_OK;
    for (const SigmaProb &p : plan.probs)
        if (p.np > kMaxNpExact)
            return set_error(h, IFCI_ERR_UNSUPPORTED, "FP64E: npair %d > %d (exact level sums)", p.np, kMaxNpExact);
    if (!h->d_err) return set_error(h, IFCI_ERR_INVALID_ARG, "FP64E: no error flag");
    const size_t smem = 1024 + kWStage + kAStage;
    static bool configured = false;
    if (!configured) {
        IFCI_CUDA_TRY(h, cudaFuncSetAttribute(oz_contract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        configured = true;
    }
    const int grid = std::min(w.ntc, device_sm_count(h->device));
    ProfScope ps(h, s, PK_CONTRACT);
    oz_contract_kernel<<<grid, kTM, smem, s>>>(plan.d_probs, plan.d_tctiles + w.tc0, w.ntc, (double *)G, h->d_err);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

}  // namespace ifci
