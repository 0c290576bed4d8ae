// Tensor-core (tcgen05) contraction G = W D for the BF16 and TF32 paths, with
// the gather D = E+ c fused into the construction of the MMA's A operand.
//
// One tile = 128 determinants (the MMA's M, one TMEM lane each) x all npair
// output pairs (N <= 256 columns of FP32 in TMEM) x all npair input pairs (K).
//   A (M x K, K-major, SWIZZLE_128B) : D^T rows, built in shared memory by
//       512 threads, four per determinant, from the sorted alpha/beta
//       excitation lists (no atomics, one rounding per element); for
//       spin-flip-symmetric vectors from the alpha pair map only (sigma.cu)
//   B (N x K, K-major, SWIZZLE_128B) : the folded integrals W of the
//       problem, a pre-swizzled BF16 image copied with one bulk async copy
//       (cp.async.bulk) whenever the CTA moves to a new problem
//   D (M x N, FP32, TMEM)            : G^T of the tile; the epilogue reads it
//       with tcgen05.ld (one determinant per thread) and stores G[A][K] so
//       that a warp writes 32 consecutive determinants per pair.
// CTAs are persistent and claim tiles from a global counter; the tiles of a
// problem are consecutive, so W is reloaded mostly at problem boundaries.  Every mbarrier wait is bounded; on a timeout the
// kernel records an error flag, frees its TMEM and returns.
#include "sigma.cuh"
#include "tc_gather.cuh"
#include "tcgen05.cuh"

namespace ifci {

namespace {

using namespace tc;

constexpr int kBfThreads = 512;   // four threads per determinant row

__global__ void __launch_bounds__(kBfThreads, 1)
tc_contract_bf16_kernel(const SigmaProb *__restrict__ probs, const WorkItem *__restrict__ tiles, int ntile,
                        size_t w_bytes_max, size_t a_bytes_max, const float *__restrict__ Q,
                        float *__restrict__ G, int *__restrict__ err, int *__restrict__ counter) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_w, bar_mma;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_tile, s_next;
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *Wsm = base;
    uint8_t *Asm = base + ((w_bytes_max + 1023) & ~(size_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (kTM - 1), q = tid >> 7;            // determinant row, quarter
    const uint32_t bw = smem_u32(&bar_w), bm = smem_u32(&bar_mma);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
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

    // tiles are handed out by a global counter (dynamic load balance; the
    // tiles of a problem are consecutive, so W is reloaded only when the
    // claimed tile belongs to another problem)
    int cur = -1;
    uint32_t ph_w = 0, ph_m = 0;
    bool ok = true;
    if (tid == 0) s_tile = tcg::claim_tile(counter, probs, tiles, ntile);
    __syncthreads();
    for (int t = s_tile; t < ntile && ok;) {
        if (tid == 0) s_next = tcg::claim_tile(counter, probs, tiles, ntile);
        const WorkItem tile = tiles[t];
        const SigmaProb &p = probs[tile.prob];
        const int np = p.np, N = n_pad(np), KA = k_atoms(np), KS = round_up(np, 16) / 16;
        const int nstr = p.nstr;
        const tcg::TileGeom geo = tcg::tile_geom(tile.start, nstr);
        if (tile.prob != cur) {
            if (tid == 0) bulk_load(smem_u32(Wsm), p.Wtc, (uint32_t)(KA * N * kAtomBytes), bw);
            // block-wide vote so that every thread leaves the loop together
            if (!__syncthreads_and(mbar_wait(bw, ph_w))) { ok = false; break; }
            ph_w ^= 1;
            cur = tile.prob;
        }
        // ---- fused gather: row `row` of A = D^T of determinant K; thread q owns the
        // 16-pair blocks q, q + 4, ... and writes them as whole 16-byte chunks
        const bool live = row < geo.R * geo.Cw;
        const int r = live ? row / geo.Cw : 0;
        const int ka = geo.ka0 + r, kb = geo.kb0 + (live ? row % geo.Cw : 0);
        const long long K = (long long)ka * nstr + kb;
        const float *c = Q + p.qoff;   // FP32 copy of the input vector
        for (int b = q; b < KA * 4; b += 4) {
            float x[16];
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = 0.0f;
            if (live) {
                if (p.sym) tcg::gather_alpha16<float>(p, c, ka, kb, b, x);
                else tcg::gather_block16<float>(p, c, ka, kb, b, x);
            }
#pragma unroll
            for (int half = 0; half < 2; half++) {
                const int ch = 2 * (b & 3) + half;   // chunk within the atom
                uint4 w = make_uint4(pack_bf16x2f(x[8 * half + 0], x[8 * half + 1]),
                                     pack_bf16x2f(x[8 * half + 2], x[8 * half + 3]),
                                     pack_bf16x2f(x[8 * half + 4], x[8 * half + 5]),
                                     pack_bf16x2f(x[8 * half + 6], x[8 * half + 7]));
                *(uint4 *)(Asm + (b >> 2) * (kTM * kAtomBytes) + row * kAtomBytes + ((ch ^ (row & 7)) << 4)) = w;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // ---- MMA issue (one thread)
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = idesc_bf16(kTM, N);
            const uint32_t a0 = smem_u32(Asm), b0 = smem_u32(Wsm);
            for (int ks = 0; ks < KS; ks++) {
                const uint32_t koff = (uint32_t)((ks & 3) * 32);   // 16 BF16 = 32 B inside the atom
                const uint32_t aaddr = a0 + (uint32_t)(ks >> 2) * (kTM * kAtomBytes) + koff;
                const uint32_t baddr = b0 + (uint32_t)(ks >> 2) * (uint32_t)(N * kAtomBytes) + koff;
                mma_f16(tmem, smem_desc(aaddr), smem_desc(baddr), idesc, ks > 0 ? 1u : 0u);
            }
            mma_commit(bm);
        }
        __syncwarp();
        if (!__syncthreads_and(mbar_wait(bm, ph_m))) { ok = false; break; }
        ph_m ^= 1;
        // read before the closing barrier: thread 0 overwrites s_next after it
        const int t_next = s_next;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---- epilogue: TMEM -> G[A][K]; warps sharing a TMEM lane quarter split the columns
        float *Gp = G + p.doff;
        const long long ndet = p.ndet;
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        for (int c0 = 16 * (warp >> 2); c0 < N; c0 += 64) {
            float v[16];
            tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
            if (live) {
#pragma unroll
                for (int j = 0; j < 16; j++)
                    if (c0 + j < np) Gp[(long long)(c0 + j) * ndet + K] = v[j];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        t = t_next;
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// BF16 image of W in the B-operand layout: [atom a][row n < N][128 B], the
// 16-byte chunk c of row n stored at chunk c ^ (n % 8); zero padding.
__global__ void pack_w_bf16_kernel(const SigmaProb *__restrict__ probs) {
    const SigmaProb &p = probs[blockIdx.x];
    const int np = p.np, N = n_pad(np), KA = k_atoms(np);
    uint8_t *img = (uint8_t *)const_cast<void *>(p.Wtc);
    for (int t = threadIdx.x; t < N * KA * 8; t += blockDim.x) {
        const int n = t / (KA * 8), ch = t % (KA * 8);
        uint32_t pk[4];
        for (int e = 0; e < 8; e += 2) {
            int k0 = ch * 8 + e, k1 = k0 + 1;
            double v0 = (n < np && k0 < np) ? p.W[(long long)n * p.ld + k0] : 0.0;
            double v1 = (n < np && k1 < np) ? p.W[(long long)n * p.ld + k1] : 0.0;
            pk[e / 2] = pack_bf16x2(v0, v1);
        }
        const int a = ch >> 3, cc = ch & 7;
        uint4 *dst = (uint4 *)(img + (size_t)a * N * kAtomBytes + (size_t)n * kAtomBytes + ((cc ^ (n & 7)) << 4));
        *dst = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

// ---------------------------------------------------------------- TF32
// The same contraction with TF32 operands (kind::tf32, K = 8 per MMA): a
// 128-byte swizzle atom holds 32 pairs, so A (128 x npair FP32, built whole
// by the fused gather) and W no longer both fit in shared memory for npair
// above ~170; W streams through two atom stages by bulk async copy instead
// (W stays in L2: every tile reads the same image).  Both operands are
// rounded to TF32 with cvt.rna (to nearest, ties away from zero); the
// tensor cores accumulate in FP32.
constexpr int kTfAtomPairs = 32;
__host__ __device__ inline int tf_atoms(int np) { return (np + kTfAtomPairs - 1) / kTfAtomPairs; }

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Instruction descriptor, kind::tf32: TF32 x TF32 -> FP32, A and B K-major.
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
    return (1u << 4)                      // D format FP32
         | (2u << 7)                      // A format TF32
         | (2u << 10)                     // B format TF32
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__global__ void __launch_bounds__(kBfThreads, 1)
tc_contract_tf32_kernel(const SigmaProb *__restrict__ probs, const WorkItem *__restrict__ tiles, int ntile,
                        size_t w_stage_max, const float *__restrict__ Q, float *__restrict__ G,
                        int *__restrict__ err, int *__restrict__ counter) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_w[2], bar_free[2], bar_mma;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_tile, s_next;
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const size_t wst = (w_stage_max + 1023) & ~(size_t)1023;
    uint8_t *Wsm = base;                    // two stages of one W atom: [row n < N][128 B]
    uint8_t *Asm = base + 2 * wst;          // [atom][128 rows][128 B]
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (kTM - 1), q = tid >> 7;
    const uint32_t bw[2] = {smem_u32(&bar_w[0]), smem_u32(&bar_w[1])};
    const uint32_t bf[2] = {smem_u32(&bar_free[0]), smem_u32(&bar_free[1])};
    const uint32_t bm = smem_u32(&bar_mma);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bw[0], 1);
        mbar_init(bw[1], 1);
        mbar_init(bf[0], 1);
        mbar_init(bf[1], 1);
        mbar_init(bm, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // completions seen per stage barrier (thread 0 only): the next wait's parity
    uint32_t nw[2] = {0, 0}, nf[2] = {0, 0}, ni[2] = {0, 0};   // waits, commits, loads issued
    uint32_t ph_m = 0;
    bool ok = true;
    if (tid == 0) s_tile = tcg::claim_tile(counter, probs, tiles, ntile);
    __syncthreads();
    for (int t = s_tile; t < ntile && ok;) {
        if (tid == 0) s_next = tcg::claim_tile(counter, probs, tiles, ntile);
        const WorkItem tile = tiles[t];
        const SigmaProb &p = probs[tile.prob];
        const int np = p.np, N = n_pad(np), KA = tf_atoms(np), KS = round_up(np, 8) / 8;
        const uint32_t wbytes = (uint32_t)(N * kAtomBytes);
        const uint8_t *wimg = (const uint8_t *)p.Wtc;
        // the first two W atoms of the tile start loading while the gather runs
        // (both stages are free: the previous tile's MMAs have completed)
        if (tid == 0)
            for (int a = 0; a < 2 && a < KA; a++) {
                bulk_load(smem_u32(Wsm + a * wst), wimg + (size_t)a * wbytes, wbytes, bw[a]);
                ni[a]++;
            }
        const int nstr = p.nstr;
        const tcg::TileGeom geo = tcg::tile_geom(tile.start, nstr);
        const bool live = row < geo.R * geo.Cw;
        const int r = live ? row / geo.Cw : 0;
        const int ka = geo.ka0 + r, kb = geo.kb0 + (live ? row % geo.Cw : 0);
        const long long K = (long long)ka * nstr + kb;
        const float *c = Q + p.qoff;
        // ---- fused gather: 16-pair block b is half of atom b / 2 (four 16-byte chunks)
        for (int b = q; b < KA * 2; b += 4) {
            float x[16];
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = 0.0f;
            if (live) {
                if (p.sym) tcg::gather_alpha16<float>(p, c, ka, kb, b, x);
                else tcg::gather_block16<float>(p, c, ka, kb, b, x);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int ch = 4 * (b & 1) + u;
                uint4 w = make_uint4(tf32_rna(x[4 * u]), tf32_rna(x[4 * u + 1]), tf32_rna(x[4 * u + 2]),
                                     tf32_rna(x[4 * u + 3]));
                *(uint4 *)(Asm + (b >> 1) * (kTM * kAtomBytes) + row * kAtomBytes + ((ch ^ (row & 7)) << 4)) = w;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // ---- one thread: per atom, wait for its W stage, issue its MMAs, and
        // refill the stage with atom a + 2 once those MMAs have read it
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = idesc_tf32(kTM, N);
            const uint32_t a0 = smem_u32(Asm);
            for (int a = 0; a < KA && ok; a++) {
                const int st = a & 1;
                ok = mbar_wait(bw[st], nw[st] & 1);
                if (!ok) break;
                nw[st]++;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t b0 = smem_u32(Wsm + st * wst);
                for (int ks = 4 * a; ks < KS && ks < 4 * a + 4; ks++) {
                    const uint32_t koff = (uint32_t)((ks & 3) * 32);   // 8 TF32 = 32 B inside the atom
                    mma_tf32(tmem, smem_desc(a0 + (uint32_t)a * (kTM * kAtomBytes) + koff), smem_desc(b0 + koff),
                             idesc, ks > 0 ? 1u : 0u);
                }
                if (a + 2 < KA) {
                    mma_commit(bf[st]);
                    ok = mbar_wait(bf[st], nf[st] & 1);
                    nf[st]++;
                    if (ok) {
                        bulk_load(smem_u32(Wsm + st * wst), wimg + (size_t)(a + 2) * wbytes, wbytes, bw[st]);
                        ni[st]++;
                    }
                }
            }
            mma_commit(bm);
        }
        __syncwarp();
        // every thread leaves together; thread 0 alone may hold ok = false
        if (!__syncthreads_and(tid == 0 ? (ok && mbar_wait(bm, ph_m)) : 1)) { ok = false; break; }
        ph_m ^= 1;
        const int t_next = s_next;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float *Gp = G + p.doff;
        const long long ndet = p.ndet;
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        for (int c0 = 16 * (warp >> 2); c0 < N; c0 += 64) {
            float v[16];
            tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
            if (live) {
#pragma unroll
                for (int j = 0; j < 16; j++)
                    if (c0 + j < np) Gp[(long long)(c0 + j) * ndet + K] = v[j];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        t = t_next;
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    // W copies still in flight after a timeout: wait for them (bounded) before leaving
    if (!ok && tid == 0)
        for (int st = 0; st < 2; st++)
            for (; nw[st] < ni[st]; nw[st]++) (void)mbar_wait(bw[st], nw[st] & 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// TF32 image of W: [atom a][row n < N][128 B], 32 pairs per atom row, the
// 16-byte chunk c of row n stored at chunk c ^ (n % 8); zero padding.
__global__ void pack_w_tf32_kernel(const SigmaProb *__restrict__ probs) {
    const SigmaProb &p = probs[blockIdx.x];
    const int np = p.np, N = n_pad(np), KA = tf_atoms(np);
    uint8_t *img = (uint8_t *)const_cast<void *>(p.Wtc);
    for (int t = threadIdx.x; t < N * KA * 8; t += blockDim.x) {
        const int n = t / (KA * 8), ch = t % (KA * 8);
        uint32_t pk[4];
        for (int e = 0; e < 4; e++) {
            const int k = ch * 4 + e;
            pk[e] = tf32_rna((n < np && k < np) ? (float)p.W[(long long)n * p.ld + k] : 0.0f);
        }
        const int a = ch >> 3, cc = ch & 7;
        uint4 *dst = (uint4 *)(img + (size_t)a * N * kAtomBytes + (size_t)n * kAtomBytes + ((cc ^ (n & 7)) << 4));
        *dst = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

size_t tc_smem_bytes(int max_np) {
    size_t w = (size_t)k_atoms(max_np) * n_pad(max_np) * kAtomBytes;
    size_t a = (size_t)k_atoms(max_np) * kTM * kAtomBytes;
    return 1024 + ((w + 1023) & ~(size_t)1023) + a;
}

}  // namespace

int tc_supported(int precision) { return (precision == IFCI_BF16 || precision == IFCI_TF32) ? 1 : 0; }

int tc_operand_bytes(int np, int precision) {
    return (precision == IFCI_TF32 ? tf_atoms(np) : k_atoms(np)) * n_pad(np) * kAtomBytes;
}

int launch_tc_pack_w(ifci_handle_t h, int nprob, const SigmaProb *d_probs, int precision, cudaStream_t s) {
    if (!tc_supported(precision)) return set_error(h, IFCI_ERR_UNSUPPORTED, "tensor-core precision %d", precision);
    if (nprob <= 0) return IFCI_OK;
    if (precision == IFCI_TF32) pack_w_tf32_kernel<<<nprob, 256, 0, s>>>(d_probs);
    else pack_w_bf16_kernel<<<nprob, 256, 0, s>>>(d_probs);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_tc_contract(ifci_handle_t h, const SigmaPlan &plan, const SigmaWave &w, int precision, const void *D,
                       void *G, cudaStream_t s) {
    // D holds the FP32 copies of the input vectors (quantise_kernel)
    if (!tc_supported(precision)) return set_error(h, IFCI_ERR_UNSUPPORTED, "tensor-core precision %d", precision);
    if (w.ntc == 0) return IFCI_OK;
    int max_np = 0;
    for (const SigmaProb &p : plan.probs) max_np = std::max(max_np, p.np);
    if (max_np > 256) return set_error(h, IFCI_ERR_UNSUPPORTED, "tensor-core path: npair %d > 256", max_np);
    if (!h->d_err) return set_error(h, IFCI_ERR_INVALID_ARG, "tensor-core path: no error flag");
    if (!h->d_counter) return set_error(h, IFCI_ERR_INVALID_ARG, "tensor-core path: no tile counter");
    if (precision == IFCI_TF32) {
        // two W atom stages + the whole A tile; at least 116 KB so that one CTA runs per SM
        const size_t wst = (size_t)n_pad(max_np) * kAtomBytes;
        const size_t smem = std::max(1024 + 2 * ((wst + 1023) & ~(size_t)1023) +
                                         (size_t)tf_atoms(max_np) * kTM * kAtomBytes,
                                     (size_t)116 * 1024);
        static SmemOptIn opt_tf;
        IFCI_CUDA_TRY(h, ensure_smem(opt_tf, h->device, tc_contract_tf32_kernel, (int)smem));
        const int grid = std::min(w.ntc, device_sm_count(h->device));
        IFCI_CUDA_TRY(h, cudaMemsetAsync(h->d_counter, 0, sizeof(int), s));
        ProfScope ps(h, s, PK_CONTRACT);
        tc_contract_tf32_kernel<<<grid, kBfThreads, smem, s>>>(plan.d_probs, plan.d_tctiles + w.tc0, w.ntc, wst,
                                                               (const float *)D, (float *)G, h->d_err, h->d_counter);
        IFCI_LAUNCH_CHECK(h);
        return IFCI_OK;
    }
    // at least 116 KB of shared memory: one CTA per SM, so TMEM allocation never waits
    const size_t smem = std::max(tc_smem_bytes(max_np), (size_t)116 * 1024);
    const size_t wmax = (size_t)k_atoms(max_np) * n_pad(max_np) * kAtomBytes;
    const size_t amax = (size_t)k_atoms(max_np) * kTM * kAtomBytes;
    static SmemOptIn opt;
    IFCI_CUDA_TRY(h, ensure_smem(opt, h->device, tc_contract_bf16_kernel, (int)smem));
    const int grid = std::min(w.ntc, device_sm_count(h->device));
    IFCI_CUDA_TRY(h, cudaMemsetAsync(h->d_counter, 0, sizeof(int), s));
    ProfScope ps(h, s, PK_CONTRACT);
    tc_contract_bf16_kernel<<<grid, kBfThreads, smem, s>>>(plan.d_probs, plan.d_tctiles + w.tc0, w.ntc, wmax, amax,
                                                    (const float *)D, (float *)G, h->d_err, h->d_counter);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

}  // namespace ifci
