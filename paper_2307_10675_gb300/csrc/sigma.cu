// Sigma build sigma = H c for a batch of CI problems (Knowles–Handy-style
// resolution of the identity over singly excited determinants):
//
//   D[A][K] = <K| E+_A |c>          gather over K's own alpha and beta excitations
//   G[A][K] = sum_B W[A][B] D[B][K]  dense contraction (W folds h1 into the ERIs)
//   sigma_I = sum_A <I| E+_A |K> G[A][K]   gather over I's own excitations
//
// E+_pq = E_pq + E_qp (p != q), E+_pp = E_pp.  Each string's excitation list
// holds at most one entry per pair, sorted by pair, so D rows are built by a
// merge of the alpha and beta lists with no atomics, and sigma is a gather.
// D and G are pair-major planes [A][K] so that the alpha parts (whole rows
// c[J_alpha][:]) are read and written with consecutive K across a warp.
//
// Spin-flip-symmetric vectors (C = C^T, the singlet sector the Davidson
// solver works in): with X_A the (symmetric) string matrix of E+_A, the beta
// part of D is the transpose of the alpha part, D_beta[A] = C X_A = (X_A C)^T,
// so G = G_a + G_a^T with G_a = W D_alpha, and
//   sigma = sum_A X_A G[A] + G[A] X_A = S + S^T,  S = sum_A X_A G_a[A] + G_a[A] X_A.
// The tensor-core paths then gather alpha excitations only (every thread of
// a tile row shares one alpha list, read from a dense pair map), run the
// unchanged scatter on G_a to get S, and add the transpose of S.
#include <algorithm>

#include "sigma.cuh"
#include "tc_gather.cuh"

namespace ifci {

size_t sigma_elem_bytes(int precision) { return (precision == IFCI_FP64 || precision == IFCI_FP64E) ? 8 : 4; }

template <typename TD>
__global__ void __launch_bounds__(kGatherChunk)
gather_kernel(const SigmaProb *__restrict__ probs, const WorkItem *__restrict__ items, TD *__restrict__ D) {
    const WorkItem it = items[blockIdx.x];
    const SigmaProb &p = probs[it.prob];
    if (p.active && !*p.active) return;
    const long long K = it.start + threadIdx.x;
    if (K >= p.ndet) return;
    const int nstr = p.nstr, nexc = p.nexc, np = p.np;
    const long long ndet = p.ndet;
    const int ka = (int)(K / nstr), kb = (int)(K % nstr);
    const double *__restrict__ c = p.cbase + (p.cslot ? (long long)*p.cslot : 0ll) * p.stride;
    const int32_t *__restrict__ ea = p.exc + (size_t)ka * nexc;
    const int32_t *__restrict__ eb = p.exc + (size_t)kb * nexc;
    int ia = 0, ib = 0;
    int32_t xa = ea[0], xb = eb[0];
    int pa = exc_pair(xa), pb = exc_pair(xb);
    TD *__restrict__ out = D + p.doff + K;
    const double *crow = c + (long long)ka * nstr;
    for (int A = 0; A < np; A++) {
        double v = 0.0;
        if (pa == A) {
            v += exc_sign(xa) * c[(long long)exc_J(xa) * nstr + kb];
            if (++ia < nexc) { xa = ea[ia]; pa = exc_pair(xa); } else pa = -1;
        }
        if (pb == A) {
            v += exc_sign(xb) * crow[exc_J(xb)];
            if (++ib < nexc) { xb = eb[ib]; pb = exc_pair(xb); } else pb = -1;
        }
        out[(long long)A * ndet] = (TD)v;
    }
}

// G = W D on CUDA cores (FP64 or FP32), 64x64 output tiles, K step 16.
template <typename T>
__global__ void __launch_bounds__(256)
contract_simt_kernel(const SigmaProb *__restrict__ probs, const WorkItem *__restrict__ tiles,
                     const T *__restrict__ D, T *__restrict__ G) {
    const WorkItem t = tiles[blockIdx.x];
    const SigmaProb &p = probs[t.prob];
    if (p.active && !*p.active) return;
    const T *__restrict__ W;
    if constexpr (sizeof(T) == 8) W = reinterpret_cast<const T *>(p.W); else W = reinterpret_cast<const T *>(p.Wf);
    const int np = p.np, ld = p.ld;
    const long long ndet = p.ndet;
    const int m0 = t.sub;
    const long long n0 = t.start;
    __shared__ T As[kGemmTK][kGemmTM];
    __shared__ T Bs[kGemmTK][kGemmTN];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = T(0);
    const T *Dp = D + p.doff;
    for (int k0 = 0; k0 < np; k0 += kGemmTK) {
#pragma unroll
        for (int r = 0; r < 4; r++) {
            int e = threadIdx.x + 256 * r;       // 0..1023
            int kk = e % kGemmTK, mm = e / kGemmTK;
            int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < np && k < np) ? W[(long long)m * ld + k] : T(0);
            int nn = e % kGemmTN, kb = e / kGemmTN;
            long long n = n0 + nn;
            int kr = k0 + kb;
            Bs[kb][nn] = (n < ndet && kr < np) ? Dp[(long long)kr * ndet + n] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGemmTK; kk++) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    T *Gp = G + p.doff;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int m = m0 + ty * 4 + i;
        if (m >= np) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            long long n = n0 + tx + 16 * j;
            if (n < ndet) Gp[(long long)m * ndet + n] = acc[i][j];
        }
    }
}

template <typename TG>
__global__ void __launch_bounds__(kGatherChunk)
scatter_kernel(const SigmaProb *__restrict__ probs, const WorkItem *__restrict__ items, const TG *__restrict__ G) {
    const WorkItem it = items[blockIdx.x];
    const SigmaProb &p = probs[it.prob];
    if (p.active && !*p.active) return;
    const long long I = it.start + threadIdx.x;
    if (I >= p.ndet) return;
    const int nstr = p.nstr, nexc = p.nexc;
    const long long ndet = p.ndet;
    const int ia = (int)(I / nstr), ib = (int)(I % nstr);
    const int32_t *__restrict__ ea = p.exc + (size_t)ia * nexc;
    const int32_t *__restrict__ eb = p.exc + (size_t)ib * nexc;
    const TG *__restrict__ Gp = G + p.doff;
    double v = 0.0;
    for (int e = 0; e < nexc; e++) {
        int32_t x = ea[e];
        v += exc_sign(x) * (double)Gp[(long long)exc_pair(x) * ndet + (long long)exc_J(x) * nstr + ib];
    }
    const long long rowb = (long long)ia * nstr;
    for (int e = 0; e < nexc; e++) {
        int32_t x = eb[e];
        v += exc_sign(x) * (double)Gp[(long long)exc_pair(x) * ndet + rowb + exc_J(x)];
    }
    double *s = p.sbase + (p.sslot ? (long long)*p.sslot : 0ll) * p.stride;
    s[I] = v;
}

// Quantised copy of c for the tensor-core gathers, written into the D buffer
// (which those paths do not need): FP32 for BF16, and for FP64E the fixed
// point integer X = round(c * 2^38 / dscale), so that their gathers run in FP32
// or integer arithmetic (GB300 issues FP64 at a small fraction of FP32).
template <int KIND>
__global__ void __launch_bounds__(kGatherChunk)
quantise_kernel(const SigmaProb *__restrict__ probs, const WorkItem *__restrict__ items, char *__restrict__ qbuf) {
    const WorkItem it = items[blockIdx.x];
    const SigmaProb &p = probs[it.prob];
    if (p.active && !*p.active) return;
    const long long I = it.start + threadIdx.x;
    if (I >= p.ndet) return;
    const double *c = p.cbase + (p.cslot ? (long long)*p.cslot : 0ll) * p.stride;
    const long long off = p.qoff;
    // symmetric gathers read the negated copy at off + ndet (sign by address)
    if (KIND == 0) {
        const float v = (float)c[I];
        reinterpret_cast<float *>(qbuf)[off + I] = v;
        if (p.sym) reinterpret_cast<float *>(qbuf)[off + p.ndet + I] = -v;
    } else {
        const double sc = 274877906944.0 / p.dscale;   // 2^38 / dscale
        const long long v = __double2ll_rn(c[I] * sc);
        reinterpret_cast<long long *>(qbuf)[off + I] = v;
        if (p.sym) reinterpret_cast<long long *>(qbuf)[off + p.ndet + I] = -v;
    }
}

// sigma = S + S^T in place for the spin-flip-symmetric problems (each
// unordered pair of determinants (ka, kb), (kb, ka) is owned by one thread).
__global__ void __launch_bounds__(kGatherChunk)
sym_sum_kernel(const SigmaProb *__restrict__ probs, const WorkItem *__restrict__ items) {
    const WorkItem it = items[blockIdx.x];
    const SigmaProb &p = probs[it.prob];
    if (!p.sym || (p.active && !*p.active)) return;
    const long long K = it.start + threadIdx.x;
    if (K >= p.ndet) return;
    const int nstr = p.nstr;
    const int ka = (int)(K / nstr), kb = (int)(K % nstr);
    if (ka > kb) return;
    double *s = p.sbase + (p.sslot ? (long long)*p.sslot : 0ll) * p.stride;
    const long long T = (long long)kb * nstr + ka;
    const double v = s[K] + s[T];
    s[K] = v;
    s[T] = v;
}

// Scatter of the FP64-emulating path: G is int64 fixed point with one scale
// per problem (2^-45 Wscale dscale), so sigma_I sums integers exactly and
// converts once.
__global__ void __launch_bounds__(kGatherChunk)
scatter_fixed_kernel(const SigmaProb *__restrict__ probs, const WorkItem *__restrict__ items,
                     const long long *__restrict__ G) {
    const WorkItem it = items[blockIdx.x];
    const SigmaProb &p = probs[it.prob];
    if (p.active && !*p.active) return;
    const long long I = it.start + threadIdx.x;
    if (I >= p.ndet) return;
    const int nstr = p.nstr, nexc = p.nexc;
    const long long ndet = p.ndet;
    const int ia = (int)(I / nstr), ib = (int)(I % nstr);
    const int32_t *__restrict__ ea = p.exc + (size_t)ia * nexc;
    const int32_t *__restrict__ eb = p.exc + (size_t)ib * nexc;
    const long long *__restrict__ Gp = G + p.doff;
    const uint8_t *__restrict__ pact = p.pact;   // G rows of other pairs are not written (their W is zero)
    long long acc = 0;
    for (int e = 0; e < nexc; e++) {
        const int32_t x = ea[e];
        if (pact && !pact[exc_pair(x)]) continue;
        const long long gv = Gp[(long long)exc_pair(x) * ndet + (long long)exc_J(x) * nstr + ib];
        acc += (x & 1) ? -gv : gv;
    }
    const long long rowb = (long long)ia * nstr;
    for (int e = 0; e < nexc; e++) {
        const int32_t x = eb[e];
        if (pact && !pact[exc_pair(x)]) continue;
        const long long gv = Gp[(long long)exc_pair(x) * ndet + rowb + exc_J(x)];
        acc += (x & 1) ? -gv : gv;
    }
    double *s = p.sbase + (p.sslot ? (long long)*p.sslot : 0ll) * p.stride;
    s[I] = (double)acc * (p.Wexp[0] * p.dscale * 0x1p-45);
}

int plan_sigma(ifci_handle_t h, SigmaPlan &plan, long long budget, int precision) {
    plan.waves.clear();
    plan.items.clear();
    plan.tiles.clear();
    plan.tctiles.clear();
    plan.max_delems = 0;
    plan.max_qelems = 0;
    const bool tc = precision == IFCI_BF16 || precision == IFCI_TF32;
    SigmaWave w{};
    auto close_wave = [&](int next_prob) {
        if (w.nprob) {
            plan.max_delems = std::max(plan.max_delems, w.delems);
            plan.max_qelems = std::max(plan.max_qelems, w.qelems);
            plan.waves.push_back(w);
        }
        w = SigmaWave{};
        w.prob0 = next_prob;
        w.item0 = (int)plan.items.size();
        w.tile0 = (int)plan.tiles.size();
        w.tc0 = (int)plan.tctiles.size();
    };
    for (size_t i = 0; i < plan.probs.size(); i++) {
        SigmaProb &p = plan.probs[i];
        // the alpha-only form is a tensor-core gather; the CUDA-core paths build the full D
        p.sym = (p.sym && (tc || precision == IFCI_FP64E) && 2 * p.ndet < (1ll << 31)) ? 1 : 0;
        long long need = sigma_elems(p.np, p.ndet);
        if (need > budget && precision == IFCI_FP64E && p.sym) {
            // row slabs of G: each its own wave, the scatter accumulating into S
            if (p.npc <= 0 || !p.act) p.npc = p.np;
            const int rpt = tcg::rows_per_tile(p.nstr);
            const long long row_elems = (long long)p.np * p.nstr;
            int rows = (int)std::min<long long>(p.nstr, budget / row_elems);
            rows = rows / rpt * rpt;
            if (rows < 1)
                return set_error(h, IFCI_ERR_OOM, "sigma: one alpha row block needs %lld intermediate elements, "
                                 "budget %lld", row_elems * rpt, budget);
            close_wave((int)i);
            const int nchunk = (((p.npc + 63) / 64) + 2) / 3;
            for (int r0 = 0; r0 < p.nstr; r0 += rows) {
                const int r1 = std::min(p.nstr, r0 + rows);
                w.nprob = 1;
                p.doff = 0;
                p.qoff = 0;
                w.delems = (long long)p.np * (r1 - r0) * p.nstr;
                w.qelems = 3 * p.ndet;   // +-Q and the int64 accumulator S
                w.k0 = (long long)r0 * p.nstr;
                w.kn = (long long)(r1 - r0) * p.nstr;
                w.slab_first = r0 == 0;
                w.slab_last = r1 == p.nstr;
                for (long long s0 = 0; s0 < p.ndet; s0 += kGatherChunk) {
                    plan.items.push_back(WorkItem{(int)i, 0, s0});
                    w.nitem++;
                }
                for (int n0 = 0; n0 < p.npc; n0 += oz_tile_n())
                    for (int kc = 0; kc < nchunk; kc++) {
                        size_t before = plan.tctiles.size();
                        tcg::append_row_tiles(plan.tctiles, (int)i, n0 | (kc << 16), p.nstr, r0, r1);
                        w.ntc += (int)(plan.tctiles.size() - before);
                    }
                close_wave((int)i);
            }
            w.prob0 = (int)i + 1;
            continue;
        }
        if (need > budget)
            return set_error(h, IFCI_ERR_OOM, "sigma: one problem needs %lld intermediate elements, budget %lld",
                             need, budget);
        if (w.delems + need > budget) close_wave((int)i);
        w.nprob++;
        p.doff = w.delems;
        w.delems += need;
        p.qoff = w.qelems;
        w.qelems += p.sym ? 2 * p.ndet : p.ndet;
        for (long long s0 = 0; s0 < p.ndet; s0 += kGatherChunk) {
            plan.items.push_back(WorkItem{(int)i, 0, s0});
            w.nitem++;
        }
        if (tc) {
            // one tile = up to 128 determinants of whole alpha rows x all pairs (sigma_tc.cu)
            size_t before = plan.tctiles.size();
            tcg::append_row_tiles(plan.tctiles, (int)i, 0, p.nstr);
            w.ntc += (int)(plan.tctiles.size() - before);
        } else if (precision == IFCI_FP64E) {
            // one tile = up to 128 determinants x oz_tile_n() output pairs (sigma_oz.cu);
            // the output-pair tiles of a problem run back to back so W stays resident longer
            if (p.npc <= 0 || !p.act) p.npc = p.np;
            // K chunks of 192 pairs keep every level sum exact (sigma_oz.cu)
            const int nchunk = (((p.npc + 63) / 64) + 2) / 3;
            for (int n0 = 0; n0 < p.npc; n0 += oz_tile_n())
                for (int kc = 0; kc < nchunk; kc++) {
                    size_t before = plan.tctiles.size();
                    tcg::append_row_tiles(plan.tctiles, (int)i, n0 | (kc << 16), p.nstr);
                    w.ntc += (int)(plan.tctiles.size() - before);
                }
        } else {
            for (int m0 = 0; m0 < p.np; m0 += kGemmTM)
                for (long long s0 = 0; s0 < p.ndet; s0 += kGemmTN) {
                    plan.tiles.push_back(WorkItem{(int)i, m0, s0});
                    w.ntile++;
                }
        }
    }
    close_wave((int)plan.probs.size());
    plan.any_sym = false;
    for (const SigmaProb &p : plan.probs) plan.any_sym = plan.any_sym || p.sym;
    // dynamically scheduled tensor-core tiles: largest problems first (longest
    // tiles start early), stable within a problem
    for (const SigmaWave &wv : plan.waves)
        std::stable_sort(plan.tctiles.begin() + wv.tc0, plan.tctiles.begin() + wv.tc0 + wv.ntc,
                         [&](const WorkItem &x, const WorkItem &y) {
                             return plan.probs[x.prob].np > plan.probs[y.prob].np;
                         });
    return IFCI_OK;
}

size_t plan_device_bytes(const SigmaPlan &plan) {
    return ws_round(plan.probs.size() * sizeof(SigmaProb)) + ws_round(plan.items.size() * sizeof(WorkItem)) +
           ws_round(plan.tiles.size() * sizeof(WorkItem)) + ws_round(plan.tctiles.size() * sizeof(WorkItem));
}

int upload_plan(ifci_handle_t h, SigmaPlan &plan, cudaStream_t s) {
    for (const SigmaProb &p : plan.probs)
        if (p.sym && !p.pmap) return set_error(h, IFCI_ERR_INVALID_ARG, "sigma plan: symmetric problem without pair map");
    plan.d_probs = ws_take<SigmaProb>(h, std::max<size_t>(1, plan.probs.size()));
    plan.d_items = ws_take<WorkItem>(h, std::max<size_t>(1, plan.items.size()));
    plan.d_tiles = ws_take<WorkItem>(h, std::max<size_t>(1, plan.tiles.size()));
    plan.d_tctiles = ws_take<WorkItem>(h, std::max<size_t>(1, plan.tctiles.size()));
    if (!plan.d_probs || !plan.d_items || !plan.d_tiles || !plan.d_tctiles)
        return set_error(h, IFCI_ERR_OOM, "sigma plan: workspace too small");
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(plan.d_probs, plan.probs.data(), plan.probs.size() * sizeof(SigmaProb),
                                     cudaMemcpyHostToDevice, s));
    if (!plan.items.empty())
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(plan.d_items, plan.items.data(), plan.items.size() * sizeof(WorkItem),
                                         cudaMemcpyHostToDevice, s));
    if (!plan.tiles.empty())
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(plan.d_tiles, plan.tiles.data(), plan.tiles.size() * sizeof(WorkItem),
                                         cudaMemcpyHostToDevice, s));
    if (!plan.tctiles.empty())
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(plan.d_tctiles, plan.tctiles.data(),
                                         plan.tctiles.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
    return IFCI_OK;
}

// Copies the plan's descriptor arrays to the device arrays the caller set in
// plan.d_probs, d_items, d_tiles, d_tctiles (each holding at least one entry).
int upload_plan_to(ifci_handle_t h, SigmaPlan &plan, cudaStream_t s) {
    for (const SigmaProb &p : plan.probs)
        if (p.sym && !p.pmap) return set_error(h, IFCI_ERR_INVALID_ARG, "sigma plan: symmetric problem without pair map");
    if (!plan.d_probs || !plan.d_items || !plan.d_tiles || !plan.d_tctiles)
        return set_error(h, IFCI_ERR_INVALID_ARG, "sigma plan: device arrays not set");
    if (!plan.probs.empty())
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(plan.d_probs, plan.probs.data(), plan.probs.size() * sizeof(SigmaProb),
                                         cudaMemcpyHostToDevice, s));
    if (!plan.items.empty())
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(plan.d_items, plan.items.data(), plan.items.size() * sizeof(WorkItem),
                                         cudaMemcpyHostToDevice, s));
    if (!plan.tiles.empty())
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(plan.d_tiles, plan.tiles.data(), plan.tiles.size() * sizeof(WorkItem),
                                         cudaMemcpyHostToDevice, s));
    if (!plan.tctiles.empty())
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(plan.d_tctiles, plan.tctiles.data(),
                                         plan.tctiles.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
    return IFCI_OK;
}

// The same for one row slab of a spin-flip-symmetric problem (SigmaWave::kn):
// G holds alpha rows [r0, r1) only; the alpha loop takes the excitations whose
// J row lies in the slab, the beta loop runs when I's own row does.  The sum
// is carried in the int64 accumulator S across the slabs (exact, so the
// result equals the unsplit scatter bit for bit) and converted on the last.
__global__ void __launch_bounds__(kGatherChunk)
scatter_fixed_slab_kernel(const SigmaProb *__restrict__ probs, const WorkItem *__restrict__ items,
                          const long long *__restrict__ G, long long *__restrict__ Qbuf, int r0, int r1, int first,
                          int last) {
    const WorkItem it = items[blockIdx.x];
    const SigmaProb &p = probs[it.prob];
    if (p.active && !*p.active) return;
    const long long I = it.start + threadIdx.x;
    if (I >= p.ndet) return;
    const int nstr = p.nstr, nexc = p.nexc;
    const long long kn = (long long)(r1 - r0) * nstr, k0 = (long long)r0 * nstr;
    const int ia = (int)(I / nstr), ib = (int)(I % nstr);
    const int32_t *__restrict__ ea = p.exc + (size_t)ia * nexc;
    const uint8_t *__restrict__ pact = p.pact;
    long long *S = Qbuf + p.qoff + 2 * p.ndet;
    long long acc = first ? 0 : S[I];
    for (int e = 0; e < nexc; e++) {
        const int32_t x = ea[e];
        const int J = exc_J(x);
        if (J < r0 || J >= r1 || (pact && !pact[exc_pair(x)])) continue;
        const long long gv = G[(long long)exc_pair(x) * kn + (long long)J * nstr + ib - k0];
        acc += (x & 1) ? -gv : gv;
    }
    if (ia >= r0 && ia < r1) {
        const int32_t *__restrict__ eb = p.exc + (size_t)ib * nexc;
        const long long rowb = (long long)ia * nstr - k0;
        for (int e = 0; e < nexc; e++) {
            const int32_t x = eb[e];
            if (pact && !pact[exc_pair(x)]) continue;
            const long long gv = G[(long long)exc_pair(x) * kn + rowb + exc_J(x)];
            acc += (x & 1) ? -gv : gv;
        }
    }
    if (last) {
        double *s = p.sbase + (p.sslot ? (long long)*p.sslot : 0ll) * p.stride;
        s[I] = (double)acc * (p.Wexp[0] * p.dscale * 0x1p-45);
    } else {
        S[I] = acc;
    }
}

int run_sigma(ifci_handle_t h, const SigmaPlan &plan, int precision, void *D, void *G, cudaStream_t s) {
    for (const SigmaWave &w : plan.waves) {
        if (w.nitem == 0) continue;
        if (precision == IFCI_FP64) {
            {
                ProfScope ps(h, s, PK_GATHER);
                gather_kernel<double><<<w.nitem, kGatherChunk, 0, s>>>(plan.d_probs, plan.d_items + w.item0,
                                                                       (double *)D);
                IFCI_LAUNCH_CHECK(h);
            }
            {
                ProfScope ps(h, s, PK_CONTRACT);
                contract_simt_kernel<double><<<w.ntile, 256, 0, s>>>(plan.d_probs, plan.d_tiles + w.tile0,
                                                                     (const double *)D, (double *)G);
                IFCI_LAUNCH_CHECK(h);
            }
            ProfScope ps(h, s, PK_SCATTER);
            scatter_kernel<double><<<w.nitem, kGatherChunk, 0, s>>>(plan.d_probs, plan.d_items + w.item0,
                                                                    (const double *)G);
            IFCI_LAUNCH_CHECK(h);
        } else if (precision == IFCI_FP32) {
            {
                ProfScope ps(h, s, PK_GATHER);
                gather_kernel<float><<<w.nitem, kGatherChunk, 0, s>>>(plan.d_probs, plan.d_items + w.item0,
                                                                      (float *)D);
                IFCI_LAUNCH_CHECK(h);
            }
            {
                ProfScope ps(h, s, PK_CONTRACT);
                contract_simt_kernel<float><<<w.ntile, 256, 0, s>>>(plan.d_probs, plan.d_tiles + w.tile0,
                                                                   (const float *)D, (float *)G);
                IFCI_LAUNCH_CHECK(h);
            }
            ProfScope ps(h, s, PK_SCATTER);
            scatter_kernel<float><<<w.nitem, kGatherChunk, 0, s>>>(plan.d_probs, plan.d_items + w.item0,
                                                                   (const float *)G);
            IFCI_LAUNCH_CHECK(h);
        } else if (precision == IFCI_FP64E) {
            {
                ProfScope ps(h, s, PK_GATHER);
                quantise_kernel<1><<<w.nitem, kGatherChunk, 0, s>>>(plan.d_probs, plan.d_items + w.item0, (char *)D);
                IFCI_LAUNCH_CHECK(h);
            }
            IFCI_TRY(launch_oz_contract(h, plan, w, D, G, s));
            ProfScope ps(h, s, PK_SCATTER);
            if (w.kn) {
                const int nstr = plan.probs[w.prob0].nstr;
                scatter_fixed_slab_kernel<<<w.nitem, kGatherChunk, 0, s>>>(
                    plan.d_probs, plan.d_items + w.item0, (const long long *)G, (long long *)D,
                    (int)(w.k0 / nstr), (int)((w.k0 + w.kn) / nstr), w.slab_first, w.slab_last);
            } else {
                scatter_fixed_kernel<<<w.nitem, kGatherChunk, 0, s>>>(plan.d_probs, plan.d_items + w.item0,
                                                                      (const long long *)G);
            }
            IFCI_LAUNCH_CHECK(h);
            if (plan.any_sym && (!w.kn || w.slab_last)) {
                sym_sum_kernel<<<w.nitem, kGatherChunk, 0, s>>>(plan.d_probs, plan.d_items + w.item0);
                IFCI_LAUNCH_CHECK(h);
            }
        } else {
            {
                ProfScope ps(h, s, PK_GATHER);
                quantise_kernel<0><<<w.nitem, kGatherChunk, 0, s>>>(plan.d_probs, plan.d_items + w.item0, (char *)D);
                IFCI_LAUNCH_CHECK(h);
            }
            IFCI_TRY(launch_tc_contract(h, plan, w, precision, D, G, s));
            ProfScope ps(h, s, PK_SCATTER);
            scatter_kernel<float><<<w.nitem, kGatherChunk, 0, s>>>(plan.d_probs, plan.d_items + w.item0,
                                                                   (const float *)G);
            IFCI_LAUNCH_CHECK(h);
            if (plan.any_sym) {
                sym_sum_kernel<<<w.nitem, kGatherChunk, 0, s>>>(plan.d_probs, plan.d_items + w.item0);
                IFCI_LAUNCH_CHECK(h);
            }
        }
    }
    return IFCI_OK;
}

// FP32 copy of the folded matrix for the FP32 path.
__global__ void convert_w_kernel(const SigmaProb *__restrict__ probs) {
    const SigmaProb &p = probs[blockIdx.x];
    float *Wf = const_cast<float *>(p.Wf);
    for (long long t = threadIdx.x; t < (long long)p.ld * p.ld; t += blockDim.x) Wf[t] = (float)p.W[t];
}

int launch_convert_w(ifci_handle_t h, int nprob, const SigmaProb *d_probs, cudaStream_t s) {
    convert_w_kernel<<<nprob, 256, 0, s>>>(d_probs);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

}  // namespace ifci

namespace ifci {

// Launches the FP64 gather, contraction and scatter of one prepared wave
// without a handle (used by the allocation-free sigma entry point).
cudaError_t launch_sigma_fp64_raw(const SigmaProb *d_probs, const WorkItem *d_items, int nitem,
                                  const WorkItem *d_tiles, int ntile, double *D, double *G, cudaStream_t s) {
    gather_kernel<double><<<nitem, kGatherChunk, 0, s>>>(d_probs, d_items, D);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    contract_simt_kernel<double><<<ntile, 256, 0, s>>>(d_probs, d_tiles, D, G);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scatter_kernel<double><<<nitem, kGatherChunk, 0, s>>>(d_probs, d_items, G);
    return cudaGetLastError();
}

}  // namespace ifci
