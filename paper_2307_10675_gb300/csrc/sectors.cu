// Exact blocks of a CI space over decoupled orbital groups.
//
// E_X is the lowest eigenvalue of H in the space of body set X (Methods,
// definition of E_c(X)).  When the orbitals of X fall into groups that no
// integral couples — h_pq and every (pq|rs) with p, q in different groups
// below a tolerance tau, as for bodies far apart on the synthetic chains —
// the number of alpha and the number of beta electrons in each group are
// conserved by H' (H with those integrals set to zero), which is then block
// diagonal over the distributions (a, b) of the alpha and beta electrons
// among the groups.  The lowest eigenvalue of H' is the minimum over the
// blocks, and a Davidson iteration started inside one block never leaves it,
// so the lowest eigenvalue is found block by block instead of by a search
// over sectors.  Each block, with its spin-flip image, is its own Davidson
// problem; all blocks of one space share one sigma build per iteration:
// their newest vectors are placed into one whole-space vector (they occupy
// disjoint determinants), sigma = H' c is built once with the integrals of
// H', and each block takes its own part back.  The lowest block's vector is
// then the start of a Davidson iteration with the full H (a polish step),
// which turns it into the eigenvector of H: its Rayleigh quotient can only
// fall, and H - H' is of order tau.
#include <algorithm>
#include <cmath>

#include "dav_driver.cuh"
#include "hamiltonian.cuh"

namespace ifci {

namespace {

// orbital pairs (p, q), p > q, coupled above tau: by h_pq or by any (pq|rs)
__global__ void __launch_bounds__(256) coupling_kernel(const CoupDesc *__restrict__ desc, double tau,
                                                       uint32_t *__restrict__ adj) {
    const CoupDesc d = desc[blockIdx.x];
    const int n = d.n, np = n * (n + 1) / 2;
    __shared__ uint32_t a[32];
    if (threadIdx.x < 32) a[threadIdx.x] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int A = warp; A < np; A += nwarp) {
        int P = 0;
        while ((P + 1) * (P + 2) / 2 <= A) P++;
        const int Q = A - P * (P + 1) / 2;
        if (P == Q) continue;
        double m = 0.0;
        for (int B = lane; B < np; B += 32) m = fmax(m, fabs(d.eri[(long long)A * np + B]));
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        m = fmax(m, fabs(d.h1[P * n + Q]));
        if (lane == 0 && m > tau) {
            atomicOr(&a[P], 1u << Q);
            atomicOr(&a[Q], 1u << P);
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) adj[blockIdx.x * 32 + threadIdx.x] = a[threadIdx.x];
}

// H' of a sectored space: integrals with a pair of orbitals from different
// groups set to zero
__global__ void __launch_bounds__(256) mask_kernel(const MaskDesc *__restrict__ desc) {
    const MaskDesc d = desc[blockIdx.x];
    const int n = d.n, np = n * (n + 1) / 2;
    __shared__ unsigned char cross[32 * 33 / 2 + 16];
    for (int A = threadIdx.x; A < np; A += blockDim.x) {
        int P = 0;
        while ((P + 1) * (P + 2) / 2 <= A) P++;
        const int Q = A - P * (P + 1) / 2;
        cross[A] = d.label[P] != d.label[Q];
    }
    __syncthreads();
    double mx = 0.0;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int p = t / n, q = t % n;
        const bool keep = d.label[p] == d.label[q];
        d.h1m[t] = keep ? d.h1[t] : 0.0;
        if (!keep) mx = fmax(mx, fabs(d.h1[t]));
    }
    for (long long t = threadIdx.x; t < (long long)np * np; t += blockDim.x) {
        const int A = (int)(t / np), B = (int)(t % np);
        const bool drop = cross[A] | cross[B];
        d.erim[t] = drop ? 0.0 : d.eri[t];
        if (drop) mx = fmax(mx, fabs(d.eri[t]));
    }
    __shared__ double red[256];
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *d.dropped = red[0];
}

// whole-space input of a sector unit's sigma: every block problem writes its
// newest vector (zero if the flag says it takes no sigma this time) at its
// determinants and, for an off-diagonal block, at their spin-flip images
__device__ __forceinline__ void sector_gather_kernel_body(const DavProb *__restrict__ probs,
                                                            const DavState *__restrict__ st,
                                                            const WorkItem *__restrict__ items,
                                                            const int *__restrict__ flag, int w_) {
    const WorkItem it = items[w_];
    const DavProb &p = probs[it.prob];
    if (!p.gc) return;
    const bool on = flag[it.prob] != 0;
    const double *x = p.B + (long long)st[it.prob].newest * p.ndet;
    const long long end = min(it.start + (long long)kVecChunk, p.ndet);
    const long long n = p.nstr;
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
        const int ia = (int)(I / p.nb), ib = (int)(I % p.nb);
        const long long ga = blk_row(p, ia), gb = blk_col(p, ib);
        const double v = on ? x[I] : 0.0;
        p.gc[ga * n + gb] = v;
        if (!p.sym) p.gc[gb * n + ga] = v;
    }
}

__global__ void __launch_bounds__(256) sector_gather_kernel(const DavProb *__restrict__ probs,
                                                            const DavState *__restrict__ st,
                                                            const WorkItem *__restrict__ items,
                                                            const int *__restrict__ flag, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) sector_gather_kernel_body(probs, st, items, flag, w);
}

// each block problem takes its part of the whole-space sigma
__device__ __forceinline__ void sector_scatter_kernel_body(const DavProb *__restrict__ probs,
                                                             const DavState *__restrict__ st,
                                                             const WorkItem *__restrict__ items,
                                                             const int *__restrict__ flag, int w_) {
    const WorkItem it = items[w_];
    const DavProb &p = probs[it.prob];
    if (!p.gc || !flag[it.prob]) return;
    double *y = p.S + (long long)st[it.prob].newest * p.ndet;
    const long long end = min(it.start + (long long)kVecChunk, p.ndet);
    const long long n = p.nstr;
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
        const int ia = (int)(I / p.nb), ib = (int)(I % p.nb);
        y[I] = p.gs[(long long)blk_row(p, ia) * n + blk_col(p, ib)];
    }
}

__global__ void __launch_bounds__(256) sector_scatter_kernel(const DavProb *__restrict__ probs,
                                                             const DavState *__restrict__ st,
                                                             const WorkItem *__restrict__ items,
                                                             const int *__restrict__ flag, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) sector_scatter_kernel_body(probs, st, items, flag, w);
}

// diagonal of a block problem from its unit's whole-space diagonal (in gs)
__device__ __forceinline__ void sector_hd_kernel_body(const DavProb *__restrict__ probs,
                                                        const WorkItem *__restrict__ items, int w_) {
    const WorkItem it = items[w_];
    const DavProb &p = probs[it.prob];
    if (!p.gc) return;
    double *hd = const_cast<double *>(p.hd);
    const long long end = min(it.start + (long long)kVecChunk, p.ndet);
    const long long n = p.nstr;
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
        const int ia = (int)(I / p.nb), ib = (int)(I % p.nb);
        hd[I] = p.gs[(long long)blk_row(p, ia) * n + blk_col(p, ib)];
    }
}

__global__ void __launch_bounds__(256) sector_hd_kernel(const DavProb *__restrict__ probs,
                                                        const WorkItem *__restrict__ items, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) sector_hd_kernel_body(probs, items, w);
}

// a unit's sigma runs (per precision) when any of its problems asks for it
__global__ void unit_flags_kernel(const int2 *__restrict__ range, int nunit, const int *__restrict__ hi,
                                  const int *__restrict__ lo, int *__restrict__ uhi, int *__restrict__ ulo) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nunit) return;
    const int2 r = range[u];
    int a = 0, b = 0;
    for (int i = r.x; i < r.x + r.y; i++) {
        a |= hi[i];
        b |= lo[i];
    }
    uhi[u] = a;
    ulo[u] = b;
}

// the whole-space vector of a block's converged vector (c_out of the block
// problem): x at the block's determinants, and at their spin-flip images for
// an off-diagonal block (both scaled by 1/sqrt 2, so the result has unit norm)
__device__ __forceinline__ void sector_expand_kernel_body(const DavProb *__restrict__ probs,
                                                            const WorkItem *__restrict__ items,
                                                            double *const *__restrict__ dst, int w_) {
    const WorkItem it = items[w_];
    const DavProb &p = probs[it.prob];
    double *out = dst[it.prob];
    if (!out || !p.c_out) return;
    const double f = p.sym ? 1.0 : 0.7071067811865476;
    const long long end = min(it.start + (long long)kVecChunk, p.ndet);
    const long long n = p.nstr;
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
        const int ia = (int)(I / p.nb), ib = (int)(I % p.nb);
        const long long ga = blk_row(p, ia), gb = blk_col(p, ib);
        const double v = f * p.c_out[I];
        out[ga * n + gb] = v;
        if (!p.sym) out[gb * n + ga] = v;
    }
}

__global__ void __launch_bounds__(256) sector_expand_kernel(const DavProb *__restrict__ probs,
                                                            const WorkItem *__restrict__ items,
                                                            double *const *__restrict__ dst, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) sector_expand_kernel_body(probs, items, dst, w);
}

// pair map of a sectored unit restricted to its active pairs
__global__ void __launch_bounds__(256) compact_pmaps_kernel(const CompactDesc *__restrict__ desc, int n) {
    for (int u = blockIdx.x; u < n; u += gridDim.x) {
        const CompactDesc d = desc[u];
        const long long tot = (long long)d.nstr * d.ldc;
        for (long long t = threadIdx.x; t < tot; t += blockDim.x) {
            const long long r = t / d.ldc;
            const int k = (int)(t % d.ldc);
            d.pmapc[t] = k < d.npc ? d.pmap[r * d.ld + d.act[k]] : -1;
        }
    }
}

}  // namespace

int launch_compact_pair_maps(ifci_handle_t h, int n, const CompactDesc *d_desc, cudaStream_t s) {
    if (n <= 0) return IFCI_OK;
    compact_pmaps_kernel<<<stride_grid(h->device, n, 8), 256, 0, s>>>(d_desc, n);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_coupling(ifci_handle_t h, int nprob, const CoupDesc *d_desc, double tau, uint32_t *d_adj, cudaStream_t s) {
    coupling_kernel<<<nprob, 256, 0, s>>>(d_desc, tau, d_adj);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_mask(ifci_handle_t h, int nprob, const MaskDesc *d_desc, cudaStream_t s) {
    mask_kernel<<<nprob, 256, 0, s>>>(d_desc);   // 256 threads: the reduction above assumes it
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_sector_gather(ifci_handle_t h, const DavBatch &b, const int *flag, cudaStream_t s) {
    sector_gather_kernel<<<stride_grid(h->device, (long long)b.vitems.size(), 8), 256, 0, s>>>(b.d_probs, b.d_state, b.d_vitems, flag, (int)b.vitems.size());
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_sector_scatter(ifci_handle_t h, const DavBatch &b, const int *flag, cudaStream_t s) {
    sector_scatter_kernel<<<stride_grid(h->device, (long long)b.vitems.size(), 8), 256, 0, s>>>(b.d_probs, b.d_state, b.d_vitems, flag, (int)b.vitems.size());
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_sector_hd(ifci_handle_t h, const DavBatch &b, cudaStream_t s) {
    sector_hd_kernel<<<stride_grid(h->device, (long long)b.vitems.size(), 8), 256, 0, s>>>(b.d_probs, b.d_vitems, (int)b.vitems.size());
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_unit_flags(ifci_handle_t h, const DavBatch &b, const int *hi, const int *lo, cudaStream_t s) {
    unit_flags_kernel<<<(b.nunit + 127) / 128, 128, 0, s>>>(b.d_urange, b.nunit, hi, lo, b.d_uhi, b.d_ulo);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_sector_expand(ifci_handle_t h, const DavBatch &b, double *const *d_dst, cudaStream_t s) {
    sector_expand_kernel<<<stride_grid(h->device, (long long)b.vitems.size(), 8), 256, 0, s>>>(b.d_probs, b.d_vitems, d_dst, (int)b.vitems.size());
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

// Connected components of the coupling graph of each problem's orbitals.
void orbital_groups(const uint32_t *adj, int n, std::vector<int> &label, int &ngroup) {
    label.assign(n, -1);
    ngroup = 0;
    for (int p = 0; p < n; p++) {
        if (label[p] >= 0) continue;
        std::vector<int> stack{p};
        label[p] = ngroup;
        while (!stack.empty()) {
            const int u = stack.back();
            stack.pop_back();
            for (uint32_t x = adj[u]; x; x &= x - 1) {
                const int v = __builtin_ctz(x);
                if (v < n && label[v] < 0) {
                    label[v] = ngroup;
                    stack.push_back(v);
                }
            }
        }
        ngroup++;
    }
}

}  // namespace ifci
