// Start vectors of the batched Davidson from a small exact eigenproblem (a
// "P-space" guess), and single Hamiltonian matrix elements.
//
// The lowest singlet of a body set can be a charge-transfer state whose
// leading determinant is not the one of lowest diagonal energy; started from
// that determinant plus a small random part, the Davidson iteration can meet
// its residual tolerance on an excited state before the ground-state component
// has grown.  The guess here diagonalises H exactly in the span of the
// spin-flip-symmetric pair functions u_K of the kPsp lowest-diagonal
// determinants K = (I_a, I_b), I_a <= I_b,
//   u_K = (|I_a I_b> + |I_b I_a>) / sqrt 2   (I_a != I_b),   u_K = |I_a I_a>,
// and starts from its lowest eigenvector.
//
// Matrix elements <I|H|J> of H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs)
// (E_pq E_rs - delta_qr E_ps) between determinants (alpha string, beta string)
// follow the Slater–Condon rules on the bit masks: zero beyond double
// excitations; for a single excitation j -> a (spin s) the sign is the parity
// of the orbitals occupied strictly between a and j; a same-spin double is two
// such excitations applied in turn; an opposite-spin double is the product of
// the two single signs.
#include "dav_driver.cuh"
#include "hamiltonian.cuh"
#include "slater.cuh"

namespace ifci {

namespace {

constexpr int kPsp = kPspMax;   // pair functions in the guess space
constexpr int kSelThreads = 256;
constexpr int kSelPer = 4;      // candidates kept per thread during selection
constexpr int kSelCand = kSelThreads * kSelPer;

// Per problem: the kPsp lowest-diagonal canonical determinants (I_a <= I_b).
// Each thread keeps its kSelPer lowest over a strided scan, then the block
// sorts the candidates (bitonic, by value then index).
__device__ __forceinline__ void psp_select_kernel_body(const DavProb *__restrict__ probs, long long *__restrict__ pidx, int *__restrict__ pcount, int w_) {
    const DavProb p = probs[w_];
    __shared__ double sv[kSelCand];
    __shared__ long long si[kSelCand];
    double bv[kSelPer];
    long long bi[kSelPer];
#pragma unroll
    for (int u = 0; u < kSelPer; u++) {
        bv[u] = 1e300;
        bi[u] = 0x7fffffffffffffffll;
    }
    const int n = p.nb;
    for (long long I = threadIdx.x; I < p.ndet; I += kSelThreads) {
        const int a = (int)(I / n), b = (int)(I % n);
        if (p.sym && a > b) continue;
        double v = p.hd[I];
        long long i = I;
        if (v < bv[kSelPer - 1] || (v == bv[kSelPer - 1] && i < bi[kSelPer - 1])) {
#pragma unroll
            for (int u = 0; u < kSelPer; u++) {   // insertion into the sorted list
                if (v < bv[u] || (v == bv[u] && i < bi[u])) {
                    const double tv = bv[u];
                    const long long ti = bi[u];
                    bv[u] = v;
                    bi[u] = i;
                    v = tv;
                    i = ti;
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < kSelPer; u++) {
        sv[threadIdx.x * kSelPer + u] = bv[u];
        si[threadIdx.x * kSelPer + u] = bi[u];
    }
    __syncthreads();
    for (int size = 2; size <= kSelCand; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < kSelCand; t += kSelThreads) {
                const int partner = t ^ stride;
                if (partner > t) {
                    const bool up = (t & size) == 0;
                    const bool gt = sv[t] > sv[partner] || (sv[t] == sv[partner] && si[t] > si[partner]);
                    if (gt == up) {
                        const double tv = sv[t];
                        const long long ti = si[t];
                        sv[t] = sv[partner];
                        si[t] = si[partner];
                        sv[partner] = tv;
                        si[partner] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    const long long nsym = p.ndim;
    const int pmax = p.gc ? kPspBlock : kPsp;
    const int P = nsym < pmax ? (int)nsym : pmax;
    if (threadIdx.x < kPsp) pidx[w_ * kPsp + threadIdx.x] = threadIdx.x < P ? si[threadIdx.x] : -1;
    if (threadIdx.x == 0) pcount[w_] = P;
}

__global__ void __launch_bounds__(kSelThreads) psp_select_kernel(const DavProb *__restrict__ probs, long long *__restrict__ pidx, int *__restrict__ pcount, int nprob_) {
    for (int w = blockIdx.x; w < nprob_; w += gridDim.x) {
        psp_select_kernel_body(probs, pidx, pcount, w);
        __syncthreads();   // shared memory is reused by the next body
    }
}

// Per problem (kPsp threads): H in the pair functions, its lowest eigenvectors
// by cyclic Jacobi (rotations applied by all threads), written to the start
// slots 0..nv-1; the random start vector is cleared on the P-space determinants.
__device__ __forceinline__ void psp_solve_kernel_body(const DavProb *__restrict__ probs, const HdiagDesc *__restrict__ hdd, const long long *__restrict__ pidx,
                 const int *__restrict__ pcount, const DavState *__restrict__ st, int max_space,
                 double *__restrict__ blk_energy, int w_) {
    extern __shared__ double psm[];
    double *A = psm;                       // [kPsp][kPsp]
    double *V = psm + kPsp * kPsp;         // [kPsp][kPsp]
    __shared__ double red[kPsp], red2[kPsp];
    const DavProb p = probs[w_];
    const HdiagDesc d = hdd[w_];
    const int P = pcount[w_];
    const int t = threadIdx.x;
    const int n = p.nb;
    const double rs2 = 0.7071067811865476;
    // row t of A: <u_t|H|u_c>, every term of the pair functions written out (in
    // an off-diagonal block, whose spin-flip image is not iterated, u_K = |K>)
    if (t < P) {
        const long long K = pidx[w_ * kPsp + t];
        const int ka = (int)(K / n), kb = (int)(K % n);
        for (int c = 0; c < P; c++) {
            const long long L = pidx[w_ * kPsp + c];
            const int la = (int)(L / n), lb = (int)(L % n);
            const int nbra = (ka == kb || !p.sym) ? 1 : 2, nket = (la == lb || !p.sym) ? 1 : 2;
            const double f = (nbra == 2 ? rs2 : 1.0) * (nket == 2 ? rs2 : 1.0);
            double v = 0.0;
            for (int x = 0; x < nbra; x++)
                for (int y = 0; y < nket; y++) {
                    // (row, column) local indices of the bra and ket determinants
                    const int ba = x ? kb : ka, bb = x ? ka : kb, ca = y ? lb : la, cb = y ? la : lb;
                    v += h_element(d.n, d.h1, d.eri, (uint32_t)d.strings[blk_row(p, ba)],
                                   (uint32_t)d.strings[blk_col(p, bb)], (uint32_t)d.strings[blk_row(p, ca)],
                                   (uint32_t)d.strings[blk_col(p, cb)]);
                }
            A[t * kPsp + c] = f * v;
            V[t * kPsp + c] = t == c ? 1.0 : 0.0;
        }
    }
    // blocks of the P-space: connected components of the coupling graph
    // (|A_ij| above 1e-12 of the largest element); distant bodies make H split
    // into (nearly) decoupled sectors, and the start block takes the lowest
    // eigenvector of each of the lowest blocks first
    __shared__ int comp[kPsp];
    if (t == 0) {
        double amax = 0.0;
        for (int i = 0; i < P; i++)
            for (int c = 0; c < P; c++) amax = fmax(amax, fabs(A[i * kPsp + c]));
        const double thr = 1e-12 * amax;
        for (int i = 0; i < P; i++) comp[i] = -1;
        int ncomp = 0;
        int stack[kPsp];
        for (int i = 0; i < P; i++) {
            if (comp[i] >= 0) continue;
            int top = 0;
            stack[top++] = i;
            comp[i] = ncomp;
            while (top > 0) {
                const int u = stack[--top];
                for (int v = 0; v < P; v++)
                    if (comp[v] < 0 && fabs(A[u * kPsp + v]) > thr) {
                        comp[v] = ncomp;
                        stack[top++] = v;
                    }
            }
            ncomp++;
        }
    }
    __syncthreads();
    // sweeps until the off-diagonal part is below 1e-26 of |A|_F^2 (a start
    // guess needs no more); a rotation whose A_pq is below 1e-18 (|A_pp| +
    // |A_qq|) only sets A_pq = A_qp = 0
    for (int sweep = 0; sweep < 40; sweep++) {
        double off = 0.0, all = 0.0;
        if (t < P)
            for (int c = 0; c < P; c++) {
                const double a2 = A[t * kPsp + c] * A[t * kPsp + c];
                all += a2;
                if (c != t) off += a2;
            }
        red[t] = off;
        red2[t] = all;
        __syncthreads();
        double tot = 0.0, fro = 0.0;
        for (int i = 0; i < P; i++) {
            tot += red[i];
            fro += red2[i];
        }
        __syncthreads();
        if (tot <= 1e-26 * fro || tot == 0.0) break;
        for (int pp = 0; pp < P - 1; pp++)
            for (int q = pp + 1; q < P; q++) {
                // every thread reads the same settled entries and derives the same
                // rotation (no barrier); zero couplings (other sectors, pair
                // functions beyond a double excitation apart) are skipped
                const double apq = A[pp * kPsp + q];
                if (fabs(apq) < 1e-300) continue;
                const double app = A[pp * kPsp + pp], aqq = A[q * kPsp + q];
                if (fabs(apq) <= 1e-18 * (fabs(app) + fabs(aqq))) {
                    __syncthreads();   // every thread has read A[pp][q]
                    if (t == 0) A[pp * kPsp + q] = A[q * kPsp + pp] = 0.0;
                    __syncthreads();
                    continue;
                }
                double c, sn;
                jacobi_rotation(app, aqq, apq, c, sn);
                __syncthreads();   // every thread has read A[pp][q], A[pp][pp], A[q][q]
                if (t < P) {
                    const double arp = A[t * kPsp + pp], arq = A[t * kPsp + q];
                    A[t * kPsp + pp] = c * arp - sn * arq;
                    A[t * kPsp + q] = sn * arp + c * arq;
                }
                __syncthreads();
                if (t < P) {
                    const double apr = A[pp * kPsp + t], aqr = A[q * kPsp + t];
                    A[pp * kPsp + t] = c * apr - sn * aqr;
                    A[q * kPsp + t] = sn * apr + c * aqr;
                    const double vrp = V[t * kPsp + pp], vrq = V[t * kPsp + q];
                    V[t * kPsp + pp] = c * vrp - sn * vrq;
                    V[t * kPsp + q] = sn * vrp + c * vrq;
                }
                __syncthreads();
            }
    }
    // the nv lowest eigenvalues' columns, each sign fixed by its largest component
    int nv, ns;
    start_block(p.ndim, max_space, p.seed != nullptr, &nv, &ns);
    if (p.seed) return;   // started from its own vector: no P-space guess
    __shared__ int cols[kStartP];
    if (t == 0) {
        // eigenvalues in ascending order; each eigenvector's block is the block
        // of its largest component
        int order[kPsp], blk[kPsp];
        bool used[kPsp];
        for (int i = 0; i < P; i++) used[i] = false;
        for (int r = 0; r < P; r++) {
            int b = -1;
            for (int i = 0; i < P; i++)
                if (!used[i] && (b < 0 || A[i * kPsp + i] < A[b * kPsp + b])) b = i;
            used[b] = true;
            order[r] = b;
            int g = 0;
            for (int i = 1; i < P; i++)
                if (fabs(V[i * kPsp + b]) > fabs(V[g * kPsp + b])) g = i;
            blk[r] = comp[g];
        }
        // rank of each block by its lowest eigenvalue: first[] = the eigenpair
        // index (in ascending order) that opens block rank 0, 1, ...
        int first[kPsp], nb = 0;
        for (int r = 0; r < P; r++) {
            bool opens = true;
            for (int q = 0; q < r; q++)
                if (blk[q] == blk[r]) opens = false;
            if (opens) first[nb++] = r;
        }
        if (blk_energy) {
            blk_energy[2 * w_] = A[order[first[0]] * kPsp + order[first[0]]];
            blk_energy[2 * w_ + 1] = nb > 1 ? A[order[first[1]] * kPsp + order[first[1]]] : 1e300;
        }
        bool taken[kPsp];
        for (int r = 0; r < P; r++) taken[r] = false;
        int nc = 0;
        const int seed = p.seed_block;
        if (seed > 0 && seed < nb) {
            // second pass: that block's lowest vector first, then the lowest
            // eigenvectors outside the blocks ranked below it
            cols[nc++] = order[first[seed]];
            taken[first[seed]] = true;
            for (int r = 0; r < P && nc < nv; r++) {
                bool lower = false;
                for (int q = 0; q < seed; q++)
                    if (blk[r] == blk[first[q]]) lower = true;
                if (!taken[r] && !lower) {
                    cols[nc++] = order[r];
                    taken[r] = true;
                }
            }
        } else {
            // first the lowest eigenvector of each block (in order of those
            // eigenvalues), then the next lowest eigenvectors
            for (int k = 0; k < nb && nc < nv; k++) {
                cols[nc++] = order[first[k]];
                taken[first[k]] = true;
            }
        }
        for (int r = 0; r < P && nc < nv; r++)
            if (!taken[r]) {
                cols[nc++] = order[r];
                taken[r] = true;
            }
    }
    __syncthreads();
    if (t < P) {
        const long long K = pidx[w_ * kPsp + t];
        const int ka = (int)(K / n), kb = (int)(K % n);
        const long long KT = (long long)kb * n + ka;
        for (int r = 0; r < nv; r++) {
            const int col = cols[r];
            int g = 0;
            for (int i = 1; i < P; i++)
                if (fabs(V[i * kPsp + col]) > fabs(V[g * kPsp + col])) g = i;
            const double y = (V[g * kPsp + col] < 0 ? -1.0 : 1.0) * V[t * kPsp + col];
            double *Br = p.B + (long long)r * p.ndet;
            if (ka == kb || !p.sym) {
                Br[K] = y;
            } else {
                Br[K] = y * rs2;
                Br[KT] = y * rs2;
            }
        }
        if (ns >= 0) {   // the random vector becomes exactly orthogonal to the block
            double *Bn = p.B + (long long)ns * p.ndet;
            Bn[K] = 0.0;
            if (p.sym) Bn[KT] = 0.0;
        }
    }
}

__global__ void __launch_bounds__(kPsp) psp_solve_kernel(const DavProb *__restrict__ probs, const HdiagDesc *__restrict__ hdd, const long long *__restrict__ pidx,
                 const int *__restrict__ pcount, const DavState *__restrict__ st, int max_space,
                 double *__restrict__ blk_energy, int nprob_) {
    for (int w = blockIdx.x; w < nprob_; w += gridDim.x) {
        psp_solve_kernel_body(probs, hdd, pidx, pcount, st, max_space, blk_energy, w);
        __syncthreads();   // shared memory is reused by the next body
    }
}

// partial |.|^2 of the random start vector per vector work item
__device__ __forceinline__ void norm_part_kernel_body(const DavProb *__restrict__ probs,
                                                        const DavState *__restrict__ st,
                                                        const WorkItem *__restrict__ items, double *__restrict__ part, int w_) {
    const WorkItem it = items[w_];
    const DavProb &p = probs[it.prob];
    const int ns = st[it.prob].noise_slot;
    double acc = 0.0;
    const long long end = min(it.start + (long long)kVecChunk, p.ndet);
    if (ns >= 0) {
        const double *v = p.B + (long long)ns * p.ndet;
        for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) acc += v[I] * v[I];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < 8; i++) s += red[i];
        part[(long long)w_ * kNP] = s;
    }
}

__global__ void __launch_bounds__(256) norm_part_kernel(const DavProb *__restrict__ probs,
                                                        const DavState *__restrict__ st,
                                                        const WorkItem *__restrict__ items, double *__restrict__ part, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) {
        norm_part_kernel_body(probs, st, items, part, w);
        __syncthreads();   // shared memory is reused by the next body
    }
}

// <bra_k|H|ket_k> for determinant index pairs (C entry point below)
__global__ void h_elements_kernel(int n, int nstr, const uint64_t *__restrict__ strings,
                                  const double *__restrict__ h1, const double *__restrict__ eri, long long count,
                                  const long long *__restrict__ bra, const long long *__restrict__ ket,
                                  double *__restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const long long I = bra[i], J = ket[i];
    out[i] = h_element(n, h1, eri, (uint32_t)strings[I / nstr], (uint32_t)strings[I % nstr],
                       (uint32_t)strings[J / nstr], (uint32_t)strings[J % nstr]);
}

}  // namespace

size_t psp_workspace_bytes(int nprob) {
    return ws_round((size_t)nprob * kPsp * sizeof(long long)) + ws_round((size_t)nprob * sizeof(int));
}

// Fills the P-space slots of every problem's start block, clears the random
// start vector on the P-space determinants and stores its |.|^2 per item in
// part (the caller normalises it).
int launch_pspace_start(ifci_handle_t h, const DavBatch &b, const HdiagDesc *d_hd, cudaStream_t s) {
    long long *pidx = b.d_pidx;
    int *pcount = b.d_pcount;
    if (!pidx || !pcount) return set_error(h, IFCI_ERR_OOM, "davidson: workspace (P-space)");
    {
        ProfScope ps(h, s, PK_SETUP);
        psp_select_kernel<<<stride_grid(h->device, b.nprob, 8), kSelThreads, 0, s>>>(b.d_probs, pidx, pcount, b.nprob);
        IFCI_LAUNCH_CHECK(h);
    }
    const int smem = 2 * kPsp * kPsp * (int)sizeof(double);   // 64 KB
    static SmemOptIn opt;
    IFCI_CUDA_TRY(h, ensure_smem(opt, h->device, psp_solve_kernel, smem));
    {
        ProfScope ps(h, s, PK_PSPACE);
        psp_solve_kernel<<<stride_grid(h->device, b.nprob, 3), kPsp, smem, s>>>(b.d_probs, d_hd, pidx, pcount,
                                                                                 b.d_state, b.max_space,
                                                                                 b.d_blk_energy, b.nprob);
        IFCI_LAUNCH_CHECK(h);
    }
    ProfScope ps(h, s, PK_SETUP);
    norm_part_kernel<<<stride_grid(h->device, (long long)b.vitems.size(), 8), 256, 0, s>>>(b.d_probs, b.d_state, b.d_vitems, b.d_part, (int)b.vitems.size());
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

}  // namespace ifci

extern "C" int ifci_h_elements(ifci_handle_t h, const ifci_strings_t *str, const double *h1, const double *eri,
                               long long count, const long long *bra, const long long *ket, double *out,
                               ifci_stream_t stream) {
    using namespace ifci;
    if (!h) return IFCI_ERR_INVALID_ARG;
    if (!str || !str->strings || !h1 || !eri || count < 0 || (count > 0 && (!bra || !ket || !out)))
        return set_error(h, IFCI_ERR_INVALID_ARG, "ifci_h_elements: bad arguments");
    int nstr = 0, nexc = 0;
    if (ifci_string_counts(str->norb, str->nelec_spin, &nstr, &nexc) != IFCI_OK || nstr != str->nstr)
        return set_error(h, IFCI_ERR_INVALID_ARG, "ifci_h_elements: inconsistent string table");
    if (count == 0) return IFCI_OK;
    IFCI_CUDA_TRY(h, cudaSetDevice(h->device));
    const int threads = 128;
    const long long blocks = (count + threads - 1) / threads;
    h_elements_kernel<<<(unsigned)blocks, threads, 0, as_cuda(stream)>>>(str->norb, nstr, str->strings, h1, eri,
                                                                          count, bra, ket, out);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}
