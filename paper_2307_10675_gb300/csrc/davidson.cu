// Batched Davidson for the lowest singlet root of many CI problems at once.
//
// Every step is a batched kernel over all problems still iterating; the
// per-problem state (subspace size, Ritz value, flags) lives on the device, so
// the host only launches and reads one counter per iteration.  All
// orthogonalisation, Rayleigh quotients and residuals are FP64.
//
// Vector passes of one iteration (k = subspace size):
//   sigma(b_new) -> subspace column <b_j|sigma_new> -> k x k Jacobi eigen-solve
//   -> residual r = sum_j y_j (sigma_j - theta b_j), correction t = r / (theta - H_II)
//   -> classical Gram-Schmidt (a second pass when the first removed more than
//   half of |t|^2) -> normalise, symmetrise (c = c^T sector).
//
// A full subspace restarts thick: it keeps the lowest Ritz vectors (up to
// kKeep, with their sigmas and a diagonal projected matrix) plus the new
// correction, so a near-degenerate pair of lowest states stays resolved by
// Rayleigh-Ritz instead of being found again after each restart.
//
// Two precisions of sigma (mixed mode), in two phases per problem.  Phase 1
// builds every sigma in the low precision (thick restarts as above) and never
// declares convergence: its residual is only as good as the low-precision
// sigma.  When that residual stops halving between restarts, falls below
// 10 r_tol, or half of max_iter is spent, the problem keeps its lowest Ritz
// vectors, rebuilds their exact (FP64 or FP64-accurate) sigmas one per
// iteration, and continues as the exact solver, whose Rayleigh quotients and
// residuals decide convergence.  The low-precision Rayleigh-Ritz may misorder
// states closer than its rounding, but it keeps them among the lowest Ritz
// vectors, and the first exact Rayleigh-Ritz over those picks the lowest.
#include <algorithm>
#include <cmath>

#include "dav_driver.cuh"
#include "hamiltonian.cuh"
#include "slater.cuh"

namespace ifci {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block reduction of NV values per thread into out[0..NV).  256 threads.
template <int NV>
__device__ void block_sum_store(double (&v)[NV], int nv, double *out) {
    __shared__ double red[8][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; j++) {
        if (j < nv) {
            double s = warp_sum(v[j]);
            if (lane == 0) red[warp][j] = s;
        }
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double s = 0.0;
        for (int w = 0; w < 8; w++) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// ------------------------------------------------------------------ setup

// Start block (orthonormal, its sigmas built one per iteration before the
// first correction): the lowest eigenvectors of H in the pair functions of the
// lowest-diagonal determinants (pspace.cu), which can lie in different
// symmetry classes of H, and a deterministic pseudo-random symmetric vector
// that gives the subspace a nonzero overlap with every state of the
// spin-flip-even sector.

__device__ __forceinline__ void init_kernel_body(const DavProb *__restrict__ probs, DavState *__restrict__ st, int max_space, int w_) {
    const DavProb p = probs[w_];
    __shared__ double bv[256];
    __shared__ long long bi[256];
    double best = 1e300;
    long long besti = 0;
    for (long long i = threadIdx.x; i < p.ndet; i += blockDim.x) {
        double v = p.hd[i];
        if (v < best) { best = v; besti = i; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            double v2 = bv[threadIdx.x + o];
            long long i2 = bi[threadIdx.x + o];
            if (v2 < bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
                bv[threadIdx.x] = v2;
                bi[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        DavState s{};
        s.k = 1;
        s.newest = 0;
        s.active = 1;
        s.restart = 0;
        s.iters = 0;
        s.status = IFCI_ERR_NOT_CONVERGED;
        s.tslot = -1;
        s.ref = bi[0];
        s.force = 0;
        s.theta = bv[0];
        s.theta_prev = 1e300;
        s.rnorm = 1e300;
        s.tnorm2 = 0.0;
        s.energy = 0.0;
        int nv, ns;
        start_block(p.ndim, max_space, p.seed != nullptr, &nv, &ns);
        s.noise_slot = ns;
        s.tgt = 0;
        for (int r = 0; r < kKeep; r++) s.rn[r] = 1e300;
        s.rebuild_to = nv + (ns >= 0 ? 1 : 0);   // sigmas of the start block, one per iteration
        st[w_] = s;
    }
}

__global__ void init_kernel(const DavProb *__restrict__ probs, DavState *__restrict__ st, int max_space, int nprob_) {
    for (int w = blockIdx.x; w < nprob_; w += gridDim.x) {
        init_kernel_body(probs, st, max_space, w);
        __syncthreads();   // shared memory is reused by the next body
    }
}

// symmetric pseudo-random value in [-1, 1) of the unordered string pair {a, b}
__device__ __forceinline__ double pair_noise(int a, int b) {
    unsigned long long lo = (unsigned long long)min(a, b), hi = (unsigned long long)max(a, b);
    unsigned long long x = (hi << 32) ^ lo ^ 0x9E3779B97F4A7C15ull;
    x ^= x >> 30; x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27; x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Start block: the P-space slots 0..nv-1 zeroed (pspace.cu fills them), the
// random vector in the noise slot (normalised after pspace.cu has cleared it
// on the P-space determinants; a function of the global string pair, so it is
// symmetric in a symmetric block).  A problem with a start vector of its own
// copies it to slot 0.
__device__ __forceinline__ void init_vec_kernel_body(const DavProb *__restrict__ probs,
                                                       const WorkItem *__restrict__ items, int max_space, int w_) {
    const WorkItem it = items[w_];
    const DavProb &p = probs[it.prob];
    int nv, ns;
    start_block(p.ndim, max_space, p.seed != nullptr, &nv, &ns);
    long long end = min(it.start + (long long)kVecChunk, p.ndet);
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
        if (p.seed) {
            p.B[I] = p.seed[I];
            continue;
        }
        for (int r = 0; r < nv; r++) p.B[(long long)r * p.ndet + I] = 0.0;
        if (ns >= 0) {
            const int a = (int)(I / p.nb), b = (int)(I % p.nb);
            p.B[(long long)ns * p.ndet + I] = pair_noise(blk_row(p, a), blk_col(p, b));
        }
    }
}

__global__ void __launch_bounds__(256) init_vec_kernel(const DavProb *__restrict__ probs,
                                                       const WorkItem *__restrict__ items, int max_space, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) init_vec_kernel_body(probs, items, max_space, w);
}

// normalise the noise slot of the start block (part: its |.|^2 per item)
__device__ __forceinline__ void init_scale_kernel_body(const DavProb *__restrict__ probs,
                                                         const DavState *__restrict__ st,
                                                         const WorkItem *__restrict__ items,
                                                         const double *__restrict__ part, int w_) {
    const WorkItem it = items[w_];
    const DavProb &p = probs[it.prob];
    const int ns = st[it.prob].noise_slot;
    if (ns < 0) return;
    double n2 = 0.0;
    for (int w = 0; w < p.nitem; w++) n2 += part[(long long)(p.item0 + w) * kNP];
    const double inv = 1.0 / sqrt(n2);
    double *v = p.B + (long long)ns * p.ndet;
    long long end = min(it.start + (long long)kVecChunk, p.ndet);
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) v[I] *= inv;
}

__global__ void __launch_bounds__(256) init_scale_kernel(const DavProb *__restrict__ probs,
                                                         const DavState *__restrict__ st,
                                                         const WorkItem *__restrict__ items,
                                                         const double *__restrict__ part, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) init_scale_kernel_body(probs, st, items, part, w);
}

// sigma selectors: the hi plan (FP64 or FP64-accurate) for exact problems, the
// lo plan for mixed-mode problems still in phase 1
__global__ void select_kernel(const DavState *__restrict__ st, int nprob, int mixed, int *__restrict__ hi,
                              int *__restrict__ lo) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nprob) return;
    const DavState s = st[i];
    int a = s.active;
    if (mixed) {
        hi[i] = a && s.exact_all;
        lo[i] = a && !s.exact_all;
    } else {
        hi[i] = a;
        lo[i] = 0;
    }
}

// ------------------------------------------------------------------ subspace

// partial[item][j] = <b_j | sigma_new> over the item's determinants, j <= newest.
__device__ __forceinline__ void dots_kernel_body(const DavProb *__restrict__ probs, const DavState *__restrict__ st,
                                                   const WorkItem *__restrict__ items, double *__restrict__ part, int w_) {
    const WorkItem it = items[w_];
    const DavState s = st[it.prob];
    if (!s.active) return;
    const DavProb &p = probs[it.prob];
    const int k = s.newest + 1;
    double acc[kMaxSpace];
#pragma unroll
    for (int j = 0; j < kMaxSpace; j++) acc[j] = 0.0;
    const double *Sn = p.S + (long long)s.newest * p.ndet;
    long long end = min(it.start + (long long)kVecChunk, p.ndet);
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
        const double sv = Sn[I];
#pragma unroll
        for (int j = 0; j < kMaxSpace; j++)
            if (j < k) acc[j] += p.B[(long long)j * p.ndet + I] * sv;
    }
    block_sum_store<kMaxSpace>(acc, k, part + (long long)w_ * kNP);
}

__global__ void __launch_bounds__(256) dots_kernel(const DavProb *__restrict__ probs, const DavState *__restrict__ st,
                                                   const WorkItem *__restrict__ items, double *__restrict__ part, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) {
        dots_kernel_body(probs, st, items, part, w);
        __syncthreads();   // shared memory is reused by the next body
    }
}

// Cyclic Jacobi on the symmetric k x k matrix A (shared memory, row stride
// kSolveLd) by one warp: every lane derives the same rotation from the
// settled entries, then lane r rotates row r / column r (columns, rows and V
// in turn, as the serial sweep does, so the arithmetic per element is the
// same).  A sweep ends the iteration once the off-diagonal part is below
// 1e-26 of |A|_F^2 (eigenvalue errors ~1e-26 |A| / gap); a rotation whose
// A_pq is below 1e-18 (|A_pp| + |A_qq|) only sets A_pq = A_qp = 0.
constexpr int kSolveLd = kMaxSpace + 1;
constexpr int kSolveWarps = 4;

__device__ void jacobi_warp(double *A, double *V, int k, int lane) {
    if (lane < k)
        for (int j = 0; j < k; j++) V[lane * kSolveLd + j] = lane == j ? 1.0 : 0.0;
    __syncwarp();
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0, tot = 0.0;
        if (lane < k)
            for (int j = 0; j < k; j++) {
                const double a = A[lane * kSolveLd + j];
                tot += a * a;
                if (j != lane) off += a * a;
            }
        off = warp_sum(off);
        tot = warp_sum(tot);
        if (off <= 1e-26 * tot || off == 0.0) break;
        for (int pp = 0; pp < k - 1; pp++)
            for (int q = pp + 1; q < k; q++) {
                const double apq = A[pp * kSolveLd + q];
                if (apq == 0.0) continue;
                const double app = A[pp * kSolveLd + pp], aqq = A[q * kSolveLd + q];
                __syncwarp();   // every lane has read the rotation's entries
                if (fabs(apq) <= 1e-18 * (fabs(app) + fabs(aqq))) {
                    if (lane == 0) A[pp * kSolveLd + q] = A[q * kSolveLd + pp] = 0.0;
                    __syncwarp();
                    continue;
                }
                double c, sn;
                jacobi_rotation(app, aqq, apq, c, sn);
                if (lane < k) {
                    const double arp = A[lane * kSolveLd + pp], arq = A[lane * kSolveLd + q];
                    A[lane * kSolveLd + pp] = c * arp - sn * arq;
                    A[lane * kSolveLd + q] = sn * arp + c * arq;
                }
                __syncwarp();
                if (lane < k) {
                    const double apr = A[pp * kSolveLd + lane], aqr = A[q * kSolveLd + lane];
                    A[pp * kSolveLd + lane] = c * apr - sn * aqr;
                    A[q * kSolveLd + lane] = sn * apr + c * aqr;
                    const double vrp = V[lane * kSolveLd + pp], vrq = V[lane * kSolveLd + q];
                    V[lane * kSolveLd + pp] = c * vrp - sn * vrq;
                    V[lane * kSolveLd + q] = sn * vrp + c * vrq;
                }
                __syncwarp();
            }
    }
}

// One warp per problem: finish the subspace column and solve the projected
// problem (its kKeep lowest Ritz pairs).
__device__ __forceinline__ void solve_warp_body(const DavProb *__restrict__ probs, DavState *__restrict__ st,
                                                const double *__restrict__ part, double *__restrict__ gs,
                                                double *__restrict__ ys, int i, double *A, double *V) {
    const int lane = threadIdx.x & 31;
    DavState s = st[i];
    if (!s.active) return;
    const DavProb &p = probs[i];
    const int k = s.newest + 1;
    double *Gm = gs + (long long)i * kMaxSpace * kMaxSpace;
    if (lane < k) {
        double v = 0.0;
        for (int w = 0; w < p.nitem; w++) v += part[(long long)(p.item0 + w) * kNP + lane];
        Gm[lane * kMaxSpace + s.newest] = v;
        Gm[s.newest * kMaxSpace + lane] = v;
    }
    __syncwarp();
    if (lane < k)
        for (int b = 0; b < k; b++) A[lane * kSolveLd + b] = 0.5 * (Gm[lane * kMaxSpace + b] + Gm[b * kMaxSpace + lane]);
    __syncwarp();
    jacobi_warp(A, V, k, lane);
    if (lane == 0) {
        // the nk lowest eigenpairs in ascending order; each vector's largest
        // component made positive (deterministic sign)
        const int nk = k < kKeep ? k : kKeep;
        double *yo = ys + (long long)i * kYStride;
        bool used[kMaxSpace];
        for (int j = 0; j < k; j++) used[j] = false;
        for (int r = 0; r < kKeep; r++) {
            if (r >= nk) {
                for (int j = 0; j < kNP; j++) yo[r * kNP + j] = 0.0;
                continue;
            }
            int best = -1;
            for (int j = 0; j < k; j++)
                if (!used[j] && (best < 0 || A[j * kSolveLd + j] < A[best * kSolveLd + best])) best = j;
            used[best] = true;
            int big = 0;
            for (int j = 1; j < k; j++)
                if (fabs(V[j * kSolveLd + best]) > fabs(V[big * kSolveLd + best])) big = j;
            const double sg = V[big * kSolveLd + best] < 0 ? -1.0 : 1.0;
            for (int j = 0; j < kNP; j++) yo[r * kNP + j] = j < k ? sg * V[j * kSolveLd + best] : 0.0;
            yo[r * kNP + kMaxSpace] = A[best * kSolveLd + best];
            if (r == 0) s.theta = A[best * kSolveLd + best];
        }
        s.iters += 1;
        st[i] = s;
    }
    __syncwarp();   // A and V are reused by the warp's next problem
}

__global__ void __launch_bounds__(32 * kSolveWarps) solve_kernel(const DavProb *__restrict__ probs,
                                                                 DavState *__restrict__ st,
                                                                 const double *__restrict__ part,
                                                                 double *__restrict__ gs, double *__restrict__ ys,
                                                                 int nprob_) {
    __shared__ double sm[kSolveWarps][2][kMaxSpace * kSolveLd];
    const int warp = threadIdx.x >> 5;
    for (int w = blockIdx.x * kSolveWarps + warp; w < nprob_; w += gridDim.x * kSolveWarps)
        solve_warp_body(probs, st, part, gs, ys, w, sm[warp][0], sm[warp][1]);
}

// For the targeted Ritz pair (theta, y): t = sum_j y_j (S_j - theta B_j);
// ||t||^2; t /= (theta - H_II); dots <b_j|t>.
__device__ __forceinline__ void residual_kernel_body(const DavProb *__restrict__ probs,
                                                       const DavState *__restrict__ st,
                                                       const WorkItem *__restrict__ items,
                                                       const double *__restrict__ ys, int max_space,
                                                       double *__restrict__ part, int w_) {
    const WorkItem it = items[w_];
    const DavState s = st[it.prob];
    if (!s.active) return;
    const DavProb &p = probs[it.prob];
    const int k = s.newest + 1;
    // the targeted Ritz root (rank tgt among the lowest kKeep)
    const int tgt = s.tgt < min(k, kKeep) ? s.tgt : 0;
    const double *yt = ys + (long long)it.prob * kYStride + tgt * kNP;
    const double theta = yt[kMaxSpace];
    double y[kMaxSpace];
#pragma unroll
    for (int j = 0; j < kMaxSpace; j++) y[j] = yt[j];
    double acc[kMaxSpace + 2];
#pragma unroll
    for (int j = 0; j < kMaxSpace + 2; j++) acc[j] = 0.0;
    double *T = p.B + (long long)max_space * p.ndet;   // scratch slot for the correction
    long long end = min(it.start + (long long)kVecChunk, p.ndet);
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
        double r = 0.0;
        double bv[kMaxSpace];
#pragma unroll
        for (int j = 0; j < kMaxSpace; j++) {
            if (j < k) {
                bv[j] = p.B[(long long)j * p.ndet + I];
                r += y[j] * (p.S[(long long)j * p.ndet + I] - theta * bv[j]);
            }
        }
        acc[kMaxSpace + 1] += r * r;
        double den = theta - p.hd[I];
        if (fabs(den) < 1e-4) den = den < 0 ? -1e-4 : 1e-4;
        double t = r / den;
        T[I] = t;
#pragma unroll
        for (int j = 0; j < kMaxSpace; j++)
            if (j < k) acc[j] += bv[j] * t;
        acc[kMaxSpace] += t * t;
    }
    // layout of part: [0..k) dots, kMaxSpace: |t|^2, kMaxSpace+1: |r|^2
    __shared__ double red[8][kMaxSpace + 2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kMaxSpace + 2; j++) {
        if (j < k || j >= kMaxSpace) {
            double v = warp_sum(acc[j]);
            if (lane == 0) red[warp][j] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < kMaxSpace + 2 && (threadIdx.x < k || threadIdx.x >= kMaxSpace)) {
        double v = 0.0;
        for (int w = 0; w < 8; w++) v += red[w][threadIdx.x];
        part[(long long)w_ * kNP + threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(256) residual_kernel(const DavProb *__restrict__ probs,
                                                       const DavState *__restrict__ st,
                                                       const WorkItem *__restrict__ items,
                                                       const double *__restrict__ ys, int max_space,
                                                       double *__restrict__ part, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) {
        residual_kernel_body(probs, st, items, ys, max_space, part, w);
        __syncthreads();   // shared memory is reused by the next body
    }
}

// Convergence test, restart decision, CGS coefficients.  One block per problem.
__device__ __forceinline__ void check_kernel_body(const DavProb *__restrict__ probs, DavState *__restrict__ st,
                             const double *__restrict__ part, double *__restrict__ coef, const double *__restrict__ ys,
                             double *__restrict__ gs, int max_space, int restart_at, int keep_max, int mixed,
                             int max_iter, double e_tol, double r_tol, int *__restrict__ nactive, int w_) {
    const int i = w_;
    DavState s = st[i];
    if (!s.active) return;
    const DavProb p = probs[i];
    const int k = s.newest + 1;
    __shared__ double sum[kMaxSpace + 2];
    if (threadIdx.x < kMaxSpace + 2 && (threadIdx.x < k || threadIdx.x >= kMaxSpace)) {
        double v = 0.0;
        for (int w = 0; w < p.nitem; w++) v += part[(long long)(p.item0 + w) * kNP + threadIdx.x];
        sum[threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    s.rnorm = sqrt(sum[kMaxSpace + 1]);
    const double *ys_i = ys + (long long)i * kYStride;
    const bool lowmix = mixed && !s.exact_all;   // phase 1: every sigma in low precision
    const int nk = min(k, kKeep);
    const int tgt = s.tgt < nk ? s.tgt : 0;
    s.rn[tgt] = s.rnorm;
    s.tcur = tgt;
    if (s.rebuild_to > 0) {
        if (k < s.rebuild_to) {
            // phase switch: the kept Ritz vectors still wait for exact sigmas; no
            // check and no correction (advance_kernel moves to the next slot)
            atomicAdd(nactive, 1);
            s.restart = 0;
            s.tslot = -1;
            st[i] = s;
            return;
        }
        s.rebuild_to = 0;   // every basis vector has its exact sigma: a normal iteration
    }
    // a competitive higher root: within kCompete of the lowest and not yet
    // resolved.  A problem started from a vector of its own refines that root
    // only (its sector was chosen before), and so does a block of a sectored
    // space: the search over its decoupled sectors is the set of blocks
    const double tol2 = fmax(sqrt(r_tol), 10.0 * r_tol);
    int comp = -1;
    for (int r = 1; r < nk && comp < 0 && !p.seed && !p.gc; r++)
        if (ys_i[r * kNP + kMaxSpace] - ys_i[kMaxSpace] < kCompete && s.rn[r] > tol2) comp = r;
    // only exact sigmas decide convergence: the lowest root's residual below
    // r_tol, a settled energy, and no competitive root left unresolved
    const bool conv = !lowmix && tgt == 0 && s.rnorm < r_tol && fabs(s.theta - s.theta_prev) < e_tol && comp < 0;
    if (!lowmix && tgt == 0) s.theta_prev = s.theta;
    // next target: a competitive root after each correction of the lowest one,
    // and for as long as the lowest one is already converged
    s.tgt = (comp > 0 && (tgt == 0 || s.rn[0] < r_tol)) ? comp : 0;
    if (conv || (!lowmix && tgt == 0 && s.rnorm == 0.0)) {
        s.active = 0;
        s.status = IFCI_OK;
        s.energy = s.theta + p.e_core;
        s.tslot = -1;
        st[i] = s;
        return;
    }
    if (s.iters >= max_iter) {
        s.active = 0;
        s.status = IFCI_ERR_NOT_CONVERGED;
        s.energy = s.theta + p.e_core;
        s.tslot = -1;
        st[i] = s;
        return;
    }
    atomicAdd(nactive, 1);
    double *c = coef + (long long)i * kNP;
    double *Gm = gs + (long long)i * kMaxSpace * kMaxSpace;
    // dimension of the space iterated (the spin-flip-even sector of a symmetric block)
    const long long nsym = p.ndim;
    const int ra = lowmix ? restart_at : max_space;
    if (k >= ra || k >= nsym || s.force) {
        const bool exhausted = k >= nsym || s.force;
        s.force = 0;
        s.restart = 1;
        s.kold = k;
        bool to_exact = false;
        if (lowmix) {
            const double r0 = s.rn[0];   // lowest root's latest residual
            to_exact = exhausted || r0 < 10.0 * r_tol || 2 * s.iters >= max_iter ||
                       (s.rnorm_exact_prev > 0.0 && r0 > 0.5 * s.rnorm_exact_prev);
            s.rnorm_exact_prev = r0;
        }
        if (to_exact) {
            // phase 2 keeps the lowest Ritz vectors; their exact sigmas are built
            // over the next iterations (slot 0 first), the correction is dropped
            const int keep = min(keep_max, k);
            s.exact_all = 1;
            s.nform = keep;
            s.rebuild_to = keep;
            s.tgt = 0;
            for (int r = 0; r < kKeep; r++) s.rn[r] = 1e300;   // exact residuals from here on
            s.k = 1;
            s.newest = 0;
            s.tslot = -1;
        } else {
            // thick restart: basis becomes [x_0 .. x_{keep-1}, t] with the lowest
            // Ritz vectors x_r = sum_j Y_r[j] b_j (projected matrix diag(theta_r))
            // and <x_r|t> = sum_j Y_r[j] <b_j|t>
            const int keep = min(keep_max, k);
            for (int j = 0; j < kNP; j++) c[j] = 0.0;
            for (int r = 0; r < keep; r++) {
                double xt = 0.0;
                for (int j = 0; j < k; j++) xt += ys_i[r * kNP + j] * sum[j];
                c[r] = xt;
            }
            for (int a = 0; a < keep; a++)
                for (int b2 = 0; b2 < keep; b2++) Gm[a * kMaxSpace + b2] = a == b2 ? ys_i[a * kNP + kMaxSpace] : 0.0;
            s.k = keep;
            s.nform = keep;
            s.tslot = keep;
        }
    } else {
        s.restart = 0;
        for (int j = 0; j < kNP; j++) c[j] = j < k ? sum[j] : 0.0;
        s.tslot = k;
    }
    s.tnorm2 = sum[kMaxSpace];
    st[i] = s;
}

__global__ void check_kernel(const DavProb *__restrict__ probs, DavState *__restrict__ st,
                             const double *__restrict__ part, double *__restrict__ coef, const double *__restrict__ ys,
                             double *__restrict__ gs, int max_space, int restart_at, int keep_max, int mixed,
                             int max_iter, double e_tol, double r_tol, int *__restrict__ nactive, int nprob_) {
    for (int w = blockIdx.x; w < nprob_; w += gridDim.x) {
        check_kernel_body(probs, st, part, coef, ys, gs, max_space, restart_at, keep_max, mixed, max_iter, e_tol, r_tol, nactive, w);
        __syncthreads();   // shared memory is reused by the next body
    }
}

// Restart: B_r <- sum_j Y_r[j] B_j and S_r <- sum_j Y_r[j] S_j for the kept
// Ritz vectors r < nform; a thick restart (tslot >= 0) also moves the
// correction from the scratch slot to slot nform, a phase switch of the mixed
// mode (tslot < 0) drops it and rebuilds the S_r exactly.  Every old slot of
// an element is read before any is written.
__device__ __forceinline__ void restart_kernel_body(const DavProb *__restrict__ probs,
                                                      const DavState *__restrict__ st,
                                                      const WorkItem *__restrict__ items, const double *__restrict__ ys,
                                                      int max_space, int mixed, int w_) {
    const WorkItem it = items[w_];
    const DavState s = st[it.prob];
    if (!s.active || !s.restart) return;
    const DavProb &p = probs[it.prob];
    const bool thick = s.tslot >= 0;   // a phase switch drops the correction
    const int keep = s.nform;
    const double *yr = ys + (long long)it.prob * kYStride;
    long long end = min(it.start + (long long)kVecChunk, p.ndet);
    const double *T = p.B + (long long)max_space * p.ndet;
    const int kk = s.kold;   // only the slots of the old subspace are read
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
        double bv[kMaxSpace], sv[kMaxSpace];
#pragma unroll
        for (int j = 0; j < kMaxSpace; j++) {
            bv[j] = j < kk ? p.B[(long long)j * p.ndet + I] : 0.0;
            sv[j] = j < kk ? p.S[(long long)j * p.ndet + I] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < kKeep; r++) {
            if (r < keep) {
                double x = 0.0, sx = 0.0;
#pragma unroll
                for (int j = 0; j < kMaxSpace; j++) {
                    x += yr[r * kNP + j] * bv[j];
                    sx += yr[r * kNP + j] * sv[j];
                }
                p.B[(long long)r * p.ndet + I] = x;
                p.S[(long long)r * p.ndet + I] = sx;
            }
        }
        if (thick) p.B[(long long)keep * p.ndet + I] = T[I];
    }
}

__global__ void __launch_bounds__(256) restart_kernel(const DavProb *__restrict__ probs,
                                                      const DavState *__restrict__ st,
                                                      const WorkItem *__restrict__ items, const double *__restrict__ ys,
                                                      int max_space, int mixed, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) restart_kernel_body(probs, st, items, ys, max_space, mixed, w);
}

// t -= sum_{j<k} coef_j b_j ; then dots <b_j|t> and |t|^2 for the next pass.
__device__ __forceinline__ void ortho_kernel_body(const DavProb *__restrict__ probs, const DavState *__restrict__ st,
                                                    const WorkItem *__restrict__ items,
                                                    const double *__restrict__ coef, int max_space,
                                                    double *__restrict__ part, int pass, int w_) {
    const WorkItem it = items[w_];
    const DavState s = st[it.prob];
    if (!s.active || s.tslot < 0) return;
    if (pass == 1 && s.skip2) return;
    const DavProb &p = probs[it.prob];
    const int k = s.k;
    double c[kMaxSpace];
#pragma unroll
    for (int j = 0; j < kMaxSpace; j++) c[j] = coef[(long long)it.prob * kNP + j];
    double *T = p.B + (long long)s.tslot * p.ndet;
    if (!s.restart && s.tslot == k) T = p.B + (long long)max_space * p.ndet;
    double acc[kMaxSpace + 1];
#pragma unroll
    for (int j = 0; j <= kMaxSpace; j++) acc[j] = 0.0;
    long long end = min(it.start + (long long)kVecChunk, p.ndet);
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
        double t = T[I];
        double bv[kMaxSpace];
#pragma unroll
        for (int j = 0; j < kMaxSpace; j++)
            if (j < k) {
                bv[j] = p.B[(long long)j * p.ndet + I];
                t -= c[j] * bv[j];
            }
        T[I] = t;
#pragma unroll
        for (int j = 0; j < kMaxSpace; j++)
            if (j < k) acc[j] += bv[j] * t;
        acc[kMaxSpace] += t * t;
    }
    __shared__ double red[8][kMaxSpace + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j <= kMaxSpace; j++) {
        if (j < k || j == kMaxSpace) {
            double v = warp_sum(acc[j]);
            if (lane == 0) red[warp][j] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x <= kMaxSpace && (threadIdx.x < k || threadIdx.x == kMaxSpace)) {
        double v = 0.0;
        for (int w = 0; w < 8; w++) v += red[w][threadIdx.x];
        part[(long long)w_ * kNP + threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(256) ortho_kernel(const DavProb *__restrict__ probs, const DavState *__restrict__ st,
                                                    const WorkItem *__restrict__ items,
                                                    const double *__restrict__ coef, int max_space,
                                                    double *__restrict__ part, int pass, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) {
        ortho_kernel_body(probs, st, items, coef, max_space, part, pass, w);
        __syncthreads();   // shared memory is reused by the next body
    }
}

// After Gram-Schmidt pass `pass`: the coefficients of the next pass and |t|^2.
// The second pass runs only when the first one removed more than half of
// |t|^2 (the DGKS criterion with eta = 1/sqrt 2: a first pass that kept
// |t| >= |t_before| / sqrt 2 leaves t orthogonal to working precision).
__device__ __forceinline__ void reduce_coef_kernel_body(const DavProb *__restrict__ probs, DavState *__restrict__ st,
                                   const double *__restrict__ part, double *__restrict__ coef, int pass, int w_) {
    const int i = w_;
    DavState s = st[i];
    if (!s.active || s.tslot < 0) return;
    if (pass == 1 && s.skip2) return;
    const DavProb p = probs[i];
    const int k = s.k;
    if (threadIdx.x < k || threadIdx.x == kMaxSpace) {
        double v = 0.0;
        for (int w = 0; w < p.nitem; w++) v += part[(long long)(p.item0 + w) * kNP + threadIdx.x];
        if (threadIdx.x == kMaxSpace) {
            if (pass == 0) st[i].skip2 = v >= 0.5 * s.tnorm2 ? 1 : 0;
            st[i].tnorm2 = v;
        } else {
            coef[(long long)i * kNP + threadIdx.x] = v;
        }
    }
    if (threadIdx.x > k && threadIdx.x < kMaxSpace) coef[(long long)i * kNP + threadIdx.x] = 0.0;
}

__global__ void reduce_coef_kernel(const DavProb *__restrict__ probs, DavState *__restrict__ st,
                                   const double *__restrict__ part, double *__restrict__ coef, int pass, int nprob_) {
    for (int w = blockIdx.x; w < nprob_; w += gridDim.x) reduce_coef_kernel_body(probs, st, part, coef, pass, w);
}

// b_k = t / |t|, symmetrised over (I_a, I_b) <-> (I_b, I_a) in a symmetric
// block; the new slot becomes the next sigma target.  One thread per pair
// (I, I^T) with I_a >= I_b (per element in an off-diagonal block).
__device__ __forceinline__ void normalize_kernel_body(const DavProb *__restrict__ probs,
                                                        const DavState *__restrict__ st,
                                                        const WorkItem *__restrict__ items, int max_space, int w_) {
    const WorkItem it = items[w_];
    const DavState s = st[it.prob];
    if (!s.active || s.tslot < 0) return;
    const DavProb &p = probs[it.prob];
    const double inv = s.tnorm2 > 0.0 ? 1.0 / sqrt(s.tnorm2) : 0.0;
    double *T = p.B + (long long)s.tslot * p.ndet;
    double *dst = T;
    if (!s.restart && s.tslot == s.k) {
        T = p.B + (long long)max_space * p.ndet;
        dst = p.B + (long long)s.k * p.ndet;
    }
    long long end = min(it.start + (long long)kVecChunk, p.ndet);
    if (!p.sym) {
        for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) dst[I] = T[I] * inv;
        return;
    }
    const int n = p.nb;
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
        int a = (int)(I / n), b = (int)(I % n);
        if (a < b) continue;
        long long It = (long long)b * n + a;
        double v = 0.5 * (T[I] + T[It]) * inv;
        dst[I] = v;
        dst[It] = v;
    }
}

__global__ void __launch_bounds__(256) normalize_kernel(const DavProb *__restrict__ probs,
                                                        const DavState *__restrict__ st,
                                                        const WorkItem *__restrict__ items, int max_space, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) normalize_kernel_body(probs, st, items, max_space, w);
}

__global__ void advance_kernel(const DavProb *__restrict__ probs, DavState *__restrict__ st, int nprob,
                               double r_tol, int mixed) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nprob) return;
    DavState s = st[i];
    if (!s.active) return;
    if (s.tslot >= 0 && s.tnorm2 < 1e-28 && mixed && !s.exact_all) {
        // phase 1 with an exhausted subspace: keep it, rebuild sigma of the newest
        // vector and switch to the exact phase at the next check
        s.force = 1;
        s.restart = 0;
        st[i] = s;
        return;
    }
    if (s.tslot >= 0 && s.tnorm2 < 1e-28 && s.tcur != 0) {
        // the correction of a higher (competitive) root vanished: that root is
        // resolved; no vector is added, and after a restart this iteration the
        // last kept vector becomes the newest (its sigma is rebuilt, unchanged)
        s.rn[s.tcur] = 0.0;
        if (s.restart) s.newest = s.k - 1;
        s.tslot = -1;
        s.restart = 0;
        st[i] = s;
        return;
    }
    if (s.tslot >= 0 && s.tnorm2 < 1e-28) {
        // the correction of the lowest root vanished after orthogonalisation:
        // the subspace is exhausted; the lowest root's own residual decides
        s.active = 0;
        s.status = s.rn[0] < r_tol ? IFCI_OK : IFCI_ERR_NOT_CONVERGED;
        s.energy = s.theta + probs[i].e_core;
        st[i] = s;
        return;
    }
    if (s.tslot >= 0) {
        s.newest = s.tslot;
        s.k = s.tslot + 1;
    } else if (s.rebuild_to > 0 && !s.restart) {
        s.newest += 1;   // next kept Ritz vector whose exact sigma is rebuilt
        s.k = s.newest + 1;
    }
    s.restart = 0;
    st[i] = s;
}

// c_out = sum_j y_j B_j for every finished problem that asked for it
__device__ __forceinline__ void ritz_out_kernel_body(const DavProb *__restrict__ probs,
                                                       const DavState *__restrict__ st,
                                                       const WorkItem *__restrict__ items,
                                                       const double *__restrict__ ys, int w_) {
    const WorkItem it = items[w_];
    const DavProb &p = probs[it.prob];
    if (!p.c_out) return;
    const DavState s = st[it.prob];
    const int k = s.newest + 1;
    double y[kMaxSpace];
#pragma unroll
    for (int j = 0; j < kMaxSpace; j++) y[j] = ys[(long long)it.prob * kYStride + j];
    long long end = min(it.start + (long long)kVecChunk, p.ndet);
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
        double x = 0.0;
#pragma unroll
        for (int j = 0; j < kMaxSpace; j++)
            if (j < k) x += y[j] * p.B[(long long)j * p.ndet + I];
        p.c_out[I] = x;
    }
}

__global__ void __launch_bounds__(256) ritz_out_kernel(const DavProb *__restrict__ probs,
                                                       const DavState *__restrict__ st,
                                                       const WorkItem *__restrict__ items,
                                                       const double *__restrict__ ys, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) ritz_out_kernel_body(probs, st, items, ys, w);
}

// Selected-CI problems: sigma of the newest slot zeroed outside the selection
// (the iteration then stays in the span of the selected determinants).
__device__ __forceinline__ void mask_sigma_kernel_body(const DavProb *__restrict__ probs,
                                                         const DavState *__restrict__ st,
                                                         const WorkItem *__restrict__ items, int w_) {
    const WorkItem it = items[w_];
    const DavProb &p = probs[it.prob];
    if (!p.mask) return;
    const DavState s = st[it.prob];
    if (!s.active) return;
    double *S = p.S + (long long)s.newest * p.ndet;
    const long long end = min(it.start + (long long)kVecChunk, p.ndet);
    for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x)
        if (!p.mask[I]) S[I] = 0.0;
}

__global__ void __launch_bounds__(256) mask_sigma_kernel(const DavProb *__restrict__ probs,
                                                         const DavState *__restrict__ st,
                                                         const WorkItem *__restrict__ items, int nitem_) {
    for (int w = blockIdx.x; w < nitem_; w += gridDim.x) mask_sigma_kernel_body(probs, st, items, w);
}

// ------------------------------------------------------------------ driver

int dav_init(ifci_handle_t h, DavBatch &b, const HdiagDesc *d_hd, cudaStream_t s) {
    const int nvi = (int)b.vitems.size();
    {
        ProfScope ps(h, s, PK_SETUP);
        init_kernel<<<stride_grid(h->device, b.nprob, 8), 256, 0, s>>>(b.d_probs, b.d_state, b.max_space, b.nprob);
        IFCI_LAUNCH_CHECK(h);
        init_vec_kernel<<<stride_grid(h->device, nvi, 8), 256, 0, s>>>(b.d_probs, b.d_vitems, b.max_space, nvi);
        IFCI_LAUNCH_CHECK(h);
    }
    IFCI_TRY(launch_pspace_start(h, b, d_hd, s));   // its solve is profiled as PK_PSPACE
    ProfScope ps(h, s, PK_SETUP);
    init_scale_kernel<<<stride_grid(h->device, nvi, 8), 256, 0, s>>>(b.d_probs, b.d_state, b.d_vitems, b.d_part, nvi);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

// One Davidson iteration over the whole batch (no host synchronisation).
static int dav_step(ifci_handle_t h, DavBatch &b, SigmaPlan &hi_plan, SigmaPlan *lo_plan, int *d_hi, int *d_lo,
                    void *D, void *G, cudaStream_t s) {
    const int nitem = (int)b.vitems.size();
    // grid-stride kernels: resident grids over the vector items and the problems
    const int gi = stride_grid(h->device, nitem, 8), gp = stride_grid(h->device, b.nprob, 32);
    const bool mixed = lo_plan != nullptr;
    const int restart_at = b.max_space;
    select_kernel<<<(b.nprob + 127) / 128, 128, 0, s>>>(b.d_state, b.nprob, mixed ? 1 : 0, d_hi, d_lo);
    IFCI_LAUNCH_CHECK(h);
    IFCI_TRY(launch_unit_flags(h, b, d_hi, d_lo, s));
    // blocks of a sectored space: their newest vectors form one whole-space
    // input, whose sigma each block takes its part of
    auto sector_move = [&](bool in, const int *flag) -> int {
        if (!b.any_sector) return IFCI_OK;
        ProfScope ps(h, s, PK_OTHER);
        return in ? launch_sector_gather(h, b, flag, s) : launch_sector_scatter(h, b, flag, s);
    };
    IFCI_TRY(sector_move(true, d_hi));
    IFCI_TRY(run_sigma(h, hi_plan, b.hi_precision, D, G, s));
    IFCI_TRY(sector_move(false, d_hi));
    if (mixed) {
        IFCI_TRY(sector_move(true, d_lo));
        IFCI_TRY(run_sigma(h, *lo_plan, b.precision, D, G, s));
        IFCI_TRY(sector_move(false, d_lo));
    }
    if (b.any_mask) {
        ProfScope ps(h, s, PK_OTHER);
        mask_sigma_kernel<<<gi, 256, 0, s>>>(b.d_probs, b.d_state, b.d_vitems, nitem);
        IFCI_LAUNCH_CHECK(h);
    }
    ProfScope vec_scope(h, s, PK_VECTOR);
    dots_kernel<<<gi, 256, 0, s>>>(b.d_probs, b.d_state, b.d_vitems, b.d_part, nitem);
    IFCI_LAUNCH_CHECK(h);
    solve_kernel<<<stride_grid(h->device, (b.nprob + kSolveWarps - 1) / kSolveWarps, 8), 32 * kSolveWarps, 0, s>>>(
        b.d_probs, b.d_state, b.d_part, b.d_gs, b.d_y, b.nprob);
    IFCI_LAUNCH_CHECK(h);
    residual_kernel<<<gi, 256, 0, s>>>(b.d_probs, b.d_state, b.d_vitems, b.d_y, b.max_space, b.d_part, nitem);
    IFCI_LAUNCH_CHECK(h);
    IFCI_CUDA_TRY(h, cudaMemsetAsync(b.d_nactive, 0, sizeof(int), s));
    // check_kernel records the subspace size before a restart (kold) for restart_kernel
    check_kernel<<<gp, 32, 0, s>>>(b.d_probs, b.d_state, b.d_part, b.d_coef, b.d_y, b.d_gs, b.max_space,
                                        restart_at, b.keep, mixed ? 1 : 0, b.max_iter, b.e_tol, b.r_tol,
                                        b.d_nactive, b.nprob);
    IFCI_LAUNCH_CHECK(h);
    restart_kernel<<<gi, 256, 0, s>>>(b.d_probs, b.d_state, b.d_vitems, b.d_y, b.max_space, mixed ? 1 : 0, nitem);
    IFCI_LAUNCH_CHECK(h);
    for (int pass = 0; pass < 2; pass++) {
        ortho_kernel<<<gi, 256, 0, s>>>(b.d_probs, b.d_state, b.d_vitems, b.d_coef, b.max_space, b.d_part, pass, nitem);
        IFCI_LAUNCH_CHECK(h);
        reduce_coef_kernel<<<gp, 32, 0, s>>>(b.d_probs, b.d_state, b.d_part, b.d_coef, pass, b.nprob);
        IFCI_LAUNCH_CHECK(h);
    }
    normalize_kernel<<<gi, 256, 0, s>>>(b.d_probs, b.d_state, b.d_vitems, b.max_space, nitem);
    IFCI_LAUNCH_CHECK(h);
    advance_kernel<<<(b.nprob + 127) / 128, 128, 0, s>>>(b.d_probs, b.d_state, b.nprob, b.r_tol, mixed ? 1 : 0);
    IFCI_LAUNCH_CHECK(h);
    if (h->prof) prof_end(h, s);
    return IFCI_OK;
}

// Iterates until every problem has stopped.  Eager mode launches each
// iteration and reads the active count after it; graph mode (b.graph_iters > 0,
// profiling off) runs the first iteration eagerly (it also configures the
// kernels), then captures b.graph_iters iterations into one CUDA graph on a
// stream of its own (ordered after `s` by an event) and replays it, reading
// the active count after each replay.  Problems that stop inside a block make
// the remaining iterations of the block no-ops, so both modes give the same
// results.
int dav_iterate(ifci_handle_t h, DavBatch &b, SigmaPlan &hi_plan, SigmaPlan *lo_plan, int *d_hi, int *d_lo,
                void *D, void *G, int *h_nactive, cudaStream_t s) {
    const int nitem = (int)b.vitems.size();
    const bool graph = b.graph_iters > 0 && !h->prof;
    cudaStream_t ws = s;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long launches_per_graph = 0;
    int st = IFCI_OK;
    if (graph) {
        IFCI_CUDA_TRY(h, cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
        IFCI_CUDA_TRY(h, cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
        IFCI_CUDA_TRY(h, cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
        IFCI_CUDA_TRY(h, cudaEventRecord(ev_in, s));
        IFCI_CUDA_TRY(h, cudaStreamWaitEvent(ws, ev_in, 0));
    }
    for (int it = 0; it < b.max_iter + 2 && st == IFCI_OK;) {
        if (graph && it > 0) {
            if (!exec) {
                const long long l0 = h->launches;
                if (cudaStreamBeginCapture(ws, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                    st = set_error(h, IFCI_ERR_CUDA, "davidson: stream capture could not begin");
                    break;
                }
                for (int g = 0; g < b.graph_iters && st == IFCI_OK; g++)
                    st = dav_step(h, b, hi_plan, lo_plan, d_hi, d_lo, D, G, ws);
                const cudaError_t ec = cudaStreamEndCapture(ws, &gr);
                if (st != IFCI_OK) break;
                if (ec != cudaSuccess || cudaGraphInstantiate(&exec, gr, 0) != cudaSuccess) {
                    cudaGetLastError();
                    st = set_error(h, IFCI_ERR_CUDA, "davidson: graph capture failed");
                    break;
                }
                launches_per_graph = h->launches - l0;
                h->launches = l0;   // counted when replayed
            }
            if (cudaGraphLaunch(exec, ws) != cudaSuccess) {
                st = set_error(h, IFCI_ERR_CUDA, "davidson: graph launch failed");
                break;
            }
            h->launches += launches_per_graph;
            it += b.graph_iters;
        } else {
            st = dav_step(h, b, hi_plan, lo_plan, d_hi, d_lo, D, G, ws);
            if (st != IFCI_OK) break;
            it += 1;
        }
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(h_nactive, b.d_nactive, sizeof(int), cudaMemcpyDeviceToHost, ws));
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(h_nactive + 1, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, ws));
        IFCI_CUDA_TRY(h, cudaStreamSynchronize(ws));
        if (h_nactive[1]) {
            cudaMemsetAsync(h->d_err, 0, sizeof(int), ws);
            st = set_error(h, IFCI_ERR_TIMEOUT, "davidson: a bounded device wait ran out");
            break;
        }
        if (*h_nactive == 0) break;
    }
    if (st == IFCI_OK) {
        ritz_out_kernel<<<stride_grid(h->device, nitem, 8), 256, 0, ws>>>(b.d_probs, b.d_state, b.d_vitems, b.d_y, nitem);
        IFCI_LAUNCH_CHECK(h);
    }
    if (graph) {
        cudaEventRecord(ev_out, ws);
        cudaStreamWaitEvent(s, ev_out, 0);
        cudaStreamSynchronize(ws);
        if (exec) cudaGraphExecDestroy(exec);
        if (gr) cudaGraphDestroy(gr);
        cudaEventDestroy(ev_in);
        cudaEventDestroy(ev_out);
        cudaStreamDestroy(ws);
    }
    return st;
}

}  // namespace ifci
