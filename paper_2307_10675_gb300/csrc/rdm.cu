// Gradient of the iFCI energy with respect to the integrals (reverse mode of
// Eqs. 1-5): Hellmann–Feynman on every E_Y, summed with the expansion weights
//   E_iFCI = E_0 + sum_{|X|<=n} eps_X = (1 - sum_Y w_Y) E_0 + sum_Y w_Y E_Y,
//   w_Y = (-1)^(n-|Y|) C(N-|Y|-1, n-|Y|).
//
// Per body set Y with converged vector c (spin-flip-even, normalised):
//   D+[A][K] = <K|E+_A|c>                     (the gather of the sigma build)
//   M[A][B]  = sum_K D+[A][K] D+[B][K] = <c|E+_A E+_B|c>    (SYRK, split over K)
//   gamma+_A = sum_K c_K D+[A][K]             (an extra row of D+ holding c)
// so the packed active 2-RDM is Gamma+_AB = M[A][B] - sum_{pq in A, rs in B}
// delta_qr gamma_ps.  The frozen core enters through the chain rule of
// E_core and h1 (Coulomb and exchange with the core orbitals).  Contributions
// of all body sets are summed with FP64 atomics into dh and dV; dV is
// symmetrised at the end (the packed entries V[A][B] and V[B][A] are one
// parameter of the symmetric H).
#include <algorithm>
#include <cmath>
#include <map>

#include "dav_driver.cuh"
#include "hamiltonian.cuh"
#include "system.cuh"

namespace ifci {

namespace {

constexpr int kSyrkT = 64;          // SYRK output tile
constexpr int kSyrkChunk = 16384;   // determinants per split-K chunk

struct RdmProb {
    int n, np, nstr, nexc, nA, nC;
    long long ndet;
    const int32_t *exc;
    const double *c;        // converged vector
    const int *orbs;        // [active nA ..., core nC ...] global orbital indices
    double w;               // expansion weight x grad_out
    long long doff;         // element offset of this problem's (np+1) x ndet block of D+
    int chunk0, nchunk;     // split-K chunks of this problem in the partial buffer
    double *M;              // (np+1)^2 reduced moments
};

struct SyrkJob {
    int prob, chunk, ta, tb;
};

// D+[A][K] for A < np (merge of the sorted alpha/beta lists) and D+[np][K] = c_K
__global__ void __launch_bounds__(256) rdm_gather_kernel(const RdmProb *__restrict__ probs,
                                                         const WorkItem *__restrict__ items, double *__restrict__ D) {
    const WorkItem it = items[blockIdx.x];
    const RdmProb &p = probs[it.prob];
    const long long K = it.start + threadIdx.x;
    if (K >= p.ndet) return;
    const int nstr = p.nstr, nexc = p.nexc, np = p.np;
    const long long ndet = p.ndet;
    const int ka = (int)(K / nstr), kb = (int)(K % nstr);
    const double *c = p.c;
    const int32_t *ea = p.exc + (size_t)ka * nexc, *eb = p.exc + (size_t)kb * nexc;
    int ia = 0, ib = 0;
    int32_t xa = ea[0], xb = eb[0];
    int pa = exc_pair(xa), pb = exc_pair(xb);
    double *out = D + p.doff + K;
    for (int A = 0; A < np; A++) {
        double v = 0.0;
        if (pa == A) {
            v += exc_sign(xa) * c[(long long)exc_J(xa) * nstr + kb];
            if (++ia < nexc) { xa = ea[ia]; pa = exc_pair(xa); } else pa = -1;
        }
        if (pb == A) {
            v += exc_sign(xb) * c[(long long)ka * nstr + exc_J(xb)];
            if (++ib < nexc) { xb = eb[ib]; pb = exc_pair(xb); } else pb = -1;
        }
        out[(long long)A * ndet] = v;
    }
    out[(long long)np * ndet] = c[K];
}

// partial[job] = sum_{K in chunk} D+[ta*64 + i][K] D+[tb*64 + j][K]   (64 x 64 tile)
__global__ void __launch_bounds__(256) rdm_syrk_kernel(const RdmProb *__restrict__ probs,
                                                       const SyrkJob *__restrict__ jobs,
                                                       const double *__restrict__ D, double *__restrict__ part) {
    const SyrkJob jb = jobs[blockIdx.x];
    const RdmProb &p = probs[jb.prob];
    const int rows = p.np + 1;
    const long long ndet = p.ndet;
    const long long k0 = (long long)(jb.chunk - p.chunk0) * kSyrkChunk;
    const long long k1 = min(ndet, k0 + kSyrkChunk);
    const double *Dp = D + p.doff;
    __shared__ double As[16][kSyrkT], Bs[16][kSyrkT];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
    for (long long kk = k0; kk < k1; kk += 16) {
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int e = threadIdx.x + 256 * r;
            const int kq = e % 16, m = e / 16;
            const long long K = kk + kq;
            const int A = jb.ta * kSyrkT + m, B = jb.tb * kSyrkT + m;
            As[kq][m] = (A < rows && K < k1) ? Dp[(long long)A * ndet + K] : 0.0;
            Bs[kq][m] = (B < rows && K < k1) ? Dp[(long long)B * ndet + K] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kq = 0; kq < 16; kq++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kq][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kq][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    double *out = part + (size_t)blockIdx.x * kSyrkT * kSyrkT;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) out[(ty * 4 + i) * kSyrkT + tx + 16 * j] = acc[i][j];
}

// M = sum over the problem's chunks of the partial tiles (fixed order), symmetric fill
__global__ void rdm_reduce_kernel(const RdmProb *__restrict__ probs, const int *__restrict__ job0,
                                  const double *__restrict__ part) {
    const int pi = blockIdx.x;
    const RdmProb &p = probs[pi];
    const int rows = p.np + 1, T = (rows + kSyrkT - 1) / kSyrkT;
    const int ntt = T * (T + 1) / 2;   // tiles ta <= tb per chunk
    for (int e = threadIdx.x; e < rows * rows; e += blockDim.x) {
        const int A = e / rows, B = e % rows;
        const int a = min(A, B), b = max(A, B);
        const int ta = a / kSyrkT, tb = b / kSyrkT;
        const int tix = ta * T - ta * (ta - 1) / 2 + (tb - ta);   // index of (ta, tb) among ta <= tb
        // the (ta, tb) tile holds sum_K D+[64 ta + i][K] D+[64 tb + j][K]
        const int i = (A <= B ? A : B) - ta * kSyrkT, j = (A <= B ? B : A) - tb * kSyrkT;
        double s = 0.0;
        for (int ch = 0; ch < p.nchunk; ch++)
            s += part[((size_t)job0[pi] + (size_t)ch * ntt + tix) * kSyrkT * kSyrkT + (size_t)i * kSyrkT + j];
        p.M[e] = s;
    }
}

__device__ __forceinline__ int pair_local(int P, int Q) { return P >= Q ? P * (P + 1) / 2 + Q : Q * (Q + 1) / 2 + P; }

// Weighted contributions of one body set to dh (norb^2) and dV (npair_g^2).
__global__ void rdm_accum_kernel(const RdmProb *__restrict__ probs, int norb, double *__restrict__ dh,
                                 double *__restrict__ dV) {
    const RdmProb &p = probs[blockIdx.x];
    const int n = p.nA, nC = p.nC, np = p.np, rows = np + 1;
    const double w = p.w;
    if (w == 0.0) return;
    const long long npg = (long long)norb * (norb + 1) / 2;
    const int *act = p.orbs, *core = p.orbs + n;
    const double *M = p.M;
    auto gam = [&](int a, int b) -> double {   // active 1-RDM gamma_ab
        const double g = M[(long long)pair_local(a, b) * rows + np];
        return a == b ? g : 0.5 * g;
    };
    auto Vg = [&](int P, int Q, int R, int S) -> double * {
        return dV + (long long)pair_of(P, Q) * npg + pair_of(R, S);
    };
    // (i) one-electron: dh = gamma (active), 2 (core)
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int a = t / n, b = t % n;
        atomicAdd(dh + (long long)act[a] * norb + act[b], w * gam(a, b));
    }
    for (int k = threadIdx.x; k < nC; k += blockDim.x) atomicAdd(dh + (long long)core[k] * norb + core[k], 2.0 * w);
    // (ii) active 2-RDM, packed: 1/2 (M[A][B] - sum_{pq in A, rs in B} d_qr gamma_ps)
    for (int t = threadIdx.x; t < np * np; t += blockDim.x) {
        const int A = t / np, B = t % np;
        int P = 0;
        while ((P + 1) * (P + 2) / 2 <= A) P++;
        const int Q = A - P * (P + 1) / 2;
        int R = 0;
        while ((R + 1) * (R + 2) / 2 <= B) R++;
        const int S = B - R * (R + 1) / 2;
        double corr = 0.0;
        const int pq[2][2] = {{P, Q}, {Q, P}}, rs[2][2] = {{R, S}, {S, R}};
        const int na = P == Q ? 1 : 2, nb = R == S ? 1 : 2;
        for (int u = 0; u < na; u++)
            for (int v = 0; v < nb; v++)
                if (pq[u][1] == rs[v][0]) corr += gam(pq[u][0], rs[v][1]);
        const double g2 = M[(long long)A * rows + B] - corr;
        atomicAdd(Vg(act[P], act[Q], act[R], act[S]), 0.5 * w * g2);
    }
    // (iii) h1 = h + sum_c [2 (pq|cc) - (pc|cq)]: Coulomb and exchange with the core
    for (int t = threadIdx.x; t < np * nC; t += blockDim.x) {
        const int A = t / nC, k = t % nC;
        int P = 0;
        while ((P + 1) * (P + 2) / 2 <= A) P++;
        const int Q = A - P * (P + 1) / 2;
        const double gplus = M[(long long)A * rows + np];
        atomicAdd(Vg(act[P], act[Q], core[k], core[k]), 2.0 * w * gplus);
    }
    for (int t = threadIdx.x; t < n * n * nC; t += blockDim.x) {
        const int a = t / (n * nC), b = (t / nC) % n, k = t % nC;
        atomicAdd(Vg(act[a], core[k], core[k], act[b]), -w * gam(a, b));
    }
    // (iv) E_core = sum_c 2 h_cc + sum_{c,d} [2 (cc|dd) - (cd|dc)]
    for (int t = threadIdx.x; t < nC * nC; t += blockDim.x) {
        const int k = t / nC, l = t % nC;
        atomicAdd(Vg(core[k], core[k], core[l], core[l]), 2.0 * w);
        atomicAdd(Vg(core[k], core[l], core[l], core[k]), -w);
    }
}

// E_0 terms with weight w0 over the bonding orbitals.
__global__ void rdm_reference_kernel(const int *__restrict__ bond, int nb, double w0, int norb, double *__restrict__ dh,
                                     double *__restrict__ dV) {
    const long long npg = (long long)norb * (norb + 1) / 2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nb * nb; t += gridDim.x * blockDim.x) {
        const int k = t / nb, l = t % nb;
        const int c = bond[k], d = bond[l];
        if (k == l) atomicAdd(dh + (long long)c * norb + c, 2.0 * w0);
        atomicAdd(dV + (long long)pair_of(c, c) * npg + pair_of(d, d), 2.0 * w0);
        atomicAdd(dV + (long long)pair_of(c, d) * npg + pair_of(d, c), -w0);
    }
}

// dV <- (dV + dV^T) / 2
__global__ void rdm_symmetrise_kernel(long long npg, double *__restrict__ dV) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < npg * npg;
         t += (long long)gridDim.x * blockDim.x) {
        const long long A = t / npg, B = t % npg;
        if (A < B) {
            const double s = 0.5 * (dV[A * npg + B] + dV[B * npg + A]);
            dV[A * npg + B] = s;
            dV[B * npg + A] = s;
        }
    }
}

long long expansion_weight(int nbody, int k, int max_order) {
    // (-1)^(n-|Y|) C(N-|Y|-1, n-|Y|); a set of all N bodies has weight 1
    if (k == nbody) return 1;
    long long c = binom(nbody - k - 1, max_order - k);
    return ((max_order - k) & 1) ? -c : c;
}

}  // namespace

}  // namespace ifci

extern "C" int ifci_rdm_backward(ifci_handle_t h, const ifci_system_t *sys, int max_order,
                                 const ifci_davidson_opts_t *opts, double grad_out, double *dh, double *deri,
                                 int recompute_vectors, ifci_stream_t stream) {
    using namespace ifci;
    if (!h) return IFCI_ERR_INVALID_ARG;
    IFCI_TRY(validate_system(h, sys, max_order));
    if (!dh || !deri) return set_error(h, IFCI_ERR_INVALID_ARG, "rdm_backward: null output");
    if (opts && opts->hbci_max_rounds > 0)
        return set_error(h, IFCI_ERR_UNSUPPORTED, "rdm_backward: no gradient of the HBCI energy (its PT2 part)");
    IFCI_CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = as_cuda(stream);
    const int norb = sys->norb;
    const long long npg = (long long)norb * (norb + 1) / 2;
    bool have = h->kept.valid && h->kept.nbody == sys->nbody && h->kept.max_order == max_order &&
                h->kept.norb == norb &&
                std::equal(h->kept.body_offset.begin(), h->kept.body_offset.end(), sys->body_offset);
    if (!recompute_vectors && !have)
        return set_error(h, IFCI_ERR_INVALID_ARG, "rdm_backward: no kept vectors for this system (run "
                                                   "ifci_increments first or ask for recomputation)");
    if (recompute_vectors || !have) {
        long long ns = 0;
        ifci_num_subsets(sys->nbody, max_order, &ns);
        std::vector<double> eps(ns);
        double e0 = 0, et = 0;
        ifci_davidson_opts_t o;
        ifci_davidson_default_opts(&o);
        if (opts) o = *opts;
        if (o.refine < 0) o.refine = 1;   // the vectors must be kept
        IFCI_TRY(ifci_increments(h, sys, max_order, &o, &e0, nullptr, eps.data(), &et, nullptr, nullptr, stream));
    }
    SubsetPlan P;
    plan_subsets(sys, max_order, P);
    // expansion weights: closed form, or (screened expansion) the derivative of
    // the recursion of Eqs. 2-5 at the forward call's inclusion pattern; the
    // screened sets (no vector, weight 0) leave the plan
    std::vector<double> wts(P.subsets.size());
    std::vector<long long> kvec_off;
    {
        const bool scr = h->kept.screened && h->kept.included.size() == P.subsets.size();
        if (scr) wts = screened_weights(P, h->kept.included);
        else
            for (size_t x = 0; x < P.subsets.size(); x++)
                wts[x] = (double)expansion_weight(sys->nbody, (int)P.subsets[x].size(), max_order);
        SubsetPlan Q;
        Q.orbs = P.orbs;
        std::vector<double> w2;
        for (size_t x = 0; x < P.subsets.size(); x++) {
            if (scr && !h->kept.included[x]) continue;
            Q.subsets.push_back(P.subsets[x]);
            Q.nA.push_back(P.nA[x]);
            Q.nC.push_back(P.nC[x]);
            Q.orb_off.push_back(P.orb_off[x]);
            kvec_off.push_back(h->kept.vec_off[x]);
            w2.push_back(wts[x]);
        }
        P = std::move(Q);
        wts = std::move(w2);
    }
    const int ns = (int)P.subsets.size();

    // problems, D+ waves and split-K jobs
    std::vector<RdmProb> probs(ns);
    double wsum = 0.0;
    long long dtotal = 0, maxd = 0;
    for (int x = 0; x < ns; x++) {
        RdmProb &r = probs[x];
        r.n = P.nA[x];
        r.nC = P.nC[x];
        r.nA = r.n;
        r.np = r.n * (r.n + 1) / 2;
        const int m = (int)P.subsets[x].size();
        r.nstr = (int)binom(r.n, m);
        r.nexc = m * (r.n - m + 1);
        r.ndet = (long long)r.nstr * r.nstr;
        r.c = h->kept.vec + kvec_off[x];
        const double wy = wts[x];
        r.w = wy * grad_out;
        wsum += wy;
        const long long need = (long long)(r.np + 1) * r.ndet;
        maxd = std::max(maxd, need);
        dtotal += need;
    }
    const long long budget = std::max(maxd, std::min(dtotal, 1ll << 28));
    // string tables per class
    size_t need = ws_round(ns * sizeof(RdmProb)) + ws_round(P.orbs.size() * 4) + ws_round(sys->nbody * 4) +
                  ws_round((size_t)budget * 8);
    std::map<std::pair<int, int>, int> cls;
    size_t tab_bytes = 0;
    long long mtot = 0;
    for (int x = 0; x < ns; x++) {
        auto key = std::make_pair(probs[x].n, (int)P.subsets[x].size());
        if (!cls.count(key)) {
            cls[key] = 1;
            tab_bytes += ws_round((size_t)probs[x].nstr * 8) + ws_round((size_t)probs[x].nstr * probs[x].nexc * 4);
        }
        mtot += (long long)(probs[x].np + 1) * (probs[x].np + 1);
    }
    need += tab_bytes + ws_round((size_t)mtot * 8);
    // per-wave work lists and partials are sized for the largest wave below
    std::vector<std::pair<int, int>> waves;
    {
        int first = 0;
        long long acc = 0;
        for (int x = 0; x < ns; x++) {
            const long long d = (long long)(probs[x].np + 1) * probs[x].ndet;
            if (acc + d > budget && x > first) {
                waves.push_back({first, x});
                first = x;
                acc = 0;
            }
            acc += d;
        }
        waves.push_back({first, ns});
    }
    size_t wave_max = 0;
    for (auto &wv : waves) {
        long long items = 0, jobs = 0;
        for (int x = wv.first; x < wv.second; x++) {
            const int T = (probs[x].np + 1 + kSyrkT - 1) / kSyrkT;
            const long long nch = (probs[x].ndet + kSyrkChunk - 1) / kSyrkChunk;
            items += (probs[x].ndet + 255) / 256;
            jobs += nch * T * (T + 1) / 2;
        }
        wave_max = std::max(wave_max, ws_round(items * sizeof(WorkItem)) + ws_round(jobs * sizeof(SyrkJob)) +
                                          ws_round(jobs * kSyrkT * kSyrkT * 8) + ws_round((wv.second - wv.first) * 4));
    }
    need += wave_max + 4096;
    IFCI_TRY(ws_reserve(h, need));
    auto *d_probs = ws_take<RdmProb>(h, ns);
    int *d_orbs = ws_take<int>(h, P.orbs.size());
    int *d_bond = ws_take<int>(h, sys->nbody);
    double *D = ws_take<double>(h, budget);
    double *Mall = ws_take<double>(h, mtot);
    if (!d_probs || !d_orbs || !d_bond || !D || !Mall) return set_error(h, IFCI_ERR_OOM, "rdm_backward: workspace");
    std::map<std::pair<int, int>, int32_t *> tables;
    for (int x = 0; x < ns; x++) {
        auto key = std::make_pair(probs[x].n, (int)P.subsets[x].size());
        if (!tables.count(key)) {
            uint64_t *st = ws_take<uint64_t>(h, probs[x].nstr);
            int32_t *ex = ws_take<int32_t>(h, (size_t)probs[x].nstr * probs[x].nexc);
            if (!st || !ex) return set_error(h, IFCI_ERR_OOM, "rdm_backward: workspace (strings)");
            IFCI_TRY(ifci_build_strings(h, key.first, key.second, st, ex, stream));
            tables[key] = ex;
        }
    }
    {
        long long moff = 0;
        for (int x = 0; x < ns; x++) {
            probs[x].exc = tables[{probs[x].n, (int)P.subsets[x].size()}];
            probs[x].orbs = d_orbs + P.orb_off[x];
            probs[x].M = Mall + moff;
            moff += (long long)(probs[x].np + 1) * (probs[x].np + 1);
        }
    }
    std::vector<int> bond(sys->nbody);
    for (int b = 0; b < sys->nbody; b++) bond[b] = sys->body_offset[b];
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_orbs, P.orbs.data(), P.orbs.size() * 4, cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_bond, bond.data(), sys->nbody * 4, cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemsetAsync(dh, 0, (size_t)norb * norb * 8, s));
    IFCI_CUDA_TRY(h, cudaMemsetAsync(deri, 0, (size_t)npg * npg * 8, s));
    const size_t mark = h->ws_top;
    for (auto &wv : waves) {
        h->ws_top = mark;
        std::vector<WorkItem> items;
        std::vector<SyrkJob> jobs;
        std::vector<int> job0;
        long long doff = 0;
        int chunk = 0;
        for (int x = wv.first; x < wv.second; x++) {
            RdmProb &r = probs[x];
            r.doff = doff;
            doff += (long long)(r.np + 1) * r.ndet;
            for (long long s0 = 0; s0 < r.ndet; s0 += 256) items.push_back(WorkItem{x - wv.first, 0, s0});
            const int T = (r.np + 1 + kSyrkT - 1) / kSyrkT;
            r.nchunk = (int)((r.ndet + kSyrkChunk - 1) / kSyrkChunk);
            r.chunk0 = chunk;
            job0.push_back((int)jobs.size());
            for (int ch = 0; ch < r.nchunk; ch++)
                for (int ta = 0; ta < T; ta++)
                    for (int tb = ta; tb < T; tb++) jobs.push_back(SyrkJob{x - wv.first, chunk + ch, ta, tb});
            chunk += r.nchunk;
        }
        const int nw = wv.second - wv.first;
        auto *d_items = ws_take<WorkItem>(h, items.size());
        auto *d_jobs = ws_take<SyrkJob>(h, jobs.size());
        double *part = ws_take<double>(h, jobs.size() * kSyrkT * kSyrkT);
        int *d_job0 = ws_take<int>(h, nw);
        if (!d_items || !d_jobs || !part || !d_job0) return set_error(h, IFCI_ERR_OOM, "rdm_backward: workspace (wave)");
        RdmProb *d_wp = d_probs + wv.first;
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_wp, probs.data() + wv.first, nw * sizeof(RdmProb), cudaMemcpyHostToDevice, s));
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(SyrkJob), cudaMemcpyHostToDevice, s));
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_job0, job0.data(), nw * 4, cudaMemcpyHostToDevice, s));
        rdm_gather_kernel<<<(int)items.size(), 256, 0, s>>>(d_wp, d_items, D);
        IFCI_LAUNCH_CHECK(h);
        rdm_syrk_kernel<<<(int)jobs.size(), 256, 0, s>>>(d_wp, d_jobs, D, part);
        IFCI_LAUNCH_CHECK(h);
        rdm_reduce_kernel<<<nw, 256, 0, s>>>(d_wp, d_job0, part);
        IFCI_LAUNCH_CHECK(h);
        rdm_accum_kernel<<<nw, 256, 0, s>>>(d_wp, norb, dh, deri);
        IFCI_LAUNCH_CHECK(h);
        // the host vectors above are staged by cudaMemcpyAsync before it returns;
        // synchronise before the next wave reuses the workspace
        IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));
    }
    const double w0 = (1.0 - wsum) * grad_out;
    rdm_reference_kernel<<<4, 256, 0, s>>>(d_bond, sys->nbody, w0, norb, dh, deri);
    IFCI_LAUNCH_CHECK(h);
    rdm_symmetrise_kernel<<<1024, 256, 0, s>>>(npg, deri);
    IFCI_LAUNCH_CHECK(h);
    IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));
    return IFCI_OK;
}
