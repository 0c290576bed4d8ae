// The iFCI expansion (Methods, Eqs. 1-5): body sets, frozen-body CI problems,
// batched Davidson, and the FP64 increments eps_X with their sum.
#include <algorithm>
#include <cmath>

#include "dav_driver.cuh"
#include "hamiltonian.cuh"
#include "system.cuh"

namespace ifci {

// eps_X = sum over non-empty Y subset of X of (-1)^(|X|-|Y|) (E_Y - E_0)
// (the solution of Eqs. 2-5).  sub_idx lists, for each X, the positions of
// its subsets; sub_sgn the matching signs.
__global__ void increments_kernel(int nsub, const long long *__restrict__ sub_off, const int *__restrict__ sub_idx,
                                  const signed char *__restrict__ sub_sgn, const double *__restrict__ ex,
                                  const double *__restrict__ e0, double *__restrict__ eps) {
    int X = blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= nsub) return;
    const double E0 = *e0;
    double v = 0.0;
    for (long long t = sub_off[X]; t < sub_off[X + 1]; t++) v += (double)sub_sgn[t] * (ex[sub_idx[t]] - E0);
    eps[X] = v;
}

// Under screening, Eqs. 2-5 taken recursively for the sets x0..x1-1 (one
// size): eps_X = E_c(X) - sum over the proper subsets Y of eps_Y, a screened
// set's increment being 0 (its subsets' increments are already final).
__global__ void increments_rec_kernel(int x0, int x1, const long long *__restrict__ sub_off,
                                      const int *__restrict__ sub_idx, const char *__restrict__ incl,
                                      const double *__restrict__ ex, const double *__restrict__ e0,
                                      double *__restrict__ eps) {
    const int X = x0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= x1) return;
    if (!incl[X]) {
        eps[X] = 0.0;
        return;
    }
    double v = ex[X] - *e0;
    for (long long t = sub_off[X]; t < sub_off[X + 1]; t++) {
        const int y = sub_idx[t];
        if (y != X) v -= eps[y];
    }
    eps[X] = v;
}

// E_total = E_0 + sum_X eps_X, compensated summation in a fixed order.
__global__ void total_kernel(int nsub, const double *__restrict__ eps, const double *__restrict__ e0,
                             double *__restrict__ total) {
    if (threadIdx.x || blockIdx.x) return;
    double s = 0.0, c = 0.0;
    for (int i = 0; i < nsub; i++) {
        double y = eps[i] - c;
        double t = s + y;
        c = (t - s) - y;
        s = t;
    }
    *total = *e0 + s;
}

}  // namespace ifci

extern "C" {

int ifci_num_subsets(int nbody, int max_order, long long *count) {
    if (nbody < 1 || max_order < 1 || max_order > nbody || !count) return IFCI_ERR_INVALID_ARG;
    long long c = 0;
    for (int k = 1; k <= max_order; k++) c += ifci::binom(nbody, k);
    *count = c;
    return IFCI_OK;
}

int ifci_increments(ifci_handle_t h, const ifci_system_t *sys, int max_order, const ifci_davidson_opts_t *opts,
                    double *e0, double *e_x, double *eps, double *e_total, int *iters, int *status,
                    ifci_stream_t stream) {
    using namespace ifci;
    if (!h) return IFCI_ERR_INVALID_ARG;
    IFCI_TRY(validate_system(h, sys, max_order));
    if (!e0 || !eps || !e_total) return set_error(h, IFCI_ERR_INVALID_ARG, "increments: null output");
    ifci_davidson_opts_t o;
    ifci_davidson_default_opts(&o);
    if (opts) o = *opts;
    IFCI_TRY(check_opts(h, o));
    IFCI_CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = as_cuda(stream);
    const int norb = sys->norb;
    for (int b = 0; b < sys->nbody; b++)
        if (sys->body_offset[b + 1] - sys->body_offset[b] > kMaxNorb)
            return set_error(h, IFCI_ERR_INVALID_ARG, "increments: body %d too large", b);
    const long long npg = (long long)norb * (norb + 1) / 2;
    SubsetPlan P;
    plan_subsets(sys, max_order, P);
    const int ns = (int)P.subsets.size();
    for (int x = 0; x < ns; x++)
        if (P.nA[x] > kMaxNorb || binom(P.nA[x], (int)P.subsets[x].size()) >= kMaxStr)
            return set_error(h, IFCI_ERR_INVALID_ARG, "increments: body set %d has %d active orbitals", x, P.nA[x]);

    // keep the converged vectors for the backward pass (exact CI only)
    const bool keep = o.refine >= 0 && o.hbci_max_rounds == 0;
    std::vector<long long> vec_off(ns + 1, 0);
    for (int x = 0; x < ns; x++) {
        long long nstr = binom(P.nA[x], (int)P.subsets[x].size());
        vec_off[x + 1] = vec_off[x] + nstr * nstr;
    }
    if (keep) {
        size_t need = (size_t)vec_off[ns] * 8;
        if (h->kept.vec_bytes < need) {
            IFCI_CUDA_TRY(h, cudaDeviceSynchronize());
            if (h->kept.vec) cudaFree(h->kept.vec);
            h->kept.vec = nullptr;
            h->kept.vec_bytes = 0;
            cudaError_t e = cudaMalloc(&h->kept.vec, need);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return set_error(h, IFCI_ERR_OOM, "increments: %zu bytes for kept vectors", need);
            }
            h->kept.vec_bytes = need;
        }
        h->kept.valid = false;
    }

    // workspace: system copy, frozen-core outputs, subset tables, then Davidson batches
    size_t fixed = ws_round(ns * sizeof(FrozenDesc)) + ws_round(P.orbs.size() * 4) + ws_round((size_t)ns * 8) * 3 +
                   ws_round(8) * 2 + ws_round((ns + 1) * 8) + ws_round(P.sub_idx.size() * 4) +
                   ws_round(P.sub_sgn.size()) + ws_round(sys->nbody * 4) + ws_round(ns);
    if (sys->on_host) fixed += ws_round((size_t)norb * norb * 8) + ws_round((size_t)npg * npg * 8);
    std::vector<long long> h1_off(ns + 1, 0), eri_off(ns + 1, 0);
    for (int x = 0; x < ns; x++) {
        long long na = P.nA[x], npa = na * (na + 1) / 2;
        h1_off[x + 1] = h1_off[x] + na * na;
        eri_off[x + 1] = eri_off[x] + npa * npa;
    }
    fixed += ws_round((size_t)h1_off[ns] * 8) + ws_round((size_t)eri_off[ns] * 8);

    // Davidson batches under a vector-memory cap (the solves take their memory
    // from the handle's Davidson workspace)
    const size_t cap = (size_t)120 << 30;
    IFCI_TRY(ws_reserve(h, fixed));

    const double *dh = sys->h, *dV = sys->eri;
    if (sys->on_host) {
        double *th = ws_take<double>(h, (size_t)norb * norb);
        double *tV = ws_take<double>(h, (size_t)npg * npg);
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(th, sys->h, (size_t)norb * norb * 8, cudaMemcpyHostToDevice, s));
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(tV, sys->eri, (size_t)npg * npg * 8, cudaMemcpyHostToDevice, s));
        dh = th;
        dV = tV;
    }
    auto *d_fd = ws_take<FrozenDesc>(h, ns);
    int *d_orbs = ws_take<int>(h, P.orbs.size());
    double *d_ecore = ws_take<double>(h, ns);
    double *d_ex = ws_take<double>(h, ns);
    double *d_eps = ws_take<double>(h, ns);
    double *d_e0 = ws_take<double>(h, 1);
    double *d_tot = ws_take<double>(h, 1);
    long long *d_soff = ws_take<long long>(h, ns + 1);
    int *d_sidx = ws_take<int>(h, P.sub_idx.size());
    signed char *d_ssgn = ws_take<signed char>(h, P.sub_sgn.size());
    int *d_bond = ws_take<int>(h, sys->nbody);
    double *d_h1 = ws_take<double>(h, h1_off[ns]);
    double *d_eri = ws_take<double>(h, eri_off[ns]);
    if (!d_fd || !d_orbs || !d_ecore || !d_ex || !d_eps || !d_e0 || !d_tot || !d_soff || !d_sidx || !d_ssgn ||
        !d_bond || !d_h1 || !d_eri)
        return set_error(h, IFCI_ERR_OOM, "increments: workspace");
    std::vector<FrozenDesc> fd(ns);
    for (int x = 0; x < ns; x++)
        fd[x] = FrozenDesc{P.nA[x], P.nC[x], P.orb_off[x], d_h1 + h1_off[x], d_eri + eri_off[x], d_ecore + x};
    std::vector<int> bond(sys->nbody);
    for (int b = 0; b < sys->nbody; b++) bond[b] = sys->body_offset[b];
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_fd, fd.data(), ns * sizeof(FrozenDesc), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_orbs, P.orbs.data(), P.orbs.size() * 4, cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_soff, P.sub_off.data(), (ns + 1) * 8, cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_sidx, P.sub_idx.data(), P.sub_idx.size() * 4, cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_ssgn, P.sub_sgn.data(), P.sub_sgn.size(), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_bond, bond.data(), sys->nbody * 4, cudaMemcpyHostToDevice, s));
    IFCI_TRY(launch_frozen_core(h, ns, d_fd, d_orbs, dh, dV, norb, s));
    IFCI_TRY(launch_reference_energy(h, d_bond, sys->nbody, dh, dV, norb, d_e0, s));
    std::vector<double> ecore(ns);
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(ecore.data(), d_ecore, ns * 8, cudaMemcpyDeviceToHost, s));
    IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));

    std::vector<double> ex(ns, 0.0);
    std::vector<int> st(ns, IFCI_OK), its(ns, 0);
    int ret = IFCI_OK;
    // solves the listed sets, in batches under the vector-memory cap
    auto solve_sets = [&](const std::vector<int> &xs) -> int {
        size_t first = 0, acc = 0;
        for (size_t j = 0; j <= xs.size(); j++) {
            size_t vb = 0;
            if (j < xs.size()) {
                const long long nstr = binom(P.nA[xs[j]], (int)P.subsets[xs[j]].size());
                vb = (size_t)(2 * (o.max_space + 1) + 1) * nstr * nstr * 8;
            }
            if (j == xs.size() || (acc + vb > cap && j > first)) {
                std::vector<ProbSpec> sp;
                for (size_t t = first; t < j; t++) {
                    const int x = xs[t];
                    sp.push_back(ProbSpec{P.nA[x], (int)P.subsets[x].size(), d_h1 + h1_off[x], d_eri + eri_off[x],
                                          ecore[x], keep ? h->kept.vec + vec_off[x] : nullptr});
                }
                std::vector<double> e(sp.size());
                std::vector<int> it(sp.size()), stt(sp.size());
                int r;
                if (o.hbci_max_rounds > 0) {
                    // HBCI from the reference determinant of X: every bonding
                    // orbital (each body's first) doubly occupied; X's orbitals
                    // in body order, strings ranked by increasing bit mask
                    std::vector<long long> start;
                    for (size_t t = first; t < j; t++) {
                        const std::vector<int> &X = P.subsets[xs[t]];
                        long long rank = 0;
                        int off = 0;
                        for (size_t k = 0; k < X.size(); k++) {
                            rank += binom(off, (int)k + 1);
                            off += sys->body_offset[X[k] + 1] - sys->body_offset[X[k]];
                        }
                        const long long nstr = binom(P.nA[xs[t]], (int)X.size());
                        start.push_back(rank * nstr + rank);
                    }
                    const ifci_hbci_opts_t hb{o.hbci_eps1, o.hbci_eps2, o.hbci_max_rounds};
                    std::vector<double> e2(sp.size());
                    r = hbci_solve(h, sp, start, o, hb, e.data(), e2.data(), nullptr, it.data(), stt.data(), s);
                    for (size_t t = 0; t < sp.size(); t++) e[t] += e2[t];
                } else {
                    r = dav_solve_sectors(h, sp, o, e.data(), it.data(), stt.data(), s);
                }
                if (r != IFCI_OK && r != IFCI_ERR_NOT_CONVERGED) return r;
                if (r != IFCI_OK) ret = r;
                for (size_t t = first; t < j; t++) {
                    ex[xs[t]] = e[t - first];
                    its[xs[t]] = it[t - first];
                    st[xs[t]] = stt[t - first];
                }
                first = j;
                acc = 0;
            }
            acc += vb;
        }
        return IFCI_OK;
    };
    const bool screen = o.cnb_threshold > 0 && max_order >= 3;
    std::vector<char> included(ns, 1);
    if (!screen) {
        std::vector<int> all_x(ns);
        for (int x = 0; x < ns; x++) all_x[x] = x;
        IFCI_TRY(solve_sets(all_x));
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_ex, ex.data(), ns * 8, cudaMemcpyHostToDevice, s));
        increments_kernel<<<(ns + 127) / 128, 128, 0, s>>>(ns, d_soff, d_sidx, d_ssgn, d_ex, d_e0, d_eps);
        IFCI_LAUNCH_CHECK(h);
    } else {
        // connected n-body screening: sets of 1 and 2 bodies are all solved; the
        // sets of each larger size after the increments of the smaller ones
        char *d_incl = ws_take<char>(h, ns);
        if (!d_incl) return set_error(h, IFCI_ERR_OOM, "increments: workspace (screening)");
        std::vector<int> size_off(max_order + 2, 0);
        for (int x = 0; x < ns; x++) size_off[P.subsets[x].size() + 1] = x + 1;
        std::vector<double> eps_h(ns, 0.0);
        for (int k = 1; k <= max_order; k++) {
            const int x0 = size_off[k], x1 = size_off[k + 1];
            std::vector<int> xs;
            for (int x = x0; x < x1; x++) {
                if (k >= 3) included[x] = cnb_connected(P.subsets[x], sys->nbody, eps_h, o.cnb_threshold) ? 1 : 0;
                if (included[x]) xs.push_back(x);
                else st[x] = IFCI_SCREENED;
            }
            IFCI_TRY(solve_sets(xs));
            IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_ex + x0, ex.data() + x0, (size_t)(x1 - x0) * 8, cudaMemcpyHostToDevice, s));
            IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_incl + x0, included.data() + x0, (size_t)(x1 - x0),
                                             cudaMemcpyHostToDevice, s));
            increments_rec_kernel<<<(x1 - x0 + 127) / 128, 128, 0, s>>>(x0, x1, d_soff, d_sidx, d_incl, d_ex, d_e0,
                                                                         d_eps);
            IFCI_LAUNCH_CHECK(h);
            if (k + 1 <= max_order) {
                IFCI_CUDA_TRY(h, cudaMemcpyAsync(eps_h.data() + x0, d_eps + x0, (size_t)(x1 - x0) * 8,
                                                 cudaMemcpyDeviceToHost, s));
                IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));
            }
        }
        for (int x = 0; x < ns; x++)
            if (!included[x]) ex[x] = std::nan("");
    }
    total_kernel<<<1, 32, 0, s>>>(ns, d_eps, d_e0, d_tot);
    IFCI_LAUNCH_CHECK(h);
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(eps, d_eps, ns * 8, cudaMemcpyDeviceToHost, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(e0, d_e0, 8, cudaMemcpyDeviceToHost, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(e_total, d_tot, 8, cudaMemcpyDeviceToHost, s));
    IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));
    if (e_x) std::copy(ex.begin(), ex.end(), e_x);
    if (status) std::copy(st.begin(), st.end(), status);
    if (iters) std::copy(its.begin(), its.end(), iters);
    if (keep) {
        h->kept.screened = screen;
        h->kept.included = included;
        h->kept.valid = true;
        h->kept.nbody = sys->nbody;
        h->kept.max_order = max_order;
        h->kept.norb = norb;
        h->kept.body_offset.assign(sys->body_offset, sys->body_offset + sys->nbody + 1);
        h->kept.vec_off = vec_off;
    }
    for (int x = 0; x < ns; x++)
        if (st[x] != IFCI_OK && st[x] != IFCI_SCREENED) ret = IFCI_ERR_NOT_CONVERGED;
    if (ret != IFCI_OK) set_error(h, ret, "increments: some body sets did not converge");
    return ret;
}

}  // extern "C"
