// Frozen-body effective Hamiltonians, the folded contraction matrix, the
// diagonal <I|H|I> and the reference energy.
#include "hamiltonian.cuh"

namespace ifci {

// One block per problem.  orbs = [active (nA) ..., core (nC) ...], global indices.
__global__ void frozen_core_kernel(const FrozenDesc *__restrict__ desc, const int *__restrict__ orbs_all,
                                   const double *__restrict__ h, const double *__restrict__ V, int norb) {
    const FrozenDesc d = desc[blockIdx.x];
    const int *act = orbs_all + d.orb_off;
    const int *core = act + d.nA;
    const int nA = d.nA, nC = d.nC;
    const long long npg = (long long)norb * (norb + 1) / 2;
    auto Vg = [&](int p, int q, int r, int s) -> double {
        return V[(long long)pair_of(p, q) * npg + pair_of(r, s)];
    };
    // h1_pq = h_pq + sum_c [2 (pq|cc) - (pc|cq)]
    for (int t = threadIdx.x; t < nA * nA; t += blockDim.x) {
        int p = act[t / nA], q = act[t % nA];
        double v = h[(long long)p * norb + q];
        for (int k = 0; k < nC; k++) {
            int c = core[k];
            v += 2.0 * Vg(p, q, c, c) - Vg(p, c, c, q);
        }
        d.h1[t] = v;
    }
    // (pq|rs) restricted to the active orbitals, local pair index
    const int npA = nA * (nA + 1) / 2;
    for (long long t = threadIdx.x; t < (long long)npA * npA; t += blockDim.x) {
        int A = (int)(t / npA), B = (int)(t % npA);
        int P = (int)((sqrt(8.0 * A + 1.0) - 1.0) * 0.5);
        while ((P + 1) * (P + 2) / 2 <= A) P++;
        while (P * (P + 1) / 2 > A) P--;
        int Q = A - P * (P + 1) / 2;
        int R = (int)((sqrt(8.0 * B + 1.0) - 1.0) * 0.5);
        while ((R + 1) * (R + 2) / 2 <= B) R++;
        while (R * (R + 1) / 2 > B) R--;
        int S = B - R * (R + 1) / 2;
        d.eri[t] = Vg(act[P], act[Q], act[R], act[S]);
    }
    // E_core = sum_c 2 h_cc + sum_{c,d} [2 (cc|dd) - (cd|dc)]   (fixed-order sum)
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int i = 0; i < nC; i++) {
            int c = core[i];
            e += 2.0 * h[(long long)c * norb + c];
            for (int j = 0; j < nC; j++) {
                int dd = core[j];
                e += 2.0 * Vg(c, c, dd, dd) - Vg(c, dd, dd, c);
            }
        }
        d.e_core[0] = e;
    }
}

// Folded contraction matrix W[A][B] = 1/2 [ (pq|rs) + (k_pq d_rs + d_pq k_rs) / N ],
// k_pq = h1_pq - 1/2 sum_r (pr|rq), N = 2 nelec_spin.  With it
//   H c = sum_{A,B} E+_A W[A][B] (E+_B c)        (E+_pq = E_pq + E_qp, E+_pp = E_pp)
// because sum_r E_rr = N on the CI space.  Rows/cols beyond npair are zero-padded
// up to ld (so the contraction can run on whole tiles).
__global__ void fold_kernel(const FoldDesc *__restrict__ desc) {
    const FoldDesc d = desc[blockIdx.x];
    const int n = d.n, np = n * (n + 1) / 2, ld = d.ld;
    extern __shared__ double kpair[];  // [np]
    for (int A = threadIdx.x; A < np; A += blockDim.x) {
        int P = 0;
        while ((P + 1) * (P + 2) / 2 <= A) P++;
        int Q = A - P * (P + 1) / 2;
        double k = d.h1[P * n + Q];
        for (int r = 0; r < n; r++) k -= 0.5 * d.eri[(long long)pair_of(P, r) * np + pair_of(r, Q)];
        kpair[A] = k;
    }
    __syncthreads();
    const double invN = d.nelec > 0 ? 1.0 / (double)d.nelec : 0.0;
    for (long long t = threadIdx.x; t < (long long)ld * ld; t += blockDim.x) {
        int A = (int)(t / ld), B = (int)(t % ld);
        double w = 0.0;
        if (A < np && B < np) {
            int P = 0;
            while ((P + 1) * (P + 2) / 2 <= A) P++;
            int R = 0;
            while ((R + 1) * (R + 2) / 2 <= B) R++;
            bool dA = (A - P * (P + 1) / 2) == P, dB = (B - R * (R + 1) / 2) == R;
            w = d.eri[(long long)A * np + B];
            if (dB) w += invN * kpair[A];
            if (dA) w += invN * kpair[B];
            w *= 0.5;
        }
        d.W[t] = w;
    }
}

// <I|H|I> = sum_p h_pp n_p + 1/2 sum_pq (pp|qq) n_p n_q
//           - 1/2 sum_pq (pq|qp) (na_p na_q + nb_p nb_q)
__global__ void hdiag_kernel(const HdiagDesc *__restrict__ desc, const int *__restrict__ work_prob,
                             const long long *__restrict__ work_start, int nwork, int chunk) {
    int w = blockIdx.x;
    if (w >= nwork) return;
    const HdiagDesc d = desc[work_prob[w]];
    const int n = d.n, np = n * (n + 1) / 2;
    long long I = work_start[w] + threadIdx.x;
    long long end = work_start[w] + chunk;
    if (end > (long long)d.nstr * d.nstr) end = (long long)d.nstr * d.nstr;
    for (; I < end; I += blockDim.x) {
        int ia = (int)(I / d.nstr), ib = (int)(I % d.nstr);
        uint32_t ma = (uint32_t)d.strings[ia], mb = (uint32_t)d.strings[ib];
        double e = 0.0;
        for (uint32_t x = ma; x; x &= x - 1) {
            int p = __ffs(x) - 1;
            e += d.h1[p * n + p];
        }
        for (uint32_t x = mb; x; x &= x - 1) {
            int p = __ffs(x) - 1;
            e += d.h1[p * n + p];
        }
        double two = 0.0;
        for (uint32_t x = ma; x; x &= x - 1) {
            int p = __ffs(x) - 1;
            for (uint32_t y = ma; y; y &= y - 1) {
                int q = __ffs(y) - 1;
                two += d.eri[(long long)pair_of(p, p) * np + pair_of(q, q)] -
                       d.eri[(long long)pair_of(p, q) * np + pair_of(q, p)];
            }
            for (uint32_t y = mb; y; y &= y - 1) {
                int q = __ffs(y) - 1;
                two += 2.0 * d.eri[(long long)pair_of(p, p) * np + pair_of(q, q)];
            }
        }
        for (uint32_t x = mb; x; x &= x - 1) {
            int p = __ffs(x) - 1;
            for (uint32_t y = mb; y; y &= y - 1) {
                int q = __ffs(y) - 1;
                two += d.eri[(long long)pair_of(p, p) * np + pair_of(q, q)] -
                       d.eri[(long long)pair_of(p, q) * np + pair_of(q, p)];
            }
        }
        d.hd[I] = e + 0.5 * two;
    }
}

// E_0 = sum_b 2 h_bb + sum_{b,b'} [2 (bb|b'b') - (bb'|b'b)] over bonding orbitals.
__global__ void reference_energy_kernel(const int *__restrict__ bond, int nb, const double *__restrict__ h,
                                        const double *__restrict__ V, int norb, double *__restrict__ e0) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const long long npg = (long long)norb * (norb + 1) / 2;
    double e = 0.0;
    for (int i = 0; i < nb; i++) {
        int c = bond[i];
        e += 2.0 * h[(long long)c * norb + c];
        for (int j = 0; j < nb; j++) {
            int d = bond[j];
            e += 2.0 * V[(long long)pair_of(c, c) * npg + pair_of(d, d)] -
                 V[(long long)pair_of(c, d) * npg + pair_of(d, c)];
        }
    }
    *e0 = e;
}

int launch_frozen_core(ifci_handle_t h, int nprob, const FrozenDesc *d_desc, const int *d_orbs,
                       const double *d_h, const double *d_V, int norb, cudaStream_t s) {
    if (nprob <= 0) return IFCI_OK;
    frozen_core_kernel<<<nprob, 256, 0, s>>>(d_desc, d_orbs, d_h, d_V, norb);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_fold(ifci_handle_t h, int nprob, const FoldDesc *d_desc, int max_np, cudaStream_t s) {
    if (nprob <= 0) return IFCI_OK;
    fold_kernel<<<nprob, 256, max_np * sizeof(double), s>>>(d_desc);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_hdiag(ifci_handle_t h, const HdiagDesc *d_desc, const int *d_wprob, const long long *d_wstart,
                 int nwork, int chunk, cudaStream_t s) {
    if (nwork <= 0) return IFCI_OK;
    hdiag_kernel<<<nwork, 256, 0, s>>>(d_desc, d_wprob, d_wstart, nwork, chunk);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

int launch_reference_energy(ifci_handle_t h, const int *d_bond, int nb, const double *d_h, const double *d_V,
                            int norb, double *d_e0, cudaStream_t s) {
    reference_energy_kernel<<<1, 32, 0, s>>>(d_bond, nb, d_h, d_V, norb, d_e0);
    IFCI_LAUNCH_CHECK(h);
    return IFCI_OK;
}

}  // namespace ifci

extern "C" int ifci_hdiag(ifci_handle_t h, const ifci_strings_t *str, const double *h1, const double *eri,
                          double *hd, ifci_stream_t stream) {
    if (!h || !str || !h1 || !eri || !hd) return IFCI_ERR_INVALID_ARG;
    IFCI_CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = ifci::as_cuda(stream);
    long long ndet = (long long)str->nstr * str->nstr;
    const int chunk = 4096;
    int nwork = (int)((ndet + chunk - 1) / chunk);
    size_t need = ifci::ws_round(sizeof(ifci::HdiagDesc)) + ifci::ws_round(nwork * sizeof(int)) +
                  ifci::ws_round(nwork * sizeof(long long));
    IFCI_TRY(ifci::ws_reserve(h, need));
    auto *dd = ifci::ws_take<ifci::HdiagDesc>(h, 1);
    auto *wp = ifci::ws_take<int>(h, nwork);
    auto *ws = ifci::ws_take<long long>(h, nwork);
    ifci::HdiagDesc d{str->norb, str->nstr, str->strings, h1, eri, hd};
    std::vector<int> hp(nwork, 0);
    std::vector<long long> hs(nwork);
    for (int i = 0; i < nwork; i++) hs[i] = (long long)i * chunk;
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(dd, &d, sizeof(d), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(wp, hp.data(), nwork * sizeof(int), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(ws, hs.data(), nwork * sizeof(long long), cudaMemcpyHostToDevice, s));
    IFCI_TRY(ifci::launch_hdiag(h, dd, wp, ws, nwork, chunk, s));
    // host vectors above are pageable: the copies complete before cudaMemcpyAsync returns
    return IFCI_OK;
}

namespace ifci {

cudaError_t launch_fold_raw(const FoldDesc *d_desc, int max_np, cudaStream_t s) {
    fold_kernel<<<1, 256, max_np * sizeof(double), s>>>(d_desc);
    return cudaGetLastError();
}

}  // namespace ifci
