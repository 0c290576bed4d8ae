// Heat-bath configuration interaction (HBCI) per CI space, the solver the
// paper runs for every increment (Methods, HBCI paragraph): the determinants
// that matter most are selected for a variational CI (threshold eps1), then
// second-order Epstein–Nesbet perturbation theory over the determinants
// outside the selection adds the rest (each term screened by eps2).
//
// Steps (the heat-bath criterion of the HBCI method the paper cites):
//   1. S = {start determinant} (the reference: every bonding orbital doubly
//      occupied), c = that determinant.
//   2. (E_var, c) = lowest eigenpair of H on S in the spin-flip-even sector:
//      the batched Davidson, seeded with the previous c, with sigma zeroed
//      outside S (DavProb::mask).
//   3. Every determinant a outside S with max_{i in S} |H_ai c_i| > eps1
//      joins S with its spin-flip image; back to 2 until none joins.
//   4. E_2 = sum_{a not in S} (sum_{i in S, |H_ai c_i| > eps2} H_ai c_i)^2
//      / (E_var - H_aa).
//
// GB300 layout: the determinant index of the whole CI space (I = Ia nstr +
// Ib, at most ~1e8 per space) is dense and HBM is large, so S is a byte mask
// over the space instead of a hash set, and the PT2 numerators an FP64 array
// over it (atomic adds).  The connections of a selected determinant are
// enumerated by one warp, whose lanes stride over the 2 n_s + 2 n_d + n_s^2
// single and double excitations (n_s = m (n - m) singles, n_d = C(m,2)
// C(n-m,2) same-spin doubles of one string) and evaluate H_ai by the
// Slater–Condon rules.  The variational step is the FP64E Davidson over the
// whole space (its sigma costs what an FCI sigma costs; the selection keeps
// the vectors on S).
#include <algorithm>
#include <map>

#include "dav_driver.cuh"
#include "slater.cuh"

namespace ifci {

namespace {

struct HbBinom {
    int c[33][8];   // C(p, k) for p <= 32, k <= 7 (string ranks of at most 7 electrons)
};

struct HbDesc {
    int n, m, nstr;
    long long ndet;
    const uint64_t *strings;   // class string table (ascending masks)
    const double *h1, *eri;
    unsigned char *mask, *mark;
    double *c;                 // current vector (zero outside S)
    double *num;               // EN-PT2 numerators
    double e_core;
};

__device__ __forceinline__ int hb_rank(uint32_t mask, const HbBinom &B) {
    int r = 0, k = 1;
    while (mask) {
        const int p = __ffs(mask) - 1;
        r += B.c[p][k];
        k++;
        mask &= mask - 1;
    }
    return r;
}

// position of the k-th set bit (k = 0 lowest) of x
__device__ __forceinline__ int nth_bit(uint32_t x, int k) {
    for (int i = 0; i < k; i++) x &= x - 1;
    return __ffs(x) - 1;
}

// i < j with pair index q in the lexical order of pairs of {0 .. cnt-1}
__device__ __forceinline__ void pair_decode(int q, int cnt, int &i, int &j) {
    i = 0;
    while (q >= cnt - 1 - i) {
        q -= cnt - 1 - i;
        i++;
    }
    j = i + 1 + q;
}

// the k-th single excitation of string s (n orbitals, m electrons)
__device__ __forceinline__ uint32_t single_exc(uint32_t s, int n, int m, int k) {
    const uint32_t full = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
    const int nv = n - m;
    const int i = nth_bit(s, k / nv), a = nth_bit(~s & full, k % nv);
    return s ^ (1u << i) ^ (1u << a);
}

// the k-th same-spin double excitation of string s
__device__ __forceinline__ uint32_t double_exc(uint32_t s, int n, int m, int k) {
    const uint32_t full = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
    const int nv = n - m, npv = nv * (nv - 1) / 2;
    int i, j, a, b;
    pair_decode(k / npv, m, i, j);
    pair_decode(k % npv, nv, a, b);
    const uint32_t vir = ~s & full;
    return s ^ (1u << nth_bit(s, i)) ^ (1u << nth_bit(s, j)) ^ (1u << nth_bit(vir, a)) ^ (1u << nth_bit(vir, b));
}

struct SelEntry {
    int prob;
    long long I;
};

// Per vector item: the selected determinants with c != 0 appended to the list.
__global__ void __launch_bounds__(256) hb_compact_kernel(const HbDesc *__restrict__ d, const WorkItem *__restrict__ items,
                                                         int nitem, SelEntry *__restrict__ list, long long cap,
                                                         unsigned long long *__restrict__ count) {
    for (int w = blockIdx.x; w < nitem; w += gridDim.x) {
        const WorkItem it = items[w];
        const HbDesc p = d[it.prob];
        const long long end = min(it.start + (long long)kVecChunk, p.ndet);
        for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
            if (!p.mask[I] || p.c[I] == 0.0) continue;
            const unsigned long long pos = atomicAdd(count, 1ull);
            if ((long long)pos < cap) list[pos] = SelEntry{it.prob, I};
        }
    }
}

// One warp per listed determinant i: every connected a outside S with
// |H_ai c_i| > eps.  SELECT marks a and its spin-flip image; otherwise the
// contribution is added to the PT2 numerator of a.
template <bool SELECT>
__global__ void __launch_bounds__(256) hb_connect_kernel(const HbDesc *__restrict__ d, const SelEntry *__restrict__ list,
                                                         long long nlist, double eps, HbBinom B) {
    const int lane = threadIdx.x & 31;
    const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long e = warp0; e < nlist; e += nwarp) {
        const SelEntry s = list[e];
        const HbDesc p = d[s.prob];
        const int nstr = p.nstr, n = p.n, m = p.m;
        const int ia = (int)(s.I / nstr), ib = (int)(s.I % nstr);
        const uint32_t ma = (uint32_t)p.strings[ia], mb = (uint32_t)p.strings[ib];
        const double ci = p.c[s.I];
        const int ns = m * (n - m);
        const int nd = (m * (m - 1) / 2) * ((n - m) * (n - m - 1) / 2);
        const long long total = 2ll * ns + 2ll * nd + (long long)ns * ns;
        for (long long u = lane; u < total; u += 32) {
            uint32_t ja = ma, jb = mb;
            if (u < ns) {
                ja = single_exc(ma, n, m, (int)u);
            } else if (u < 2 * ns) {
                jb = single_exc(mb, n, m, (int)(u - ns));
            } else if (u < 2 * ns + nd) {
                ja = double_exc(ma, n, m, (int)(u - 2 * ns));
            } else if (u < 2ll * ns + 2ll * nd) {
                jb = double_exc(mb, n, m, (int)(u - 2 * ns - nd));
            } else {
                const long long t = u - 2ll * ns - 2ll * nd;
                ja = single_exc(ma, n, m, (int)(t / ns));
                jb = single_exc(mb, n, m, (int)(t % ns));
            }
            const int ra = hb_rank(ja, B), rb = hb_rank(jb, B);
            const long long a = (long long)ra * nstr + rb;
            if (p.mask[a]) continue;
            const double v = h_element(n, p.h1, p.eri, ja, jb, ma, mb) * ci;
            if (!(fabs(v) > eps)) continue;
            if (SELECT) {
                p.mark[a] = 1;
                p.mark[(long long)rb * nstr + ra] = 1;
            } else {
                atomicAdd(p.num + a, v);
            }
        }
    }
}

// Marked determinants join S; per problem the new ones and the new diagonal
// ones (Ia = Ib) are counted.
__global__ void __launch_bounds__(256) hb_merge_kernel(const HbDesc *__restrict__ d, const WorkItem *__restrict__ items,
                                                       int nitem, unsigned long long *__restrict__ cnt) {
    __shared__ unsigned long long red[2][8];
    for (int w = blockIdx.x; w < nitem; w += gridDim.x) {
        const WorkItem it = items[w];
        const HbDesc p = d[it.prob];
        unsigned long long nnew = 0, ndiag = 0;
        const long long end = min(it.start + (long long)kVecChunk, p.ndet);
        for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
            if (!p.mark[I]) continue;
            p.mark[I] = 0;
            if (p.mask[I]) continue;
            p.mask[I] = 1;
            nnew++;
            if (I / p.nstr == I % p.nstr) ndiag++;
        }
        for (int o = 16; o > 0; o >>= 1) {
            nnew += __shfl_xor_sync(0xffffffffu, nnew, o);
            ndiag += __shfl_xor_sync(0xffffffffu, ndiag, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = nnew;
            red[1][threadIdx.x >> 5] = ndiag;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long a = 0, b = 0;
            for (int k = 0; k < 8; k++) {
                a += red[0][k];
                b += red[1][k];
            }
            if (a) atomicAdd(cnt + 2 * it.prob, a);
            if (b) atomicAdd(cnt + 2 * it.prob + 1, b);
        }
        __syncthreads();
    }
}

// E_2 of each problem: sum over a outside S of num_a^2 / (E_var - H_aa).
__global__ void __launch_bounds__(256) hb_pt2_kernel(const HbDesc *__restrict__ d, const WorkItem *__restrict__ items,
                                                     int nitem, const double *__restrict__ evar, double *__restrict__ e2) {
    __shared__ double red[8];
    for (int w = blockIdx.x; w < nitem; w += gridDim.x) {
        const WorkItem it = items[w];
        const HbDesc p = d[it.prob];
        double acc = 0.0;
        const long long end = min(it.start + (long long)kVecChunk, p.ndet);
        for (long long I = it.start + threadIdx.x; I < end; I += blockDim.x) {
            const double v = p.num[I];
            if (v == 0.0 || p.mask[I]) continue;
            const uint32_t ma = (uint32_t)p.strings[I / p.nstr], mb = (uint32_t)p.strings[I % p.nstr];
            const double haa = h_element(p.n, p.h1, p.eri, ma, mb, ma, mb) + p.e_core;
            acc += v * v / (evar[it.prob] - haa);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0;
            for (int k = 0; k < 8; k++) a += red[k];
            if (a != 0.0) atomicAdd(e2 + it.prob, a);
        }
        __syncthreads();
    }
}

__global__ void hb_start_kernel(const HbDesc *__restrict__ d, const long long *__restrict__ start, int nprob) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nprob) return;
    d[i].mask[start[i]] = 1;
    d[i].c[start[i]] = 1.0;
}

}  // namespace

int hbci_solve(ifci_handle_t h, const std::vector<ProbSpec> &specs, const std::vector<long long> &start,
               const ifci_davidson_opts_t &o, const ifci_hbci_opts_t &hb, double *e_var, double *e_pt2,
               long long *nsel_out, int *rounds_out, int *status, cudaStream_t s) {
    const int np_ = (int)specs.size();
    if (np_ == 0) return IFCI_OK;
    if (!(hb.eps1 >= 0) || !(hb.eps2 >= 0) || hb.max_rounds < 1)
        return set_error(h, IFCI_ERR_INVALID_ARG, "hbci: eps1, eps2 >= 0 and max_rounds >= 1 required");
    for (int i = 0; i < np_; i++) {
        const ProbSpec &p = specs[i];
        if (p.m < 1 || p.m > 7 || p.n > 32)
            return set_error(h, IFCI_ERR_UNSUPPORTED, "hbci: problem %d (norb %d, nelec_spin %d)", i, p.n, p.m);
        const long long nstr = binom(p.n, p.m);
        if (start[i] < 0 || start[i] >= nstr * nstr || start[i] / nstr != start[i] % nstr)
            return set_error(h, IFCI_ERR_INVALID_ARG, "hbci: start determinant of problem %d is not closed-shell", i);
    }
    HbBinom B{};
    for (int p = 0; p <= 32; p++)
        for (int k = 0; k < 8; k++) B.c[p][k] = (int)std::min<long long>(binom(p, k), 0x7fffffff);

    // ---- device memory of the selection (freed at the end): string tables per
    // class, then per problem mask, mark, c, num
    std::map<std::pair<int, int>, size_t> cls_off;
    size_t bytes = 0;
    for (const ProbSpec &p : specs) {
        auto key = std::make_pair(p.n, p.m);
        if (!cls_off.count(key)) {
            cls_off[key] = bytes;
            bytes += ws_round((size_t)binom(p.n, p.m) * 8);
        }
    }
    std::vector<size_t> poff(np_);
    std::vector<long long> ndet(np_);
    std::vector<WorkItem> items;
    for (int i = 0; i < np_; i++) {
        const long long nstr = binom(specs[i].n, specs[i].m);
        ndet[i] = nstr * nstr;
        poff[i] = bytes;
        bytes += 2 * ws_round((size_t)ndet[i]) + 2 * ws_round((size_t)ndet[i] * 8);
        for (long long s0 = 0; s0 < ndet[i]; s0 += kVecChunk) items.push_back(WorkItem{i, 0, s0});
    }
    const size_t off_desc = bytes;
    bytes += ws_round(np_ * sizeof(HbDesc));
    const size_t off_items = bytes;
    bytes += ws_round(items.size() * sizeof(WorkItem));
    const size_t off_small = bytes;   // start dets, counts, E_var, E_2
    bytes += ws_round(np_ * 8) + ws_round(np_ * 16) + 2 * ws_round(np_ * 8) + ws_round(8);
    char *mem = nullptr;
    IFCI_CUDA_TRY(h, cudaMalloc(&mem, bytes));
    int rc = IFCI_OK;
    auto fail = [&](int code, const char *msg) {
        if (rc == IFCI_OK) rc = set_error(h, code, "%s", msg);
    };
    for (auto &kv : cls_off) {
        const std::vector<uint32_t> st = host_strings(kv.first.first, kv.first.second);
        std::vector<uint64_t> st64(st.begin(), st.end());
        if (cudaMemcpyAsync(mem + kv.second, st64.data(), st64.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
            fail(IFCI_ERR_CUDA, "hbci: string tables");
    }
    std::vector<HbDesc> desc(np_);
    for (int i = 0; i < np_; i++) {
        const ProbSpec &p = specs[i];
        HbDesc &d = desc[i];
        d.n = p.n;
        d.m = p.m;
        d.nstr = (int)binom(p.n, p.m);
        d.ndet = ndet[i];
        d.strings = reinterpret_cast<const uint64_t *>(mem + cls_off[{p.n, p.m}]);
        d.h1 = p.h1;
        d.eri = p.eri;
        char *q = mem + poff[i];
        d.mask = reinterpret_cast<unsigned char *>(q);
        d.mark = d.mask + ws_round((size_t)ndet[i]);
        d.c = reinterpret_cast<double *>(q + 2 * ws_round((size_t)ndet[i]));
        d.num = d.c + ws_round((size_t)ndet[i] * 8) / 8;
        d.e_core = p.e_core;
        if (cudaMemsetAsync(q, 0, 2 * ws_round((size_t)ndet[i]) + ws_round((size_t)ndet[i] * 8), s) != cudaSuccess)
            fail(IFCI_ERR_CUDA, "hbci: clear");
    }
    auto *d_desc = reinterpret_cast<HbDesc *>(mem + off_desc);
    auto *d_items = reinterpret_cast<WorkItem *>(mem + off_items);
    auto *d_start = reinterpret_cast<long long *>(mem + off_small);
    auto *d_cnt = reinterpret_cast<unsigned long long *>(mem + off_small + ws_round(np_ * 8));
    auto *d_evar = reinterpret_cast<double *>(mem + off_small + ws_round(np_ * 8) + ws_round(np_ * 16));
    auto *d_e2 = d_evar + ws_round(np_ * 8) / 8;
    auto *d_count = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(d_e2) + ws_round(np_ * 8));
    if (rc == IFCI_OK &&
        (cudaMemcpyAsync(d_desc, desc.data(), np_ * sizeof(HbDesc), cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s) !=
             cudaSuccess ||
         cudaMemcpyAsync(d_start, start.data(), np_ * 8, cudaMemcpyHostToDevice, s) != cudaSuccess))
        fail(IFCI_ERR_CUDA, "hbci: descriptors");
    if (rc == IFCI_OK) {
        hb_start_kernel<<<(np_ + 127) / 128, 128, 0, s>>>(d_desc, d_start, np_);
        if (cudaGetLastError() != cudaSuccess) fail(IFCI_ERR_CUDA, "hbci: start");
        h->launches++;
    }

    // ---- rounds: Davidson on S, then selection
    std::vector<long long> nsel(np_, 1), ndiag(np_, 1);
    std::vector<int> rounds(np_, 0), stt(np_, IFCI_OK), active(np_, 1);
    std::vector<double> ev(np_, 0.0);
    ifci_davidson_opts_t od = o;
    od.decouple_tol = 0.0;
    od.sector_passes = 0;
    SelEntry *list = nullptr;
    long long list_cap = 0;
    auto build_list = [&](const std::vector<int> &probs_on, long long &nlist) -> int {
        long long need = 0;
        for (int i : probs_on) need += nsel[i];
        if (need > list_cap) {
            if (list) cudaFree(list);
            list = nullptr;
            list_cap = std::max(need, 1ll << 16);
            IFCI_CUDA_TRY(h, cudaMalloc(&list, list_cap * sizeof(SelEntry)));
        }
        // the items of the listed problems only
        std::vector<WorkItem> its;
        for (int i : probs_on)
            for (long long s0 = 0; s0 < ndet[i]; s0 += kVecChunk) its.push_back(WorkItem{i, 0, s0});
        WorkItem *d_its = nullptr;
        IFCI_CUDA_TRY(h, cudaMalloc(&d_its, std::max<size_t>(its.size(), 1) * sizeof(WorkItem)));
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_its, its.data(), its.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
        IFCI_CUDA_TRY(h, cudaMemsetAsync(d_count, 0, 8, s));
        hb_compact_kernel<<<stride_grid(h->device, (long long)its.size(), 8), 256, 0, s>>>(
            d_desc, d_its, (int)its.size(), list, list_cap, d_count);
        IFCI_LAUNCH_CHECK(h);
        unsigned long long cnt = 0;
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(&cnt, d_count, 8, cudaMemcpyDeviceToHost, s));
        IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));
        cudaFree(d_its);
        nlist = std::min<long long>((long long)cnt, list_cap);
        return IFCI_OK;
    };
    for (int round = 1; rc == IFCI_OK && round <= hb.max_rounds; round++) {
        std::vector<int> on;
        for (int i = 0; i < np_; i++)
            if (active[i]) on.push_back(i);
        if (on.empty()) break;
        std::vector<ProbSpec> sp;
        for (int i : on) {
            ProbSpec q = specs[i];
            q.c_out = desc[i].c;
            q.seed = desc[i].c;
            q.mask = desc[i].mask;
            q.ndim = (nsel[i] + ndiag[i]) / 2;
            q.seed_block = 0;
            sp.push_back(q);
        }
        std::vector<double> e(on.size());
        std::vector<int> it(on.size()), st(on.size());
        const int r = dav_solve(h, sp, od, e.data(), it.data(), st.data(), s);
        if (r != IFCI_OK && r != IFCI_ERR_NOT_CONVERGED) {
            rc = r;
            break;
        }
        for (size_t k = 0; k < on.size(); k++) {
            ev[on[k]] = e[k];
            rounds[on[k]] = round;
            if (st[k] != IFCI_OK) stt[on[k]] = st[k];
        }
        if (round == hb.max_rounds) break;
        // selection from the new vectors
        long long nlist = 0;
        rc = build_list(on, nlist);
        if (rc != IFCI_OK) break;
        if (nlist > 0) {
            hb_connect_kernel<true><<<stride_grid(h->device, (nlist + 7) / 8, 8), 256, 0, s>>>(d_desc, list, nlist,
                                                                                              hb.eps1, B);
            if (cudaGetLastError() != cudaSuccess) { fail(IFCI_ERR_CUDA, "hbci: selection"); break; }
            h->launches++;
        }
        if (cudaMemsetAsync(d_cnt, 0, np_ * 16, s) != cudaSuccess) { fail(IFCI_ERR_CUDA, "hbci: counts"); break; }
        hb_merge_kernel<<<stride_grid(h->device, (long long)items.size(), 8), 256, 0, s>>>(d_desc, d_items,
                                                                                         (int)items.size(), d_cnt);
        if (cudaGetLastError() != cudaSuccess) { fail(IFCI_ERR_CUDA, "hbci: merge"); break; }
        h->launches++;
        std::vector<unsigned long long> cnt((size_t)np_ * 2);
        if (cudaMemcpyAsync(cnt.data(), d_cnt, np_ * 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { fail(IFCI_ERR_CUDA, "hbci: counts"); break; }
        for (int i : on) {
            nsel[i] += (long long)cnt[2 * i];
            ndiag[i] += (long long)cnt[2 * i + 1];
            if (cnt[2 * i] == 0) active[i] = 0;
        }
    }

    // ---- EN-PT2 outside the final S
    if (rc == IFCI_OK) {
        std::vector<int> all(np_);
        for (int i = 0; i < np_; i++) all[i] = i;
        for (int i = 0; i < np_ && rc == IFCI_OK; i++)
            if (cudaMemsetAsync(desc[i].num, 0, (size_t)ndet[i] * 8, s) != cudaSuccess) fail(IFCI_ERR_CUDA, "hbci: pt2");
        long long nlist = 0;
        if (rc == IFCI_OK) rc = build_list(all, nlist);
        if (rc == IFCI_OK && nlist > 0) {
            hb_connect_kernel<false><<<stride_grid(h->device, (nlist + 7) / 8, 8), 256, 0, s>>>(d_desc, list, nlist,
                                                                                               hb.eps2, B);
            if (cudaGetLastError() != cudaSuccess) fail(IFCI_ERR_CUDA, "hbci: pt2 numerators");
            h->launches++;
        }
        if (rc == IFCI_OK &&
            (cudaMemcpyAsync(d_evar, ev.data(), np_ * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
             cudaMemsetAsync(d_e2, 0, np_ * 8, s) != cudaSuccess))
            fail(IFCI_ERR_CUDA, "hbci: pt2");
        if (rc == IFCI_OK) {
            hb_pt2_kernel<<<stride_grid(h->device, (long long)items.size(), 8), 256, 0, s>>>(
                d_desc, d_items, (int)items.size(), d_evar, d_e2);
            if (cudaGetLastError() != cudaSuccess) fail(IFCI_ERR_CUDA, "hbci: pt2 sum");
            h->launches++;
        }
        std::vector<double> e2(np_, 0.0);
        if (rc == IFCI_OK && (cudaMemcpyAsync(e2.data(), d_e2, np_ * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                              cudaStreamSynchronize(s) != cudaSuccess))
            fail(IFCI_ERR_CUDA, "hbci: pt2 result");
        for (int i = 0; i < np_ && rc == IFCI_OK; i++) {
            if (specs[i].c_out &&
                cudaMemcpyAsync(specs[i].c_out, desc[i].c, (size_t)ndet[i] * 8, cudaMemcpyDeviceToDevice, s) !=
                    cudaSuccess)
                fail(IFCI_ERR_CUDA, "hbci: vector out");
            if (e_var) e_var[i] = ev[i];
            if (e_pt2) e_pt2[i] = e2[i];
            if (nsel_out) nsel_out[i] = nsel[i];
            if (rounds_out) rounds_out[i] = rounds[i];
            if (status) status[i] = stt[i];
        }
    }
    cudaStreamSynchronize(s);
    if (list) cudaFree(list);
    cudaFree(mem);
    if (rc != IFCI_OK) return rc;
    for (int i = 0; i < np_; i++)
        if (stt[i] != IFCI_OK) return set_error(h, IFCI_ERR_NOT_CONVERGED, "hbci: some Davidson solves did not converge");
    return IFCI_OK;
}

}  // namespace ifci

extern "C" int ifci_hbci_batched(ifci_handle_t h, int nprob, const ifci_problem_t *probs, const long long *start_det,
                                 const ifci_davidson_opts_t *dopts, const ifci_hbci_opts_t *hopts, double *e_var,
                                 double *e_pt2, long long *nsel, int *rounds, int *status, ifci_stream_t stream) {
    using namespace ifci;
    if (!h) return IFCI_ERR_INVALID_ARG;
    if (nprob < 0 || (nprob > 0 && (!probs || !start_det || !hopts || !e_var || !e_pt2)))
        return set_error(h, IFCI_ERR_INVALID_ARG, "hbci_batched: bad arguments");
    ifci_davidson_opts_t o;
    ifci_davidson_default_opts(&o);
    if (dopts) o = *dopts;
    IFCI_TRY(check_opts(h, o));
    std::vector<ProbSpec> specs;
    std::vector<long long> start(start_det, start_det + nprob);
    for (int i = 0; i < nprob; i++) {
        const ifci_problem_t &p = probs[i];
        if (!p.h1 || !p.eri || p.nelec_spin < 1 || ifci_string_counts(p.norb, p.nelec_spin, nullptr, nullptr))
            return set_error(h, IFCI_ERR_INVALID_ARG, "hbci_batched: problem %d invalid", i);
        ProbSpec q{p.norb, p.nelec_spin, p.h1, p.eri, p.e_core, p.c_out};
        specs.push_back(q);
    }
    IFCI_CUDA_TRY(h, cudaSetDevice(h->device));
    return hbci_solve(h, specs, start, o, *hopts, e_var, e_pt2, nsel, rounds, status, as_cuda(stream));
}
