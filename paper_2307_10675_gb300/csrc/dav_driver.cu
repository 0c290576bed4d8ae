// Host driver of the batched Davidson: workspace layout, string tables per
// (norb, nelec_spin) class, folded matrices, diagonals, and the C entry point.
#include <algorithm>
#include <map>

#include "dav_driver.cuh"
#include "hamiltonian.cuh"
#include "tc_gather.cuh"

namespace ifci {

int launch_convert_w(ifci_handle_t h, int nprob, const SigmaProb *d_probs, cudaStream_t s);

static void dav_layout(const std::vector<ProbSpec> &specs, const ifci_davidson_opts_t &o, DavSizes &z) {
    z = DavSizes{};
    std::map<std::pair<int, int>, int> cls;
    const int ms = o.max_space;
    const bool lo = o.precision == IFCI_FP32 || o.precision == IFCI_TF32 || o.precision == IFCI_BF16;
    const bool tc = o.precision == IFCI_BF16 || o.precision == IFCI_TF32;
    const bool oz = hi_precision_of(o) == IFCI_FP64E;
    const size_t eb_lo = sigma_elem_bytes(o.precision);
    for (const ProbSpec &p : specs) {
        int nstr = (int)binom(p.n, p.m), nexc = p.m * (p.n - p.m + 1);
        long long ndet = (long long)nstr * nstr;
        int np = p.n * (p.n + 1) / 2;
        if (!cls.count({p.n, p.m})) {
            cls[{p.n, p.m}] = (int)cls.size();
            z.bytes += ws_round((size_t)nstr * 8) + ws_round((size_t)nstr * nexc * 4) +
                       ws_round((size_t)nstr * kBlk16Stride);
            if (tc || oz) z.bytes += ws_round((size_t)nstr * pmap_ld(np) * 4);   // pair map
        }
        z.bytes += ws_round((size_t)np * np * 8);                       // W
        if (lo) z.bytes += ws_round((size_t)np * np * 4);               // Wf
        if (tc) z.bytes += ws_round((size_t)tc_operand_bytes(np, o.precision));
        if (oz) z.bytes += ws_round((size_t)oz_operand_bytes(np));
        z.bytes += ws_round((size_t)ndet * 8);                          // hd
        z.bytes += 2 * ws_round((size_t)(ms + 1) * ndet * 8);           // B, S
        z.nitem += (int)((ndet + kVecChunk - 1) / kVecChunk);
        z.max_pd = std::max(z.max_pd, sigma_elems(np, ndet));
        z.sum_pd += sigma_elems(np, ndet);
        z.n_items_sigma += (ndet + kGatherChunk - 1) / kGatherChunk;
        z.n_tiles_sigma += ((np + kGemmTM - 1) / kGemmTM) * ((ndet + kGemmTN - 1) / kGemmTN) +
                           tcg::row_tile_count(nstr) * ((np + oz_tile_n() - 1) / oz_tile_n() + 1);
    }
    size_t n = specs.size();
    z.nclass = (int)cls.size();
    long long budget = o.det_budget > 0 ? o.det_budget : (1ll << 31);   // two 16 GB intermediates
    budget = std::max(budget, z.max_pd);
    budget = std::min(budget, std::max(z.sum_pd, z.max_pd));
    z.budget = budget;
    size_t eb = 8;  // FP64 sigma is always needed (hi path); the lo buffers share it
    (void)eb_lo;
    z.bytes += 2 * ws_round((size_t)budget * eb);                          // D, G
    z.bytes += ws_round(n * sizeof(DavProb)) + ws_round(n * sizeof(DavState)) + ws_round(z.nitem * sizeof(WorkItem));
    z.bytes += ws_round((size_t)z.nitem * kNP * 8) + ws_round(n * kMaxSpace * kMaxSpace * 8) +
               ws_round(n * kYStride * 8) + ws_round(n * kNP * 8) + ws_round(8) + 2 * ws_round(n * 4);
    z.bytes += ws_round(n * sizeof(FoldDesc)) + ws_round(n * sizeof(HdiagDesc)) + psp_workspace_bytes((int)n) +
               ws_round(n * 2 * sizeof(double));
    z.bytes += ws_round((size_t)z.nitem * sizeof(int)) + ws_round((size_t)z.nitem * sizeof(long long));
    // two sigma plans (hi and lo)
    z.bytes += 2 * (ws_round(n * sizeof(SigmaProb)) + ws_round((size_t)z.n_items_sigma * sizeof(WorkItem)) +
                    2 * ws_round((size_t)z.n_tiles_sigma * sizeof(WorkItem)));
    z.bytes += 4096;
}

size_t dav_workspace_bytes(const std::vector<ProbSpec> &specs, const ifci_davidson_opts_t &o) {
    DavSizes z;
    dav_layout(specs, o, z);
    return z.bytes;
}

int hi_precision_of(const ifci_davidson_opts_t &o) {
    if (o.precision == IFCI_FP64) return IFCI_FP64;
    if (o.precision == IFCI_FP64E) return IFCI_FP64E;
    return o.hi_precision;
}

int check_opts(ifci_handle_t h, const ifci_davidson_opts_t &o) {
    if (o.hi_precision != IFCI_FP64 && o.hi_precision != IFCI_FP64E)
        return set_error(h, IFCI_ERR_INVALID_ARG, "davidson: hi_precision %d", o.hi_precision);
    if (o.precision < IFCI_FP64 || o.precision > IFCI_FP64E)
        return set_error(h, IFCI_ERR_INVALID_ARG, "davidson: precision %d", o.precision);
    if ((o.precision == IFCI_BF16 || o.precision == IFCI_TF32) && !tc_supported(o.precision))
        return set_error(h, IFCI_ERR_UNSUPPORTED, "davidson: precision %d not built", o.precision);
    if (o.max_space < 3 || o.max_space > kMaxSpace)
        return set_error(h, IFCI_ERR_INVALID_ARG, "davidson: max_space %d outside 3..%d", o.max_space, kMaxSpace);
    if (o.max_iter < 1) return set_error(h, IFCI_ERR_INVALID_ARG, "davidson: max_iter %d", o.max_iter);
    if (!(o.e_tol > 0) || !(o.r_tol > 0)) return set_error(h, IFCI_ERR_INVALID_ARG, "davidson: tolerances");
    return IFCI_OK;
}

int dav_solve(ifci_handle_t h, const std::vector<ProbSpec> &specs, const ifci_davidson_opts_t &o, double *energies,
              int *iters, int *status, cudaStream_t s, double *blk_energy) {
    const int n = (int)specs.size();
    if (n == 0) return IFCI_OK;
    IFCI_TRY(check_opts(h, o));
    DavSizes z;
    dav_layout(specs, o, z);
    const bool lo = o.precision == IFCI_FP32 || o.precision == IFCI_TF32 || o.precision == IFCI_BF16;
    const bool tc = o.precision == IFCI_BF16 || o.precision == IFCI_TF32;
    const int hi_prec = hi_precision_of(o);
    const bool oz = hi_prec == IFCI_FP64E;
    const int ms = o.max_space;

    // string tables per class
    std::map<std::pair<int, int>, std::pair<uint64_t *, int32_t *>> tables;
    std::map<std::pair<int, int>, uint8_t *> blocks;
    std::map<std::pair<int, int>, int32_t *> pmaps;
    for (const ProbSpec &p : specs) {
        auto key = std::make_pair(p.n, p.m);
        if (tables.count(key)) continue;
        int nstr = 0, nexc = 0;
        if (ifci_string_counts(p.n, p.m, &nstr, &nexc) != IFCI_OK || p.m < 1)
            return set_error(h, IFCI_ERR_INVALID_ARG, "davidson: problem with norb=%d nelec_spin=%d", p.n, p.m);
        uint64_t *st = ws_take<uint64_t>(h, nstr);
        int32_t *ex = ws_take<int32_t>(h, (size_t)nstr * nexc);
        if (!st || !ex) return set_error(h, IFCI_ERR_OOM, "davidson: workspace (strings)");
        IFCI_TRY(ifci_build_strings(h, p.n, p.m, st, ex, (ifci_stream_t)s));
        tables[key] = {st, ex};
        uint8_t *bl = ws_take<uint8_t>(h, (size_t)nstr * kBlk16Stride);
        if (!bl) return set_error(h, IFCI_ERR_OOM, "davidson: workspace (block table)");
        IFCI_TRY(launch_exc_blocks(h, nstr, nexc, ex, bl, s));
        blocks[key] = bl;
        // Davidson vectors are spin-flip symmetric: the tensor-core sigmas use
        // the alpha-only gathers where the pair map's offsets fit in int32
        int32_t *pm = nullptr;
        if ((tc || oz) && 2ll * nstr * nstr < (1ll << 31)) {
            const int np = p.n * (p.n + 1) / 2;
            pm = ws_take<int32_t>(h, (size_t)nstr * pmap_ld(np));
            if (!pm) return set_error(h, IFCI_ERR_OOM, "davidson: workspace (pair map)");
            IFCI_TRY(launch_pair_map(h, nstr, nexc, np, ex, pm, s));
        }
        pmaps[key] = pm;
    }

    DavBatch b;
    b.nprob = n;
    b.max_space = ms;
    b.keep = std::min(kKeep, ms - 2);
    b.precision = o.precision;
    b.hi_precision = hi_prec;
    b.max_iter = o.max_iter;
    b.graph_iters = o.graph_iters > 0 ? o.graph_iters : 0;
    b.e_tol = o.e_tol;
    b.r_tol = o.r_tol;
    SigmaPlan hi, lop;
    std::vector<FoldDesc> folds(n);
    std::vector<HdiagDesc> hds(n);
    std::vector<int> hw_prob;
    std::vector<long long> hw_start;
    for (int i = 0; i < n; i++) {
        const ProbSpec &p = specs[i];
        auto tb = tables[{p.n, p.m}];
        int nstr = (int)binom(p.n, p.m), nexc = p.m * (p.n - p.m + 1);
        long long ndet = (long long)nstr * nstr;
        int np = p.n * (p.n + 1) / 2;
        double *W = ws_take<double>(h, (size_t)np * np);
        float *Wf = lo ? ws_take<float>(h, (size_t)np * np) : nullptr;
        void *Wtc = tc ? (void *)ws_take<char>(h, tc_operand_bytes(np, o.precision)) : nullptr;
        char *Woz = oz ? ws_take<char>(h, oz_operand_bytes(np)) : nullptr;
        double *hd = ws_take<double>(h, ndet);
        double *B = ws_take<double>(h, (size_t)(ms + 1) * ndet);
        double *S = ws_take<double>(h, (size_t)(ms + 1) * ndet);
        if (!W || !hd || !B || !S || (lo && !Wf) || (tc && !Wtc) || (oz && !Woz))
            return set_error(h, IFCI_ERR_OOM, "davidson: workspace (problem %d)", i);
        folds[i] = FoldDesc{p.n, 2 * p.m, np, p.h1, p.eri, W};
        hds[i] = HdiagDesc{p.n, nstr, tb.first, p.h1, p.eri, hd};
        for (long long s0 = 0; s0 < ndet; s0 += kVecChunk) {
            hw_prob.push_back(i);
            hw_start.push_back(s0);
        }
        DavProb dp{};
        dp.ndet = ndet;
        dp.nstr = nstr;
        dp.item0 = (int)b.vitems.size();
        for (long long s0 = 0; s0 < ndet; s0 += kVecChunk) b.vitems.push_back(WorkItem{i, 0, s0});
        dp.nitem = (int)b.vitems.size() - dp.item0;
        dp.B = B;
        dp.S = S;
        dp.hd = hd;
        dp.c_out = p.c_out;
        dp.e_core = p.e_core;
        dp.seed_block = p.seed_block;
        b.probs.push_back(dp);
        SigmaProb sp{};
        sp.n = p.n; sp.nstr = nstr; sp.nexc = nexc; sp.np = np; sp.ld = np;
        sp.ndet = ndet; sp.stride = ndet; sp.exc = tb.second;
        sp.blk = blocks[{p.n, p.m}];
        sp.pmap = pmaps[{p.n, p.m}];
        sp.sym = sp.pmap ? 1 : 0;   // plan_sigma keeps it for the tensor-core plans only
        sp.W = W; sp.Wf = Wf; sp.Wtc = Wtc;
        sp.Woz = Woz;
        sp.Wexp = oz ? (double *)(Woz + (oz_operand_bytes(np) - np * 8 - 256)) : nullptr;
        sp.dscale = 2.0;   // basis vectors are normalised: |D| <= 2
        sp.cbase = B; sp.sbase = S;
        hi.probs.push_back(sp);
        lop.probs.push_back(sp);
    }
    b.d_probs = ws_take<DavProb>(h, n);
    b.d_state = ws_take<DavState>(h, n);
    b.d_vitems = ws_take<WorkItem>(h, b.vitems.size());
    b.d_part = ws_take<double>(h, b.vitems.size() * kNP);
    b.d_gs = ws_take<double>(h, (size_t)n * kMaxSpace * kMaxSpace);
    b.d_y = ws_take<double>(h, (size_t)n * kYStride);
    b.d_coef = ws_take<double>(h, (size_t)n * kNP);
    b.d_nactive = ws_take<int>(h, 2);
    b.d_blk_energy = ws_take<double>(h, (size_t)n * 2);
    int *d_hi = ws_take<int>(h, n), *d_lo = ws_take<int>(h, n);
    auto *d_fold = ws_take<FoldDesc>(h, n);
    auto *d_hd = ws_take<HdiagDesc>(h, n);
    int *d_hwp = ws_take<int>(h, hw_prob.size());
    long long *d_hws = ws_take<long long>(h, hw_start.size());
    void *D = ws_take<char>(h, (size_t)z.budget * 8);
    void *G = ws_take<char>(h, (size_t)z.budget * 8);
    if (!b.d_probs || !b.d_state || !b.d_vitems || !b.d_part || !b.d_gs || !b.d_y || !b.d_coef || !b.d_nactive ||
        !d_hi || !d_lo || !d_fold || !d_hd || !d_hwp || !d_hws || !D || !G)
        return set_error(h, IFCI_ERR_OOM, "davidson: workspace (batch)");
    // sigma selection flags: hi plan for FP64 sigma, lo plan for the bulk precision
    for (int i = 0; i < n; i++) {
        hi.probs[i].cslot = &b.d_state[i].newest;
        hi.probs[i].sslot = &b.d_state[i].newest;
        hi.probs[i].active = d_hi + i;
        lop.probs[i].cslot = &b.d_state[i].newest;
        lop.probs[i].sslot = &b.d_state[i].newest;
        lop.probs[i].active = d_lo + i;
    }
    IFCI_TRY(plan_sigma(h, hi, z.budget, hi_prec));
    if (lo) {
        long long budget_lo = z.budget * 8 / (long long)sigma_elem_bytes(o.precision);
        IFCI_TRY(plan_sigma(h, lop, budget_lo, o.precision));
    }
    IFCI_TRY(upload_plan(h, hi, s));
    if (lo) IFCI_TRY(upload_plan(h, lop, s));

    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_fold, folds.data(), n * sizeof(FoldDesc), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_hd, hds.data(), n * sizeof(HdiagDesc), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_hwp, hw_prob.data(), hw_prob.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_hws, hw_start.data(), hw_start.size() * sizeof(long long),
                                     cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(b.d_probs, b.probs.data(), n * sizeof(DavProb), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(b.d_vitems, b.vitems.data(), b.vitems.size() * sizeof(WorkItem),
                                     cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemsetAsync(b.d_gs, 0, (size_t)n * kMaxSpace * kMaxSpace * 8, s));
    IFCI_CUDA_TRY(h, cudaMemsetAsync(b.d_y, 0, (size_t)n * kYStride * 8, s));
    int maxnp = 0;
    for (const ProbSpec &p : specs) maxnp = std::max(maxnp, p.n * (p.n + 1) / 2);
    IFCI_TRY(launch_fold(h, n, d_fold, maxnp, s));
    if (lo) IFCI_TRY(launch_convert_w(h, n, lop.d_probs, s));
    if (tc) IFCI_TRY(launch_tc_pack_w(h, n, lop.d_probs, o.precision, s));
    if (oz) IFCI_TRY(launch_oz_pack_w(h, n, hi.d_probs, s));
    IFCI_TRY(launch_hdiag(h, d_hd, d_hwp, d_hws, (int)hw_prob.size(), kVecChunk, s));
    IFCI_TRY(dav_init(h, b, d_hd, s));

    int *h_nactive = nullptr;
    IFCI_CUDA_TRY(h, cudaMallocHost(&h_nactive, 2 * sizeof(int)));
    int st = dav_iterate(h, b, hi, lo ? &lop : nullptr, d_hi, d_lo, D, G, h_nactive, s);
    cudaFreeHost(h_nactive);
    IFCI_TRY(st);
    std::vector<DavState> hs(n);
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(hs.data(), b.d_state, n * sizeof(DavState), cudaMemcpyDeviceToHost, s));
    if (blk_energy)
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(blk_energy, b.d_blk_energy, (size_t)n * 2 * sizeof(double),
                                         cudaMemcpyDeviceToHost, s));
    IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));
    int ret = IFCI_OK;
    for (int i = 0; i < n; i++) {
        if (energies) energies[i] = hs[i].energy;
        if (iters) iters[i] = hs[i].iters;
        if (status) status[i] = hs[i].status;
        if (hs[i].status != IFCI_OK) ret = IFCI_ERR_NOT_CONVERGED;
    }
    if (ret != IFCI_OK) set_error(h, ret, "davidson: some problems did not converge");
    return ret;
}

int dav_solve_sectors(ifci_handle_t h, const std::vector<ProbSpec> &specs, const ifci_davidson_opts_t &o,
                      double *energies, int *iters, int *status, cudaStream_t s) {
    const int n = (int)specs.size();
    if (o.sector_passes < 2 || n == 0) return dav_solve(h, specs, o, energies, iters, status, s);
    const size_t mark = h->ws_top;
    std::vector<int> st_local;
    if (!status) {   // the merge needs every problem's status
        st_local.assign(n, IFCI_OK);
        status = st_local.data();
    }
    std::vector<double> blk((size_t)n * 2, 1e300);
    const int r1 = dav_solve(h, specs, o, energies, iters, status, s, blk.data());
    if (r1 != IFCI_OK && r1 != IFCI_ERR_NOT_CONVERGED) return r1;
    // second pass: problems with a competitive second block, seeded from it
    std::vector<ProbSpec> again;
    std::vector<int> who;
    std::vector<size_t> voff;
    size_t vbytes = 0;
    for (int i = 0; i < n; i++) {
        if (!(blk[2 * i + 1] < 1e299 && blk[2 * i + 1] <= blk[2 * i] + kSectorWindow)) continue;
        ProbSpec q = specs[i];
        q.seed_block = 1;
        voff.push_back(vbytes);
        if (q.c_out) vbytes += (size_t)binom(q.n, q.m) * binom(q.n, q.m) * sizeof(double);
        again.push_back(q);
        who.push_back(i);
    }
    if (again.empty()) return r1;
    double *tmp = nullptr;
    if (vbytes) IFCI_CUDA_TRY(h, cudaMalloc(&tmp, vbytes));
    for (size_t k = 0; k < again.size(); k++)
        if (again[k].c_out) again[k].c_out = reinterpret_cast<double *>(reinterpret_cast<char *>(tmp) + voff[k]);
    std::vector<double> e2(again.size());
    std::vector<int> it2(again.size()), st2(again.size());
    h->ws_top = mark;
    const int r2 = dav_solve(h, again, o, e2.data(), it2.data(), st2.data(), s);
    int ret = IFCI_OK;
    if (r2 == IFCI_OK || r2 == IFCI_ERR_NOT_CONVERGED) {
        for (size_t k = 0; k < again.size(); k++) {
            const int i = who[k];
            if (iters) iters[i] += it2[k];
            if (st2[k] == IFCI_OK && (status[i] != IFCI_OK || e2[k] < energies[i])) {
                energies[i] = e2[k];
                status[i] = IFCI_OK;
                if (specs[i].c_out) {
                    const size_t bytes = (size_t)binom(again[k].n, again[k].m) * binom(again[k].n, again[k].m) * 8;
                    if (cudaMemcpyAsync(specs[i].c_out, again[k].c_out, bytes, cudaMemcpyDeviceToDevice, s) !=
                        cudaSuccess)
                        ret = set_error(h, IFCI_ERR_CUDA, "davidson: copy of a second-pass vector");
                }
            }
        }
        if (ret == IFCI_OK)
            for (int i = 0; i < n; i++)
                if (status[i] != IFCI_OK) ret = IFCI_ERR_NOT_CONVERGED;
    } else {
        ret = r2;
    }
    if (tmp) {
        cudaStreamSynchronize(s);
        cudaFree(tmp);
    }
    if (ret == IFCI_ERR_NOT_CONVERGED) set_error(h, ret, "davidson: some problems did not converge");
    return ret;
}

}  // namespace ifci

extern "C" {

void ifci_davidson_default_opts(ifci_davidson_opts_t *o) {
    if (!o) return;
    o->precision = IFCI_FP64;
    o->max_iter = 100;
    o->max_space = 12;
    o->e_tol = 1e-10;
    o->r_tol = 1e-6;
    o->refine = 1;
    o->hi_precision = IFCI_FP64E;
    o->det_budget = 0;
    o->graph_iters = 0;
    o->sector_passes = 0;
}

int ifci_davidson_batched(ifci_handle_t h, int nprob, const ifci_problem_t *probs, const ifci_davidson_opts_t *opts,
                          double *energies, int *iters, int *status, ifci_stream_t stream) {
    using namespace ifci;
    if (!h) return IFCI_ERR_INVALID_ARG;
    if (nprob < 0 || (nprob > 0 && (!probs || !energies)))
        return set_error(h, IFCI_ERR_INVALID_ARG, "davidson_batched: bad arguments");
    ifci_davidson_opts_t o;
    ifci_davidson_default_opts(&o);
    if (opts) o = *opts;
    std::vector<ProbSpec> specs;
    for (int i = 0; i < nprob; i++) {
        const ifci_problem_t &p = probs[i];
        if (!p.h1 || !p.eri || p.nelec_spin < 1 || ifci_string_counts(p.norb, p.nelec_spin, nullptr, nullptr))
            return set_error(h, IFCI_ERR_INVALID_ARG, "davidson_batched: problem %d invalid", i);
        specs.push_back(ProbSpec{p.norb, p.nelec_spin, p.h1, p.eri, p.e_core, p.c_out});
    }
    IFCI_TRY(check_opts(h, o));
    IFCI_CUDA_TRY(h, cudaSetDevice(h->device));
    IFCI_TRY(ws_reserve(h, dav_workspace_bytes(specs, o)));
    return dav_solve_sectors(h, specs, o, energies, iters, status, as_cuda(stream));
}

}  // extern "C"
