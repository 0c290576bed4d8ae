// Host driver of the batched Davidson: sector decomposition, workspace layout,
// string tables per (norb, nelec_spin) class, folded matrices, diagonals, and
// the C entry point.
//
// A solve is organised in sigma units and Davidson problems.  A unit is one
// CI space with its own sigma build; a problem iterates in one block of a
// unit's space.  A unit whose orbitals form one coupled group has a single
// problem, the whole space.  A unit whose orbitals split into decoupled
// groups (sectors.cu) has one problem per block of H' (the distributions of
// the alpha and beta electrons among the groups, taken with their spin-flip
// images); the lowest block's vector then starts a second run with the full
// H on the whole space (the polish), whose result is the unit's answer.
#include <algorithm>
#include <cmath>
#include <map>
#include <unordered_map>

#include "dav_driver.cuh"
#include "hamiltonian.cuh"
#include "tc_gather.cuh"

namespace ifci {

int launch_convert_w(ifci_handle_t h, int nprob, const SigmaProb *d_probs, cudaStream_t s);

namespace {

// one Davidson problem of a run: a block of one unit's space
struct BlockSpec {
    int unit;
    int na, nb, sym;
    int sa_off, sb_off;      // offsets into the run's string-index list; -1: every string in order
    long long ndet, ndim;
};

// one sigma unit of a run
struct Unit {
    ProbSpec spec;           // the CI space (its integrals are the full H)
    const double *h1, *eri;  // integrals of the Hamiltonian iterated (H' for a sectored unit)
    bool sector;             // several blocks share the unit's sigma
    const double *seed;      // start vector of the whole space, or nullptr
    int prob0, nprob;
    double *expand_to;       // sectored unit: whole-space target of the lowest block's vector, or nullptr
    std::vector<int> label;  // sectored unit: group of each orbital (its FP64E contraction runs over the
                             // pairs within one group only: H' has no other integrals)
};

// Counts (count = true) or takes (count = false) workspace pieces in one order.
struct Carver {
    ifci_handle_t h;
    bool count;
    size_t total = 0;
    bool ok = true;
    template <typename T>
    T *take(size_t n) {
        if (count) {
            total += ws_round(std::max<size_t>(n, 1) * sizeof(T));
            return reinterpret_cast<T *>(alignof(T) > 256 ? alignof(T) : 256);
        }
        T *p = ws_take<T>(h, std::max<size_t>(n, 1));
        if (!p) ok = false;
        return p;
    }
};


// Runs one batch of units and their problems to convergence.  Problem
// results land in hs (DavState per problem); blk (optional) gets the two
// lowest P-space block energies per problem; sectored units with expand_to
// receive their lowest block's vector as a whole-space vector.
int dav_run(ifci_handle_t h, std::vector<Unit> &units, const std::vector<BlockSpec> &blocks,
            const std::vector<int> &sidx, const ifci_davidson_opts_t &o, cudaStream_t s, std::vector<DavState> &hs,
            std::vector<double> *blk) {
    const int nu = (int)units.size(), n = (int)blocks.size();
    const bool lo = o.precision == IFCI_FP32 || o.precision == IFCI_TF32 || o.precision == IFCI_BF16;
    const bool tc = o.precision == IFCI_BF16 || o.precision == IFCI_TF32;
    const int hi_prec = hi_precision_of(o);
    const bool oz = hi_prec == IFCI_FP64E;
    const int ms = o.max_space;

    // ---- host-side layout: string classes, vector items, hdiag work, sigma plans
    std::map<std::pair<int, int>, int> cls;
    std::vector<std::pair<int, int>> cls_keys;
    for (const Unit &u : units) {
        auto key = std::make_pair(u.spec.n, u.spec.m);
        if (!cls.count(key)) {
            int nstr = 0, nexc = 0;
            if (ifci_string_counts(u.spec.n, u.spec.m, &nstr, &nexc) != IFCI_OK || u.spec.m < 1)
                return set_error(h, IFCI_ERR_INVALID_ARG, "davidson: problem with norb=%d nelec_spin=%d", u.spec.n,
                                 u.spec.m);
            cls[key] = (int)cls_keys.size();
            cls_keys.push_back(key);
        }
    }
    DavBatch b;
    b.nprob = n;
    b.nunit = nu;
    b.max_space = ms;
    b.keep = std::min(kKeep, ms - 2);
    b.precision = o.precision;
    b.hi_precision = hi_prec;
    b.max_iter = o.max_iter;
    b.graph_iters = o.graph_iters > 0 ? o.graph_iters : 0;
    b.e_tol = o.e_tol;
    b.r_tol = o.r_tol;
    std::vector<int> item0(n), nitem(n);
    for (int i = 0; i < n; i++) {
        item0[i] = (int)b.vitems.size();
        for (long long s0 = 0; s0 < blocks[i].ndet; s0 += kVecChunk) b.vitems.push_back(WorkItem{i, 0, s0});
        nitem[i] = (int)b.vitems.size() - item0[i];
    }
    std::vector<int> hw_prob;
    std::vector<long long> hw_start;
    long long max_pd = 0, sum_pd = 0;
    SigmaPlan hi, lop;
    for (int u = 0; u < nu; u++) {
        const ProbSpec &p = units[u].spec;
        const int nstr = (int)binom(p.n, p.m), nexc = p.m * (p.n - p.m + 1), np = p.n * (p.n + 1) / 2;
        const long long ndet = (long long)nstr * nstr;
        for (long long s0 = 0; s0 < ndet; s0 += kVecChunk) {
            hw_prob.push_back(u);
            hw_start.push_back(s0);
        }
        SigmaProb sp{};
        sp.n = p.n; sp.nstr = nstr; sp.nexc = nexc; sp.np = np; sp.ld = np;
        sp.ndet = ndet; sp.stride = ndet;
        sp.sym = ((tc || oz) && 2ll * nstr * nstr < (1ll << 31)) ? 1 : 0;   // plan_sigma keeps it for tensor cores
        // a spin-symmetric FP64E problem above the budget runs in row slabs of
        // G; any other must fit one wave whole
        if (!(oz && !lo && sp.sym)) max_pd = std::max(max_pd, sigma_elems(np, ndet));
        sum_pd += sigma_elems(np, ndet);
        sp.dscale = 2.0;   // basis vectors are normalised: |D| <= 2
        hi.probs.push_back(sp);
        lop.probs.push_back(sp);
    }
    // FP64E contraction of a sectored unit over its intra-group pairs
    std::vector<std::vector<int32_t>> act(nu);
    std::vector<std::vector<uint8_t>> pact(nu);
    for (int u = 0; u < nu; u++) {
        const Unit &U = units[u];
        if (!oz || !U.sector || U.label.empty() || !hi.probs[u].sym) continue;
        const int n = U.spec.n, np = n * (n + 1) / 2;
        pact[u].assign(np, 0);
        for (int P = 0; P < n; P++)
            for (int Q = 0; Q <= P; Q++)
                if (U.label[P] == U.label[Q]) {
                    act[u].push_back(P * (P + 1) / 2 + Q);
                    pact[u][P * (P + 1) / 2 + Q] = 1;
                }
        hi.probs[u].npc = (int)act[u].size();
    }
    std::vector<size_t> act_off(nu + 1, 0), pact_off(nu + 1, 0);
    int ncompact = 0;
    for (int u = 0; u < nu; u++) {
        act_off[u + 1] = act_off[u] + act[u].size();
        pact_off[u + 1] = pact_off[u] + pact[u].size();
        if (!act[u].empty()) ncompact++;
    }
    long long budget = o.det_budget > 0 ? o.det_budget : (1ll << 31);   // two 16 GB intermediates
    budget = std::max(budget, max_pd);
    budget = std::min(budget, std::max(sum_pd, max_pd));
    for (int u = 0; u < nu; u++)   // placeholder until the device copy exists: plan_sigma tiles over npc
        if (!act[u].empty()) hi.probs[u].act = act[u].data();
    IFCI_TRY(plan_sigma(h, hi, budget, hi_prec));
    if (lo) IFCI_TRY(plan_sigma(h, lop, budget * 8 / (long long)sigma_elem_bytes(o.precision), o.precision));

    // ---- device memory, counted then taken in the same order
    struct Mem {
        std::vector<uint64_t *> st;
        std::vector<int32_t *> ex;
        std::vector<uint8_t *> bl;
        std::vector<int32_t *> pm;
        std::vector<double *> W, gc, gs;
        std::vector<float *> Wf;
        std::vector<void *> Wtc;
        std::vector<char *> Woz;
        std::vector<double *> hd, B, S, cblk;
        std::vector<int32_t *> act, pmapc;
        std::vector<uint8_t *> pact;
        int32_t *act_all = nullptr;
        uint8_t *pact_all = nullptr;
        CompactDesc *cdesc = nullptr;
        int *sidx = nullptr;
        DavProb *probs = nullptr;
        DavState *state = nullptr;
        WorkItem *vitems = nullptr;
        double *part = nullptr, *gsm = nullptr, *y = nullptr, *coef = nullptr, *blk = nullptr;
        int *nactive = nullptr, *dhi = nullptr, *dlo = nullptr;
        int2 *urange = nullptr;
        int *uhi = nullptr, *ulo = nullptr;
        FoldDesc *fold = nullptr;
        HdiagDesc *hdu = nullptr, *hdp = nullptr;
        int *hwp = nullptr;
        long long *hws = nullptr;
        double **dst = nullptr;
        void *D = nullptr, *G = nullptr;
        SigmaProb *hi_p = nullptr, *lo_p = nullptr;
        WorkItem *hi_i = nullptr, *hi_t = nullptr, *hi_c = nullptr, *lo_i = nullptr, *lo_t = nullptr, *lo_c = nullptr;
        long long *pidx = nullptr;
        int *pcount = nullptr;
    };
    auto carve = [&](Carver &c, Mem &m) {
        const int nc = (int)cls_keys.size();
        m.st.resize(nc); m.ex.resize(nc); m.bl.resize(nc); m.pm.assign(nc, nullptr);
        for (int k = 0; k < nc; k++) {
            const int nn = cls_keys[k].first, mm = cls_keys[k].second;
            const int nstr = (int)binom(nn, mm), nexc = mm * (nn - mm + 1), np = nn * (nn + 1) / 2;
            m.st[k] = c.take<uint64_t>(nstr);
            m.ex[k] = c.take<int32_t>((size_t)nstr * nexc);
            m.bl[k] = c.take<uint8_t>((size_t)nstr * kBlk16Stride);
            // Davidson vectors are spin-flip symmetric: the tensor-core sigmas use
            // the alpha-only gathers where the pair map's offsets fit in int32
            if ((tc || oz) && 2ll * nstr * nstr < (1ll << 31)) m.pm[k] = c.take<int32_t>((size_t)nstr * pmap_ld(np));
        }
        // active pairs of every sectored unit in one array each (one copy, one
        // compaction launch for all units)
        m.act.assign(nu, nullptr); m.pmapc.assign(nu, nullptr); m.pact.assign(nu, nullptr);
        m.act_all = c.take<int32_t>(act_off.back());
        m.pact_all = c.take<uint8_t>(pact_off.back());
        m.cdesc = c.take<CompactDesc>(ncompact);
        for (int u = 0; u < nu; u++) {
            if (act[u].empty()) continue;
            const int nstr = (int)binom(units[u].spec.n, units[u].spec.m);
            if (!c.count) {
                m.act[u] = m.act_all + act_off[u];
                m.pact[u] = m.pact_all + pact_off[u];
            }
            m.pmapc[u] = c.take<int32_t>((size_t)nstr * pmap_ld((int)act[u].size()));
        }
        m.W.resize(nu); m.Wf.assign(nu, nullptr); m.Wtc.assign(nu, nullptr); m.Woz.assign(nu, nullptr);
        m.gc.assign(nu, nullptr); m.gs.assign(nu, nullptr);
        for (int u = 0; u < nu; u++) {
            const ProbSpec &p = units[u].spec;
            const int np = p.n * (p.n + 1) / 2;
            const long long ndet = binom(p.n, p.m) * binom(p.n, p.m);
            m.W[u] = c.take<double>((size_t)np * np);
            if (lo) m.Wf[u] = c.take<float>((size_t)np * np);
            if (tc) m.Wtc[u] = c.take<char>(tc_operand_bytes(np, o.precision));
            if (oz) m.Woz[u] = c.take<char>(oz_operand_bytes(np));
            if (units[u].sector) {
                m.gc[u] = c.take<double>(ndet);
                m.gs[u] = c.take<double>(ndet);
            }
        }
        m.hd.resize(n); m.B.resize(n); m.S.resize(n); m.cblk.assign(n, nullptr);
        for (int i = 0; i < n; i++) {
            const long long nd = blocks[i].ndet;
            m.hd[i] = c.take<double>(nd);
            m.B[i] = c.take<double>((size_t)(ms + 1) * nd);
            m.S[i] = c.take<double>((size_t)(ms + 1) * nd);
            if (units[blocks[i].unit].sector && units[blocks[i].unit].expand_to) m.cblk[i] = c.take<double>(nd);
        }
        m.sidx = c.take<int>(sidx.size());
        m.probs = c.take<DavProb>(n);
        m.state = c.take<DavState>(n);
        m.vitems = c.take<WorkItem>(b.vitems.size());
        m.part = c.take<double>(b.vitems.size() * kNP);
        m.gsm = c.take<double>((size_t)n * kMaxSpace * kMaxSpace);
        m.y = c.take<double>((size_t)n * kYStride);
        m.coef = c.take<double>((size_t)n * kNP);
        m.nactive = c.take<int>(2);
        m.blk = c.take<double>((size_t)n * 2);
        m.dhi = c.take<int>(n);
        m.dlo = c.take<int>(n);
        m.urange = c.take<int2>(nu);
        m.uhi = c.take<int>(nu);
        m.ulo = c.take<int>(nu);
        m.fold = c.take<FoldDesc>(nu);
        m.hdu = c.take<HdiagDesc>(nu);
        m.hdp = c.take<HdiagDesc>(n);
        m.hwp = c.take<int>(hw_prob.size());
        m.hws = c.take<long long>(hw_start.size());
        m.dst = c.take<double *>(n);
        // D holds the gathered intermediate on the CUDA-core paths, only the
        // quantised copies of c on the FP64-emulating one
        m.D = c.take<char>((size_t)((hi_prec == IFCI_FP64E && !lo) ? std::max(hi.max_qelems, 1ll)
                                                                     : std::max(budget, hi.max_qelems)) * 8);
        m.G = c.take<char>((size_t)budget * 8);
        m.hi_p = c.take<SigmaProb>(hi.probs.size());
        m.hi_i = c.take<WorkItem>(hi.items.size());
        m.hi_t = c.take<WorkItem>(hi.tiles.size());
        m.hi_c = c.take<WorkItem>(hi.tctiles.size());
        if (lo) {
            m.lo_p = c.take<SigmaProb>(lop.probs.size());
            m.lo_i = c.take<WorkItem>(lop.items.size());
            m.lo_t = c.take<WorkItem>(lop.tiles.size());
            m.lo_c = c.take<WorkItem>(lop.tctiles.size());
        }
        m.pidx = c.take<long long>((size_t)n * kPspMax);
        m.pcount = c.take<int>(n);
    };
    Mem mem;
    {
        Carver cnt{h, true};
        carve(cnt, mem);
        IFCI_TRY(ws_reserve(h, cnt.total + 4096));
    }
    Carver real{h, false};
    carve(real, mem);
    if (!real.ok) return set_error(h, IFCI_ERR_OOM, "davidson: workspace");

    // ---- string tables
    for (size_t k = 0; k < cls_keys.size(); k++) {
        const int nn = cls_keys[k].first, mm = cls_keys[k].second;
        const int nstr = (int)binom(nn, mm), nexc = mm * (nn - mm + 1), np = nn * (nn + 1) / 2;
        IFCI_TRY(ifci_build_strings(h, nn, mm, mem.st[k], mem.ex[k], (ifci_stream_t)s));
        IFCI_TRY(launch_exc_blocks(h, nstr, nexc, mem.ex[k], mem.bl[k], s));
        if (mem.pm[k]) IFCI_TRY(launch_pair_map(h, nstr, nexc, np, mem.ex[k], mem.pm[k], s));
    }

    // ---- descriptors
    std::vector<FoldDesc> folds(nu);
    std::vector<HdiagDesc> hdu(nu), hdp(n);
    std::vector<int2> urange(nu);
    for (int u = 0; u < nu; u++) {
        const Unit &U = units[u];
        const ProbSpec &p = U.spec;
        const int k = cls[{p.n, p.m}];
        const int nstr = (int)binom(p.n, p.m);
        const int np = p.n * (p.n + 1) / 2;
        folds[u] = FoldDesc{p.n, 2 * p.m, np, U.h1, U.eri, mem.W[u]};
        // whole-space diagonal: straight into the single problem's hd, or into gs
        // (then gathered per block)
        hdu[u] = HdiagDesc{p.n, nstr, mem.st[k], U.h1, U.eri, U.sector ? mem.gs[u] : mem.hd[U.prob0]};
        urange[u] = make_int2(U.prob0, U.nprob);
        for (SigmaPlan *pl : {&hi, &lop}) {
            SigmaProb &sp = pl->probs[u];
            sp.exc = mem.ex[k];
            sp.blk = mem.bl[k];
            sp.pmap = mem.pm[k];
            if (!sp.pmap) sp.sym = 0;
            sp.W = mem.W[u]; sp.Wf = mem.Wf[u]; sp.Wtc = mem.Wtc[u];
            sp.Woz = mem.Woz[u];
            sp.Wexp = oz ? (double *)(mem.Woz[u] + (oz_operand_bytes(np) - np * 8 - 256)) : nullptr;
            if (U.sector) {
                sp.cbase = mem.gc[u]; sp.sbase = mem.gs[u];
                sp.cslot = nullptr; sp.sslot = nullptr;
            } else {
                sp.cbase = mem.B[U.prob0]; sp.sbase = mem.S[U.prob0];
                sp.cslot = &mem.state[U.prob0].newest;
                sp.sslot = &mem.state[U.prob0].newest;
            }
            sp.active = (pl == &hi ? mem.uhi : mem.ulo) + u;
            if (pl == &hi && mem.act[u]) {
                sp.act = mem.act[u];
                sp.pact = mem.pact[u];
                sp.pmapc = mem.pmapc[u];
            } else {
                sp.act = nullptr;
                sp.pact = nullptr;
                sp.pmapc = nullptr;
                sp.npc = sp.np;
            }
        }
    }
    for (int i = 0; i < n; i++) {
        const BlockSpec &bs = blocks[i];
        const Unit &U = units[bs.unit];
        const ProbSpec &p = U.spec;
        const int k = cls[{p.n, p.m}];
        DavProb dp{};
        dp.ndet = bs.ndet;
        dp.ndim = bs.ndim;
        dp.nstr = (int)binom(p.n, p.m);
        dp.na = bs.na;
        dp.nb = bs.nb;
        dp.sym = bs.sym;
        dp.item0 = item0[i];
        dp.nitem = nitem[i];
        dp.seed_block = p.seed_block;
        dp.sa = bs.sa_off >= 0 ? mem.sidx + bs.sa_off : nullptr;
        dp.sb = bs.sb_off >= 0 ? mem.sidx + bs.sb_off : nullptr;
        dp.B = mem.B[i];
        dp.S = mem.S[i];
        dp.hd = mem.hd[i];
        dp.c_out = U.sector ? mem.cblk[i] : p.c_out;
        dp.seed = U.seed;
        dp.mask = U.sector ? nullptr : p.mask;
        dp.gc = U.sector ? mem.gc[bs.unit] : nullptr;
        dp.gs = U.sector ? mem.gs[bs.unit] : nullptr;
        dp.e_core = p.e_core;
        b.probs.push_back(dp);
        hdp[i] = HdiagDesc{p.n, dp.nstr, mem.st[k], U.h1, U.eri, mem.hd[i]};
    }
    b.d_probs = mem.probs;
    b.d_state = mem.state;
    b.d_vitems = mem.vitems;
    b.d_part = mem.part;
    b.d_gs = mem.gsm;
    b.d_y = mem.y;
    b.d_coef = mem.coef;
    b.d_nactive = mem.nactive;
    b.d_blk_energy = mem.blk;
    b.d_urange = mem.urange;
    b.d_uhi = mem.uhi;
    b.d_ulo = mem.ulo;
    b.any_sector = false;
    b.any_mask = false;
    for (const Unit &U : units) {
        b.any_sector = b.any_sector || U.sector;
        b.any_mask = b.any_mask || (!U.sector && U.spec.mask);
    }
    hi.d_probs = mem.hi_p; hi.d_items = mem.hi_i; hi.d_tiles = mem.hi_t; hi.d_tctiles = mem.hi_c;
    IFCI_TRY(upload_plan_to(h, hi, s));
    if (lo) {
        lop.d_probs = mem.lo_p; lop.d_items = mem.lo_i; lop.d_tiles = mem.lo_t; lop.d_tctiles = mem.lo_c;
        IFCI_TRY(upload_plan_to(h, lop, s));
    }
    if (!sidx.empty())
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(mem.sidx, sidx.data(), sidx.size() * 4, cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(mem.fold, folds.data(), nu * sizeof(FoldDesc), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(mem.hdu, hdu.data(), nu * sizeof(HdiagDesc), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(mem.hdp, hdp.data(), n * sizeof(HdiagDesc), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(mem.urange, urange.data(), nu * sizeof(int2), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(mem.hwp, hw_prob.data(), hw_prob.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(mem.hws, hw_start.data(), hw_start.size() * sizeof(long long),
                                     cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(b.d_probs, b.probs.data(), n * sizeof(DavProb), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(b.d_vitems, b.vitems.data(), b.vitems.size() * sizeof(WorkItem),
                                     cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemsetAsync(b.d_gs, 0, (size_t)n * kMaxSpace * kMaxSpace * 8, s));
    IFCI_CUDA_TRY(h, cudaMemsetAsync(b.d_y, 0, (size_t)n * kYStride * 8, s));
    if (ncompact > 0) {
        std::vector<int32_t> act_h(act_off.back());
        std::vector<uint8_t> pact_h(pact_off.back());
        std::vector<CompactDesc> cd;
        for (int u = 0; u < nu; u++) {
            if (!mem.act[u]) continue;
            std::copy(act[u].begin(), act[u].end(), act_h.begin() + act_off[u]);
            std::copy(pact[u].begin(), pact[u].end(), pact_h.begin() + pact_off[u]);
            const int k = cls[{units[u].spec.n, units[u].spec.m}];
            const int nstr = (int)binom(units[u].spec.n, units[u].spec.m), np = units[u].spec.n * (units[u].spec.n + 1) / 2;
            cd.push_back(CompactDesc{nstr, pmap_ld(np), (int)act[u].size(), pmap_ld((int)act[u].size()), mem.pm[k],
                                     mem.act[u], mem.pmapc[u]});
        }
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(mem.act_all, act_h.data(), act_h.size() * 4, cudaMemcpyHostToDevice, s));
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(mem.pact_all, pact_h.data(), pact_h.size(), cudaMemcpyHostToDevice, s));
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(mem.cdesc, cd.data(), cd.size() * sizeof(CompactDesc), cudaMemcpyHostToDevice, s));
        IFCI_TRY(launch_compact_pair_maps(h, (int)cd.size(), mem.cdesc, s));
    }
    {
        ProfScope ps(h, s, PK_SETUP);
        int maxnp = 0;
        for (const Unit &U : units) maxnp = std::max(maxnp, U.spec.n * (U.spec.n + 1) / 2);
        IFCI_TRY(launch_fold(h, nu, mem.fold, maxnp, s));
        if (lo) IFCI_TRY(launch_convert_w(h, nu, lop.d_probs, s));
        if (tc) IFCI_TRY(launch_tc_pack_w(h, nu, lop.d_probs, o.precision, s));
        if (oz) IFCI_TRY(launch_oz_pack_w(h, nu, hi.d_probs, s));
        IFCI_TRY(launch_hdiag(h, mem.hdu, mem.hwp, mem.hws, (int)hw_prob.size(), kVecChunk, s));
        if (b.any_sector) IFCI_TRY(launch_sector_hd(h, b, s));
        b.d_pidx = mem.pidx;
        b.d_pcount = mem.pcount;
    }
    IFCI_TRY(dav_init(h, b, mem.hdp, s));

    int *h_nactive = nullptr;
    IFCI_CUDA_TRY(h, cudaMallocHost(&h_nactive, 2 * sizeof(int)));
    int st = dav_iterate(h, b, hi, lo ? &lop : nullptr, mem.dhi, mem.dlo, mem.D, mem.G, h_nactive, s);
    cudaFreeHost(h_nactive);
    IFCI_TRY(st);
    hs.resize(n);
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(hs.data(), b.d_state, n * sizeof(DavState), cudaMemcpyDeviceToHost, s));
    if (blk) {
        blk->assign((size_t)n * 2, 1e300);
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(blk->data(), b.d_blk_energy, (size_t)n * 2 * sizeof(double),
                                         cudaMemcpyDeviceToHost, s));
    }
    IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));
    // lowest block of every sectored unit -> whole-space vector
    if (b.any_sector) {
        std::vector<double *> dst(n, nullptr);
        bool any = false;
        for (int u = 0; u < nu; u++) {
            const Unit &U = units[u];
            if (!U.sector || !U.expand_to) continue;
            int best = U.prob0;
            for (int i = U.prob0; i < U.prob0 + U.nprob; i++)
                if (hs[i].energy < hs[best].energy) best = i;
            dst[best] = U.expand_to;
            const long long ndet = binom(U.spec.n, U.spec.m) * binom(U.spec.n, U.spec.m);
            IFCI_CUDA_TRY(h, cudaMemsetAsync(U.expand_to, 0, (size_t)ndet * 8, s));
            any = true;
        }
        if (any) {
            IFCI_CUDA_TRY(h, cudaMemcpyAsync(mem.dst, dst.data(), n * sizeof(double *), cudaMemcpyHostToDevice, s));
            IFCI_TRY(launch_sector_expand(h, b, mem.dst, s));
            IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));
        }
    }
    return IFCI_OK;
}

}  // namespace

// Every m-electron string of n orbitals, ascending as bit masks.
std::vector<uint32_t> host_strings(int n, int m) {
    std::vector<uint32_t> out;
    uint64_t v = (1ull << m) - 1ull;
    const uint64_t lim = 1ull << n;
    while (v < lim) {
        out.push_back((uint32_t)v);
        const uint64_t t = v | (v - 1);
        v = (t + 1) | (((~t & (t + 1)) - 1) >> (__builtin_ctzll(v) + 1));
    }
    return out;
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
    if (!(o.decouple_tol >= 0)) return set_error(h, IFCI_ERR_INVALID_ARG, "davidson: decouple_tol");
    if (o.hbci_max_rounds < 0 || !(o.hbci_eps1 >= 0) || !(o.hbci_eps2 >= 0))
        return set_error(h, IFCI_ERR_INVALID_ARG, "davidson: hbci_max_rounds >= 0, hbci_eps1/2 >= 0 required");
    return IFCI_OK;
}

int dav_solve(ifci_handle_t h, const std::vector<ProbSpec> &specs, const ifci_davidson_opts_t &o, double *energies,
              int *iters, int *status, cudaStream_t s, double *blk_energy) {
    const int nspec = (int)specs.size();
    if (nspec == 0) return IFCI_OK;
    IFCI_TRY(check_opts(h, o));
    DavArena arena(h);   // every piece below comes from the Davidson workspace

    // ---- orbital groups of every problem (coupling graph above decouple_tol)
    std::vector<std::vector<int>> label(nspec);
    std::vector<int> ngroup(nspec, 1);
    if (o.decouple_tol > 0) {
        std::vector<CoupDesc> cd(nspec);
        for (int i = 0; i < nspec; i++) cd[i] = CoupDesc{specs[i].n, specs[i].h1, specs[i].eri};
        IFCI_TRY(ws_reserve(h, ws_round(nspec * sizeof(CoupDesc)) + ws_round((size_t)nspec * 32 * 4) + 1024));
        auto *d_cd = ws_take<CoupDesc>(h, nspec);
        auto *d_adj = ws_take<uint32_t>(h, (size_t)nspec * 32);
        if (!d_cd || !d_adj) return set_error(h, IFCI_ERR_OOM, "davidson: workspace (coupling)");
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_cd, cd.data(), nspec * sizeof(CoupDesc), cudaMemcpyHostToDevice, s));
        IFCI_TRY(launch_coupling(h, nspec, d_cd, o.decouple_tol, d_adj, s));
        std::vector<uint32_t> adj((size_t)nspec * 32);
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(adj.data(), d_adj, adj.size() * 4, cudaMemcpyDeviceToHost, s));
        IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));
        for (int i = 0; i < nspec; i++) orbital_groups(adj.data() + (size_t)i * 32, specs[i].n, label[i], ngroup[i]);
    }

    // ---- blocks of the sectored problems
    std::vector<Unit> units;
    std::vector<BlockSpec> blocks;
    std::vector<int> sidx;
    std::vector<int> sectored;   // spec indices with more than one group
    for (int i = 0; i < nspec; i++) {
        const ProbSpec &p = specs[i];
        const int nstr = (int)binom(p.n, p.m);
        Unit U{p, p.h1, p.eri, false, p.seed, (int)blocks.size(), 1, nullptr};
        if (ngroup[i] > 1 && ngroup[i] <= 16 && p.m >= 1 && !p.mask) {
            // class of a string = electrons per group, 4 bits per group
            std::vector<uint32_t> gmask(ngroup[i], 0u);
            for (int q = 0; q < p.n; q++) gmask[label[i][q]] |= 1u << q;
            const std::vector<uint32_t> strs = host_strings(p.n, p.m);
            std::unordered_map<uint64_t, int> cid;
            std::vector<std::vector<int>> members;
            for (int si = 0; si < nstr; si++) {
                uint64_t key = 0;
                for (int g = 0; g < ngroup[i]; g++) key |= (uint64_t)__builtin_popcount(strs[si] & gmask[g]) << (4 * g);
                auto it = cid.find(key);
                if (it == cid.end()) {
                    it = cid.emplace(key, (int)members.size()).first;
                    members.emplace_back();
                }
                members[it->second].push_back(si);
            }
            if (members.size() > 1) {
                std::vector<int> off(members.size());
                for (size_t a = 0; a < members.size(); a++) {
                    off[a] = (int)sidx.size();
                    sidx.insert(sidx.end(), members[a].begin(), members[a].end());
                }
                U.sector = true;
                U.nprob = 0;
                for (size_t a = 0; a < members.size(); a++)
                    for (size_t c = a; c < members.size(); c++) {
                        BlockSpec bs{};
                        bs.unit = (int)units.size();
                        bs.na = (int)members[a].size();
                        bs.nb = (int)members[c].size();
                        bs.sym = a == c;
                        bs.sa_off = off[a];
                        bs.sb_off = off[c];
                        bs.ndet = (long long)bs.na * bs.nb;
                        bs.ndim = bs.sym ? (long long)bs.na * (bs.na + 1) / 2 : bs.ndet;
                        blocks.push_back(bs);
                        U.nprob++;
                    }
                sectored.push_back(i);
            }
        }
        if (!U.sector) {
            BlockSpec bs{};
            bs.unit = (int)units.size();
            bs.na = bs.nb = nstr;
            bs.sym = 1;
            bs.sa_off = bs.sb_off = -1;
            bs.ndet = (long long)nstr * nstr;
            bs.ndim = p.ndim > 0 ? p.ndim : (long long)nstr * (nstr + 1) / 2;
            blocks.push_back(bs);
        }
        units.push_back(U);
    }

    // ---- H' of the sectored problems and the whole-space start vectors of the polish
    double *scratch = nullptr;   // [masked h1, masked eri] per sectored problem, then seeds
    std::vector<double *> seeds(nspec, nullptr);
    std::vector<int> polished;   // sectored problems whose dropped integrals are not negligible
    if (!sectored.empty()) {
        size_t bytes = 0;
        for (int i : sectored) {
            const long long np = specs[i].n * (specs[i].n + 1) / 2, nstr = binom(specs[i].n, specs[i].m);
            bytes += ws_round((size_t)specs[i].n * specs[i].n * 8) + ws_round((size_t)np * np * 8);
            if (!specs[i].c_out) bytes += ws_round((size_t)nstr * nstr * 8);
        }
        bytes += ws_round(sectored.size() * sizeof(double));
        IFCI_CUDA_TRY(h, cudaMalloc(&scratch, bytes + ws_round(sectored.size() * sizeof(MaskDesc))));
        char *q = reinterpret_cast<char *>(scratch);
        double *d_dropped = reinterpret_cast<double *>(q);
        q += ws_round(sectored.size() * sizeof(double));
        std::vector<MaskDesc> md;
        for (int i : sectored) {
            const long long np = specs[i].n * (specs[i].n + 1) / 2, nstr = binom(specs[i].n, specs[i].m);
            MaskDesc d{};
            d.n = specs[i].n;
            d.h1 = specs[i].h1;
            d.eri = specs[i].eri;
            d.h1m = reinterpret_cast<double *>(q);
            q += ws_round((size_t)specs[i].n * specs[i].n * 8);
            d.erim = reinterpret_cast<double *>(q);
            q += ws_round((size_t)np * np * 8);
            for (int p = 0; p < 32; p++) d.label[p] = p < specs[i].n ? (unsigned char)label[i][p] : 0;
            d.dropped = d_dropped + md.size();
            if (specs[i].c_out) {
                seeds[i] = specs[i].c_out;   // the polish copies its start vector before it writes c_out
            } else {
                seeds[i] = reinterpret_cast<double *>(q);
                q += ws_round((size_t)nstr * nstr * 8);
            }
            units[i].h1 = d.h1m;
            units[i].eri = d.erim;
            units[i].label = label[i];
            md.push_back(d);
        }
        auto *d_md = reinterpret_cast<MaskDesc *>(q);
        std::vector<double> dropped(sectored.size(), 0.0);
        int rc = IFCI_OK;
        if (cudaMemcpyAsync(d_md, md.data(), md.size() * sizeof(MaskDesc), cudaMemcpyHostToDevice, s) != cudaSuccess)
            rc = set_error(h, IFCI_ERR_CUDA, "davidson: mask descriptors");
        if (rc == IFCI_OK) rc = launch_mask(h, (int)md.size(), d_md, s);
        if (rc == IFCI_OK && (cudaMemcpyAsync(dropped.data(), d_dropped, dropped.size() * 8, cudaMemcpyDeviceToHost,
                                              s) != cudaSuccess ||
                              cudaStreamSynchronize(s) != cudaSuccess))
            rc = set_error(h, IFCI_ERR_CUDA, "davidson: dropped integrals");
        if (rc != IFCI_OK) {
            cudaStreamSynchronize(s);
            cudaFree(scratch);
            return rc;
        }
        // H - H' below kPolishTol everywhere: the lowest block's eigenpair is the
        // eigenpair of H to far below any tolerance (second order in H - H'), and
        // its vector is the result; otherwise the polish refines it with the full H
        for (size_t k = 0; k < sectored.size(); k++) {
            const int i = sectored[k];
            if (dropped[k] > kPolishTol) {
                polished.push_back(i);
                units[i].expand_to = seeds[i];
            } else if (specs[i].c_out) {
                units[i].expand_to = specs[i].c_out;
            }
        }
    }

    // ---- the run over every unit; then the polish of the sectored ones
    std::vector<DavState> hs;
    std::vector<double> blk;
    int rc = dav_run(h, units, blocks, sidx, o, s, hs, blk_energy ? &blk : nullptr);
    std::vector<DavState> hp;
    if (rc == IFCI_OK && !polished.empty()) {
        std::vector<Unit> pu;
        std::vector<BlockSpec> pb;
        for (int i : polished) {
            const ProbSpec &p = specs[i];
            const int nstr = (int)binom(p.n, p.m);
            Unit U{p, p.h1, p.eri, false, seeds[i], (int)pb.size(), 1, nullptr};
            U.spec.seed_block = 0;
            BlockSpec bs{};
            bs.unit = (int)pu.size();
            bs.na = bs.nb = nstr;
            bs.sym = 1;
            bs.sa_off = bs.sb_off = -1;
            bs.ndet = (long long)nstr * nstr;
            bs.ndim = (long long)nstr * (nstr + 1) / 2;
            pb.push_back(bs);
            pu.push_back(U);
        }
        ifci_davidson_opts_t op = o;
        op.sector_passes = 0;
        rc = dav_run(h, pu, pb, std::vector<int>(), op, s, hp, nullptr);
    }
    if (scratch) {
        cudaStreamSynchronize(s);
        cudaFree(scratch);
    }
    IFCI_TRY(rc);

    // ---- per problem: the lowest block (then its polish) for sectored problems
    int ret = IFCI_OK;
    std::vector<int> polish_of(nspec, -1);
    for (size_t k = 0; k < polished.size(); k++) polish_of[polished[k]] = (int)k;
    for (int i = 0; i < nspec; i++) {
        const Unit &U = units[i];
        int best = U.prob0, it = 0, stt = IFCI_OK;
        for (int j = U.prob0; j < U.prob0 + U.nprob; j++) {
            if (hs[j].energy < hs[best].energy) best = j;
            it = std::max(it, hs[j].iters);
            if (hs[j].status != IFCI_OK) stt = hs[j].status;
        }
        double e = hs[best].energy;
        if (polish_of[i] >= 0) {
            const DavState &q = hp[polish_of[i]];
            e = q.energy;
            it += q.iters;
            if (q.status != IFCI_OK) stt = q.status;
        }
        if (energies) energies[i] = e;
        if (iters) iters[i] = it;
        if (status) status[i] = stt;
        if (blk_energy) {
            blk_energy[2 * i] = blk[2 * best];
            blk_energy[2 * i + 1] = blk[2 * best + 1];
        }
        if (stt != IFCI_OK) ret = IFCI_ERR_NOT_CONVERGED;
    }
    if (ret != IFCI_OK) set_error(h, ret, "davidson: some problems did not converge");
    return ret;
}

int dav_solve_sectors(ifci_handle_t h, const std::vector<ProbSpec> &specs, const ifci_davidson_opts_t &o,
                      double *energies, int *iters, int *status, cudaStream_t s) {
    const int n = (int)specs.size();
    if (o.sector_passes < 2 || n == 0) return dav_solve(h, specs, o, energies, iters, status, s);
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
    o->decouple_tol = 1e-5;
    o->cnb_threshold = 0.0;
    o->hbci_max_rounds = 0;
    o->hbci_eps1 = 1e-3;
    o->hbci_eps2 = 1e-6;
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
    return dav_solve_sectors(h, specs, o, energies, iters, status, as_cuda(stream));
}

}  // extern "C"
