// C entry points for single CI spaces: ifci_sigma and ifci_frozen_core.
#include <algorithm>

#include "hamiltonian.cuh"
#include "sigma.cuh"

namespace ifci {
int launch_convert_w(ifci_handle_t h, int nprob, const SigmaProb *d_probs, cudaStream_t s);
}

extern "C" {

int ifci_sigma(ifci_handle_t h, const ifci_strings_t *str, const double *h1, const double *eri, const double *c,
               double *sigma, int precision, ifci_stream_t stream) {
    using namespace ifci;
    if (!h) return IFCI_ERR_INVALID_ARG;
    if (!str || !h1 || !eri || !c || !sigma || !str->exc)
        return set_error(h, IFCI_ERR_INVALID_ARG, "ifci_sigma: null argument");
    int nstr = 0, nexc = 0;
    if (ifci_string_counts(str->norb, str->nelec_spin, &nstr, &nexc) != IFCI_OK || nstr != str->nstr ||
        nexc != str->nexc || str->nelec_spin < 1)
        return set_error(h, IFCI_ERR_INVALID_ARG, "ifci_sigma: inconsistent string table (norb=%d nelec=%d)",
                         str->norb, str->nelec_spin);
    if (c == sigma) return set_error(h, IFCI_ERR_INVALID_ARG, "ifci_sigma: sigma aliases c");
    const bool sym_req = (precision & IFCI_SIGMA_SPIN_SYMMETRIC) != 0;
    precision &= ~IFCI_SIGMA_SPIN_SYMMETRIC;
    if (precision < IFCI_FP64 || precision > IFCI_FP64E)
        return set_error(h, IFCI_ERR_INVALID_ARG, "ifci_sigma: precision %d", precision);
    const bool tc = precision == IFCI_BF16 || precision == IFCI_TF32;
    const bool oz = precision == IFCI_FP64E;
    if (tc && !tc_supported(precision))
        return set_error(h, IFCI_ERR_UNSUPPORTED, "ifci_sigma: precision %d not built", precision);
    IFCI_CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = as_cuda(stream);
    const int n = str->norb, np = n * (n + 1) / 2, ld = np;
    const long long ndet = (long long)nstr * nstr;

    SigmaPlan plan;
    SigmaProb p{};
    p.n = n; p.nstr = nstr; p.nexc = nexc; p.np = np; p.ld = ld;
    p.ndet = ndet; p.stride = ndet; p.exc = str->exc;
    p.cbase = c; p.sbase = sigma;
    const bool sym = sym_req && (tc || oz) && 2 * ndet < (1ll << 31);
    p.sym = sym ? 1 : 0;   // the pair map is placed below, before the plan is uploaded
    plan.probs.push_back(p);
    // one wave; a spin-symmetric FP64E problem above 2^31 G elements runs in row slabs
    const long long whole = sigma_elems(np, ndet);
    IFCI_TRY(plan_sigma(h, plan, (oz && sym) ? std::min(whole, kSigmaSlabBudget) : whole, precision));
    const size_t eb = sigma_elem_bytes(precision);
    const long long delems_D = std::max(plan.max_delems, plan.max_qelems);
    size_t need = ws_round(sizeof(FoldDesc)) + ws_round((size_t)ld * ld * 8) + ws_round((size_t)ld * ld * 4) +
                  (tc ? ws_round((size_t)tc_operand_bytes(np, precision)) : 0) +
                  (oz ? ws_round((size_t)oz_operand_bytes(np)) + ws_round(8) : 0) +
                  ((tc || oz) ? ws_round((size_t)nstr * kBlk16Stride) : 0) +
                  (sym ? ws_round((size_t)nstr * pmap_ld(np) * 4) : 0) + plan_device_bytes(plan) +
                  ws_round((size_t)delems_D * eb) + ws_round((size_t)plan.max_delems * eb);
    IFCI_TRY(ws_reserve(h, need));
    auto *fd = ws_take<FoldDesc>(h, 1);
    double *W = ws_take<double>(h, (size_t)ld * ld);
    float *Wf = ws_take<float>(h, (size_t)ld * ld);
    void *Wtc = tc ? (void *)ws_take<char>(h, tc_operand_bytes(np, precision)) : nullptr;
    char *Woz = oz ? ws_take<char>(h, oz_operand_bytes(np)) : nullptr;
    plan.probs[0].W = W;
    plan.probs[0].Wf = Wf;
    plan.probs[0].Wtc = Wtc;
    plan.probs[0].Woz = Woz;
    plan.probs[0].Wexp = oz ? (double *)(Woz + (oz_operand_bytes(np) - np * 8 - 256)) : nullptr;
    plan.probs[0].dscale = 2.0;
    uint8_t *blk = (tc || oz) ? ws_take<uint8_t>(h, (size_t)nstr * kBlk16Stride) : nullptr;
    plan.probs[0].blk = blk;
    int32_t *pmap = sym ? ws_take<int32_t>(h, (size_t)nstr * pmap_ld(np)) : nullptr;
    plan.probs[0].pmap = pmap;
    FoldDesc f{n, 2 * str->nelec_spin, ld, h1, eri, W};
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(fd, &f, sizeof(f), cudaMemcpyHostToDevice, s));
    IFCI_TRY(launch_fold(h, 1, fd, np, s));
    if (blk) IFCI_TRY(launch_exc_blocks(h, nstr, nexc, str->exc, blk, s));
    if (pmap) IFCI_TRY(launch_pair_map(h, nstr, nexc, np, str->exc, pmap, s));
    IFCI_TRY(upload_plan(h, plan, s));
    if (precision == IFCI_FP32) IFCI_TRY(launch_convert_w(h, 1, plan.d_probs, s));
    if (tc) IFCI_TRY(launch_tc_pack_w(h, 1, plan.d_probs, precision, s));
    if (oz) {
        IFCI_TRY(launch_oz_pack_w(h, 1, plan.d_probs, s));
        IFCI_TRY(launch_oz_dscale(h, plan.d_probs, c, ndet, s));
    }
    void *D = ws_take<char>(h, (size_t)delems_D * eb);
    void *G = ws_take<char>(h, (size_t)plan.max_delems * eb);
    if (!D || !G) return set_error(h, IFCI_ERR_OOM, "ifci_sigma: workspace");
    return run_sigma(h, plan, precision, D, G, s);
}

int ifci_frozen_core(ifci_handle_t h, const ifci_system_t *sys, int nx, const int *bodies, double *h1,
                     double *eri_x, double *e_core, ifci_stream_t stream) {
    using namespace ifci;
    if (!h) return IFCI_ERR_INVALID_ARG;
    if (!sys || !bodies || !h1 || !eri_x || !e_core || nx < 1 || nx > sys->nbody)
        return set_error(h, IFCI_ERR_INVALID_ARG, "ifci_frozen_core: bad arguments");
    for (int i = 0; i < nx; i++)
        if (bodies[i] < 0 || bodies[i] >= sys->nbody || (i && bodies[i] <= bodies[i - 1]))
            return set_error(h, IFCI_ERR_INVALID_ARG, "ifci_frozen_core: bodies must be ascending and in range");
    IFCI_CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = as_cuda(stream);
    const int norb = sys->norb;
    const long long npg = (long long)norb * (norb + 1) / 2;
    std::vector<int> orbs;
    std::vector<char> inx(sys->nbody, 0);
    for (int i = 0; i < nx; i++) inx[bodies[i]] = 1;
    for (int b = 0; b < sys->nbody; b++)
        if (inx[b])
            for (int p = sys->body_offset[b]; p < sys->body_offset[b + 1]; p++) orbs.push_back(p);
    const int nA = (int)orbs.size();
    for (int b = 0; b < sys->nbody; b++)
        if (!inx[b]) orbs.push_back(sys->body_offset[b]);
    const int nC = (int)orbs.size() - nA;
    size_t need = ws_round(sizeof(FrozenDesc)) + ws_round(orbs.size() * sizeof(int)) + ws_round(8) +
                  (sys->on_host ? ws_round((size_t)norb * norb * 8) + ws_round((size_t)npg * npg * 8) : 0);
    IFCI_TRY(ws_reserve(h, need));
    auto *fd = ws_take<FrozenDesc>(h, 1);
    int *d_orbs = ws_take<int>(h, orbs.size());
    double *d_ec = ws_take<double>(h, 1);
    const double *dh = sys->h, *dV = sys->eri;
    if (sys->on_host) {
        double *th = ws_take<double>(h, (size_t)norb * norb);
        double *tV = ws_take<double>(h, (size_t)npg * npg);
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(th, sys->h, (size_t)norb * norb * 8, cudaMemcpyHostToDevice, s));
        IFCI_CUDA_TRY(h, cudaMemcpyAsync(tV, sys->eri, (size_t)npg * npg * 8, cudaMemcpyHostToDevice, s));
        dh = th;
        dV = tV;
    }
    FrozenDesc f{nA, nC, 0, h1, eri_x, d_ec};
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(fd, &f, sizeof(f), cudaMemcpyHostToDevice, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(d_orbs, orbs.data(), orbs.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    IFCI_TRY(launch_frozen_core(h, 1, fd, d_orbs, dh, dV, norb, s));
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(e_core, d_ec, 8, cudaMemcpyDeviceToHost, s));
    IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));
    return IFCI_OK;
}

}  // extern "C"
