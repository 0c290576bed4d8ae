// Batched sigma build: gather D = E+ c, contraction G = W D, scatter sigma = E+ G.
#pragma once
#include "common.cuh"

namespace ifci {

// One CI problem as seen by the sigma kernels.  The input vector is
// cbase + (*cslot) * stride and the output sbase + (*sslot) * stride, so a
// Davidson iteration can move its slots on the device.
struct SigmaProb {
    int n, nstr, nexc, np;   // active orbitals, strings, excitations per string, pairs
    int ld;                  // row stride of W (>= np)
    int sym;                 // 1: the vector is spin-flip symmetric (C = C^T); the tensor-core paths gather
                             // alpha excitations only and return S + S^T (set by plan_sigma, needs pmap)
    long long ndet;
    long long stride;
    const int32_t *exc;      // [nstr * nexc] excitation table of (n, nelec_spin)
    const uint8_t *blk;      // [nstr * kBlk16Stride] entry offsets per 16-pair block (tensor-core paths)
    const int32_t *pmap;     // [nstr * pmap_ld(np)] dense pair map (spin-flip-symmetric gathers) or nullptr
    const double *W;         // [ld * ld] folded contraction matrix, FP64
    const float *Wf;         // [ld * ld] FP32 copy (FP32 path) or nullptr
    const void *Wtc;         // tensor-core operand image (BF16 path) or nullptr
    const void *Woz;         // sliced operand image of the FP64-emulating path or nullptr
    double *Wexp;            // [np] power-of-two row scales of Woz
    double dscale;           // power of two >= max |D| (FP64-emulating path)
    long long qoff;          // element offset of the quantised copy of c in its wave buffer
    const double *cbase;
    double *sbase;
    const int *cslot;        // device slot index or nullptr (= 0)
    const int *sslot;        // device slot index or nullptr (= 0)
    const int *active;       // device flag or nullptr (= active)
    long long doff;          // element offset of this problem's D and G blocks in a wave
    // FP64-emulating contraction over a subset of the pairs (a sectored space,
    // whose H' has no integral joining two groups): npc pairs act[0..npc) in
    // ascending order, the pair map restricted to them (pmapc, rows of
    // pmap_ld(npc)), and a flag per pair (pact) for the scatter, which skips
    // the G rows of the other pairs.  act = nullptr: every pair (npc = np).
    int npc;
    const int32_t *act;
    const int32_t *pmapc;
    const uint8_t *pact;
};

// D/G elements one problem takes in a wave (the quantised +-c copies of the
// symmetric tensor-core gathers share the D buffer and need 2 ndet)
inline long long sigma_elems(int np, long long ndet) { return (long long)(np < 2 ? 2 : np) * ndet; }

struct WorkItem {
    int prob;
    int sub;                 // GEMM: first output pair row of the tile
    long long start;         // first determinant
};

constexpr int kGatherChunk = 256;   // determinants per gather/scatter block
constexpr long long kSigmaSlabBudget = 1ll << 31;   // G elements per row slab of ifci_sigma (16 GB int64)
constexpr int kGemmTM = 64, kGemmTN = 64, kGemmTK = 16;

struct SigmaWave {
    int prob0, nprob;        // problems of the wave (consecutive in the plan)
    int item0, nitem;        // gather/scatter items
    int tile0, ntile;        // contraction tiles
    int tc0, ntc;            // tensor-core tiles (BF16/TF32)
    long long delems;        // D (and G) elements of the wave
    long long qelems;        // elements of the quantised copies of c (sum of ndet)
    // Row slab of one spin-flip-symmetric FP64E problem too large for the
    // budget (kn > 0): G holds the determinants [k0, k0 + kn) only (whole alpha
    // rows), G[A][K - k0] with row stride kn; the scatter adds the slab's
    // contributions into an int64 accumulator S (after the problem's +-Q copy
    // in the D buffer) and converts on the last slab.  kn = 0: whole problems.
    long long k0, kn;
    int slab_first, slab_last;
};

// Host-side plan over a fixed problem set; device arrays live in caller memory.
struct SigmaPlan {
    std::vector<SigmaProb> probs;
    std::vector<SigmaWave> waves;
    std::vector<WorkItem> items, tiles, tctiles;
    long long max_delems = 0;
    long long max_qelems = 0;   // largest quantised copy of a wave (the D buffer of the FP64E path)
    bool any_sym = false;    // some problem uses the spin-flip-symmetric gathers
    SigmaProb *d_probs = nullptr;
    WorkItem *d_items = nullptr, *d_tiles = nullptr, *d_tctiles = nullptr;
};

// Splits probs into waves of at most `budget` D elements (each problem whole).
// A problem alone above the budget is split into row slabs (SigmaWave::kn)
// when it takes the spin-flip-symmetric FP64E path; otherwise it fails with
// IFCI_ERR_OOM.
int plan_sigma(ifci_handle_t h, SigmaPlan &plan, long long budget, int precision);
size_t plan_device_bytes(const SigmaPlan &plan);
// Copies the plan's descriptor arrays to device memory taken from the workspace.
int upload_plan(ifci_handle_t h, SigmaPlan &plan, cudaStream_t s);
// The same into device arrays the caller has already set in the plan.
int upload_plan_to(ifci_handle_t h, SigmaPlan &plan, cudaStream_t s);
// Launches every wave: D, G are device buffers of at least max_delems
// elements of the precision's storage type (8 B for FP64, 4 B otherwise).
int run_sigma(ifci_handle_t h, const SigmaPlan &plan, int precision, void *D, void *G, cudaStream_t s);
size_t sigma_elem_bytes(int precision);

// FP64-accurate contraction on FP16 tensor cores (sigma_oz.cu)
int oz_operand_bytes(int np);                  // bytes of one problem's sliced W image (+ row scales)
int oz_tile_n();                               // output pairs per tile
int launch_oz_pack_w(ifci_handle_t h, int nprob, const SigmaProb *d_probs, cudaStream_t s);
int launch_oz_contract(ifci_handle_t h, const SigmaPlan &plan, const SigmaWave &w, const void *Q, void *G,
                       cudaStream_t s);
int launch_oz_dscale(ifci_handle_t h, SigmaProb *d_prob, const double *c, long long n, cudaStream_t s);

// tensor-core contraction (sigma_tc.cu)
int tc_supported(int precision);
int tc_operand_bytes(int np, int precision);   // bytes of one problem's W image
int launch_tc_pack_w(ifci_handle_t h, int nprob, const SigmaProb *d_probs, int precision, cudaStream_t s);
int launch_tc_contract(ifci_handle_t h, const SigmaPlan &plan, const SigmaWave &w, int precision,
                       const void *D, void *G, cudaStream_t s);

}  // namespace ifci
