// Host-side Davidson driver shared by ifci_davidson_batched and ifci_increments.
#pragma once
#include "davidson.cuh"
#include "hamiltonian.cuh"

namespace ifci {

struct ProbSpec {
    int n, m;               // active orbitals, electrons per spin
    const double *h1;       // device n*n
    const double *eri;      // device npair*npair
    double e_core;
    double *c_out;          // device nstr*nstr or nullptr
    int seed_block = 0;     // 0: the default start block; r >= 1: start from the lowest vector of the
                            // r-th lowest decoupled block of the P-space matrix
    // selected-CI iteration (hbci.cu): start from `seed` (normalised, zero
    // outside the selection) and keep every vector on the determinants with
    // mask[I] != 0 (sigma is zeroed elsewhere); ndim = dimension of the
    // spin-flip-even vectors on the selection.  Needs decouple_tol = 0.
    const double *seed = nullptr;
    const unsigned char *mask = nullptr;
    long long ndim = 0;
};

// coupling graph of one problem's orbitals (sectors.cu)
struct CoupDesc {
    int n;
    const double *h1, *eri;
};
// H' of a sectored problem: h1, eri with every integral that joins two groups set to zero
struct MaskDesc {
    int n;
    const double *h1, *eri;
    double *h1m, *erim;
    double *dropped;           // out: largest |integral| set to zero
    unsigned char label[32];   // group of each orbital
};

// Every m-electron string of n orbitals, ascending as bit masks (host).
std::vector<uint32_t> host_strings(int n, int m);
int check_opts(ifci_handle_t h, const ifci_davidson_opts_t &o);
int hi_precision_of(const ifci_davidson_opts_t &o);   // precision of the exact (restart) sigma
// Solves every problem; its memory comes from the handle's Davidson workspace
// (DavArena), sized here.  Outputs are host arrays (may be null except
// energies).  Synchronous.
int dav_solve(ifci_handle_t h, const std::vector<ProbSpec> &specs, const ifci_davidson_opts_t &o, double *energies,
              int *iters, int *status, cudaStream_t s, double *blk_energy = nullptr);
// HBCI of every problem from its closed-shell start determinant (hbci.cu)
int hbci_solve(ifci_handle_t h, const std::vector<ProbSpec> &specs, const std::vector<long long> &start,
               const ifci_davidson_opts_t &o, const ifci_hbci_opts_t &hb, double *e_var, double *e_pt2,
               long long *nsel, int *rounds, int *status, cudaStream_t s);
// dav_solve, then (opts.sector_passes >= 2) a second pass over the problems
// whose P-space shows a competitive second block.
int dav_solve_sectors(ifci_handle_t h, const std::vector<ProbSpec> &specs, const ifci_davidson_opts_t &o,
                      double *energies, int *iters, int *status, cudaStream_t s);
int dav_init(ifci_handle_t h, DavBatch &b, const HdiagDesc *d_hd, cudaStream_t s);
size_t psp_workspace_bytes(int nprob);
int launch_pspace_start(ifci_handle_t h, const DavBatch &b, const HdiagDesc *d_hd, cudaStream_t s);
int dav_iterate(ifci_handle_t h, DavBatch &b, SigmaPlan &hi_plan, SigmaPlan *lo_plan, int *d_hi, int *d_lo,
                void *D, void *G, int *h_nactive, cudaStream_t s);

// sectors.cu
int launch_coupling(ifci_handle_t h, int nprob, const CoupDesc *d_desc, double tau, uint32_t *d_adj, cudaStream_t s);
int launch_mask(ifci_handle_t h, int nprob, const MaskDesc *d_desc, cudaStream_t s);
int launch_sector_gather(ifci_handle_t h, const DavBatch &b, const int *flag, cudaStream_t s);
int launch_sector_scatter(ifci_handle_t h, const DavBatch &b, const int *flag, cudaStream_t s);
int launch_sector_hd(ifci_handle_t h, const DavBatch &b, cudaStream_t s);
int launch_unit_flags(ifci_handle_t h, const DavBatch &b, const int *hi, const int *lo, cudaStream_t s);
int launch_sector_expand(ifci_handle_t h, const DavBatch &b, double *const *d_dst, cudaStream_t s);
void orbital_groups(const uint32_t *adj, int n, std::vector<int> &label, int &ngroup);
// per unit: pmapc[I][k] = pmap[I][act[k]] for its npc active pairs (rows of
// pmap_ld(npc), padded with -1); one block per unit, grid-stride
struct CompactDesc {
    int nstr, ld, npc, ldc;
    const int32_t *pmap, *act;
    int32_t *pmapc;
};
int launch_compact_pair_maps(ifci_handle_t h, int n, const CompactDesc *d_desc, cudaStream_t s);

}  // namespace ifci
