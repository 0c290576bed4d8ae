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
};

struct DavSizes {
    size_t bytes = 0;
    int nitem = 0, nclass = 0;
    long long max_pd = 0, sum_pd = 0, budget = 0;
    long long n_items_sigma = 0, n_tiles_sigma = 0;
};

int check_opts(ifci_handle_t h, const ifci_davidson_opts_t &o);
int hi_precision_of(const ifci_davidson_opts_t &o);   // precision of the exact (restart) sigma
// Upper bound of the workspace dav_solve takes (with ws_take) for these problems.
size_t dav_workspace_bytes(const std::vector<ProbSpec> &specs, const ifci_davidson_opts_t &o);
// Solves every problem; carves its memory from the handle workspace after
// whatever the caller already took.  Outputs are host arrays (may be null
// except energies).  Synchronous.
int dav_solve(ifci_handle_t h, const std::vector<ProbSpec> &specs, const ifci_davidson_opts_t &o, double *energies,
              int *iters, int *status, cudaStream_t s, double *blk_energy = nullptr);
// dav_solve, then (opts.sector_passes >= 2) a second pass over the problems
// whose P-space shows a competitive second block; the workspace above `mark`
// is reused by the second pass.
int dav_solve_sectors(ifci_handle_t h, const std::vector<ProbSpec> &specs, const ifci_davidson_opts_t &o,
                      double *energies, int *iters, int *status, cudaStream_t s);
int dav_init(ifci_handle_t h, DavBatch &b, const HdiagDesc *d_hd, cudaStream_t s);
size_t psp_workspace_bytes(int nprob);
int launch_pspace_start(ifci_handle_t h, const DavBatch &b, const HdiagDesc *d_hd, cudaStream_t s);
int dav_iterate(ifci_handle_t h, DavBatch &b, SigmaPlan &hi_plan, SigmaPlan *lo_plan, int *d_hi, int *d_lo,
                void *D, void *G, int *h_nactive, cudaStream_t s);

}  // namespace ifci
