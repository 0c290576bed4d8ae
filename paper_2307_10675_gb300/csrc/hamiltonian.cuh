// Device descriptors of the Hamiltonian-building kernels.
#pragma once
#include "common.cuh"

namespace ifci {

struct FrozenDesc {
    int nA, nC;          // active and core orbital counts
    long long orb_off;   // offset into the orbital list: [active..., core...]
    double *h1;          // out nA*nA
    double *eri;         // out npairA*npairA
    double *e_core;      // out scalar
};

struct FoldDesc {
    int n, nelec, ld;    // active orbitals, active electrons (2 nelec_spin), padded pair count
    const double *h1;    // nA*nA
    const double *eri;   // npair*npair
    double *W;           // out ld*ld
};

struct HdiagDesc {
    int n, nstr;
    const uint64_t *strings;
    const double *h1;
    const double *eri;
    double *hd;          // out nstr*nstr
};

int launch_frozen_core(ifci_handle_t h, int nprob, const FrozenDesc *d_desc, const int *d_orbs,
                       const double *d_h, const double *d_V, int norb, cudaStream_t s);
int launch_fold(ifci_handle_t h, int nprob, const FoldDesc *d_desc, int max_np, cudaStream_t s);
int launch_hdiag(ifci_handle_t h, const HdiagDesc *d_desc, const int *d_wprob, const long long *d_wstart,
                 int nwork, int chunk, cudaStream_t s);
int launch_reference_energy(ifci_handle_t h, const int *d_bond, int nb, const double *d_h, const double *d_V,
                            int norb, double *d_e0, cudaStream_t s);

}  // namespace ifci
