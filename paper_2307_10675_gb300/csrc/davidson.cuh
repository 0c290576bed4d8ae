// Batched Davidson over many CI problems of uneven size.
#pragma once
#include "sigma.cuh"

namespace ifci {

struct DavProb {
    long long ndet;
    int nstr;
    int item0, nitem;        // range of vector work items
    int pad_;
    double *B;               // (max_space + 1) slots of ndet: basis vectors
    double *S;               // (max_space + 1) slots of ndet: sigma of each slot
    const double *hd;        // diagonal <I|H|I> (no constant)
    double *c_out;           // converged vector or nullptr
    double e_core;
};

struct DavState {
    int k;                   // basis vectors held (slots 0..k-1)
    int newest;              // slot whose sigma is built next (k - 1)
    int active;              // 1 while iterating
    int restart;             // restart requested this iteration
    int iters;               // sigma builds so far
    int status;
    int tslot;               // slot holding the correction vector
    long long ref;           // index of the lowest-diagonal determinant (start vector)
    int force;               // mixed mode: restart at the next check (subspace exhausted)
    int kold;                // subspace size just before the last restart
    int exact_all;           // mixed mode: this problem now takes the exact sigma for every vector
    int pad_;
    double theta, theta_prev, rnorm, tnorm2, energy;
    double rnorm_exact_prev; // mixed mode: residual norm at the previous exact check
};

constexpr int kVecChunk = 4096;   // determinants per vector work item
constexpr int kMaxSpace = 24;
constexpr int kNP = kMaxSpace + 2;
// thick restart keeps the lowest kKeep Ritz vectors (a near-degenerate pair
// of lowest states is resolved by Rayleigh-Ritz instead of being re-found
// after every restart); ys holds kKeep Ritz vectors per problem, kNP doubles
// each, the Ritz value of vector r at [r * kNP + kMaxSpace]
constexpr int kKeep = 3;
constexpr int kYStride = kKeep * kNP;

struct DavBatch {
    int nprob = 0, max_space = 12;
    int keep = kKeep;             // Ritz vectors kept at a thick restart (<= max_space - 2)
    int precision = IFCI_FP64;
    int hi_precision = IFCI_FP64;
    int max_iter = 100;
    double e_tol = 1e-10, r_tol = 1e-6;
    std::vector<DavProb> probs;
    std::vector<WorkItem> vitems;
    DavProb *d_probs = nullptr;
    DavState *d_state = nullptr;
    WorkItem *d_vitems = nullptr;
    double *d_part = nullptr;     // [nitem][kNP]
    double *d_gs = nullptr;       // [nprob][kMaxSpace*kMaxSpace]
    double *d_y = nullptr;        // [nprob][kYStride] lowest Ritz vectors and values
    double *d_coef = nullptr;     // [nprob][kNP]
    int *d_nactive = nullptr;
};


}  // namespace ifci
