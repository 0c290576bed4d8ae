// Batched Davidson over many CI problems of uneven size.
#pragma once
#include "sigma.cuh"

namespace ifci {

// A Davidson problem iterates in a rectangular block of a CI space: rows are
// alpha strings sa[0..na), columns beta strings sb[0..nb) (nullptr: every
// string, in order), vector index I = ia * nb + ib.  A whole CI space is the
// block with na = nb = nstr.  sym = 1: the block is its own spin-flip image
// (sa == sb) and its vectors are kept symmetric, x[ia][ib] = x[ib][ia]; the
// space iterated is then the na (na + 1) / 2 symmetric vectors.  sym = 0: an
// off-diagonal block (alpha and beta classes differ) whose spin-flip image
// is not stored; every vector of the block counts (ndim = na * nb).
struct DavProb {
    long long ndet;          // na * nb
    long long ndim;          // dimension of the vector space iterated (see above)
    int nstr;                // strings of the whole CI space
    int na, nb, sym;
    int item0, nitem;        // range of vector work items
    int seed_block;          // 0: default start block; r >= 1: from the r-th P-space block (second pass)
    const int *sa, *sb;      // global string index of each row / column, or nullptr
    double *B;               // (max_space + 1) slots of ndet: basis vectors
    double *S;               // (max_space + 1) slots of ndet: sigma of each slot
    const double *hd;        // diagonal <I|H|I> (no constant)
    double *c_out;           // converged vector or nullptr
    const double *seed;      // start vector (ndet, normalised) instead of the start block, or nullptr
    double *gc, *gs;         // sector blocks: the whole space's sigma input / output (nstr^2) or nullptr
    const unsigned char *mask;   // selected-CI problem: determinants kept (sigma zeroed elsewhere) or nullptr
    double e_core;
};

// global string index of row / column r of a block
__host__ __device__ inline int blk_row(const DavProb &p, int r) { return p.sa ? p.sa[r] : r; }
__host__ __device__ inline int blk_col(const DavProb &p, int c) { return p.sb ? p.sb[c] : c; }

struct DavState {
    int k;                   // basis vectors held (slots 0..k-1)
    int newest;              // slot whose sigma is built next (k - 1)
    int active;              // 1 while iterating
    int restart;             // restart requested this iteration
    int iters;               // sigma builds so far
    int status;
    int tslot;               // slot holding the correction vector
    long long ref;           // index of the lowest-diagonal determinant (diagnostic)
    int force;               // mixed mode: restart at the next check (subspace exhausted)
    int kold;                // subspace size just before the last restart
    int exact_all;           // mixed mode: 0 in phase 1 (low-precision sigma), 1 in phase 2 (exact sigma)
    int rebuild_to;          // phase switch: slots 0..rebuild_to-1 get their exact sigma, one per iteration
    int nform;               // Ritz vectors formed by the last restart
    int noise_slot;          // start block: slot of the random vector, -1 if none
    double theta, theta_prev, rnorm, tnorm2, energy;
    double rnorm_exact_prev; // mixed mode, phase 1: residual norm at the previous restart
    int tgt;                 // Ritz root (rank) whose correction is built this iteration
    int skip2;               // the second Gram-Schmidt pass is not needed this iteration
    int tcur;                // Ritz root of the correction now in flight (check -> advance)
    int pad3_;
    double rn[4];            // last residual norm of each of the lowest Ritz roots (kKeep)
};

constexpr int kVecChunk = 4096;   // determinants per vector work item
constexpr int kMaxSpace = 24;
constexpr int kNP = kMaxSpace + 2;
// thick restart keeps the lowest kKeep Ritz vectors (a near-degenerate pair
// of lowest states is resolved by Rayleigh-Ritz instead of being re-found
// after every restart); ys holds kKeep Ritz vectors per problem, kNP doubles
// each, the Ritz value of vector r at [r * kNP + kMaxSpace]
constexpr int kKeep = 4;
static_assert(kKeep <= 4, "DavState::rn holds the residuals of at most 4 roots");
// a higher Ritz root within kCompete (Eh) of the lowest is corrected too, in
// alternation, until its residual is below sqrt(r_tol): when H splits into
// (nearly) decoupled sectors (e.g. charge distributions over distant bodies)
// the correction of the lowest root never enters another sector, whose
// minimum may still lie lower
constexpr double kCompete = 0.3;
constexpr int kYStride = kKeep * kNP;
// start block: up to kStartP lowest eigenvectors of H in the P-space (their
// symmetry classes differ when H has symmetries beyond spin) plus one random
// vector that vanishes on the P-space determinants (exactly orthogonal to them)
constexpr int kStartP = 3;
constexpr int kPspMax = 64;
constexpr int kPspBlock = 24;   // P-space of a block of a sectored space (the start of its own sector only)
constexpr double kSectorWindow = 0.3;   // a second P-space block this close (Eh) gets its own pass
// a sectored problem whose dropped integrals (H - H') are all below this
// needs no polish with the full H: the energy changes at second order, ~1e-24
constexpr double kPolishTol = 1e-12;

// start block layout of a problem iterating in ndim dimensions with subspace
// max_space; a problem with a start vector of its own starts from that alone
__host__ __device__ inline void start_block(long long ndim, int max_space, bool seeded, int *nv, int *noise_slot) {
    if (seeded) {
        *nv = 1;
        *noise_slot = -1;
        return;
    }
    const long long nsym = ndim;
    const bool noise = nsym > kPspMax && max_space >= 4;
    long long v = kStartP;
    if (v > nsym) v = nsym;
    if (v > max_space - 2 - (noise ? 1 : 0)) v = max_space - 2 - (noise ? 1 : 0);
    if (v < 1) v = 1;
    *nv = (int)v;
    *noise_slot = noise ? (int)v : -1;
}

struct DavBatch {
    int nprob = 0, max_space = 12;
    int keep = kKeep;             // Ritz vectors kept at a thick restart (<= max_space - 2)
    int graph_iters = 0;          // iterations per captured CUDA graph (0: eager launches)
    double *d_blk_energy = nullptr;   // [nprob][2] lowest eigenvalue of the two lowest P-space blocks
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
    // sigma units (one CI space each; a sectored space has several problems)
    int nunit = 0;
    bool any_sector = false;
    bool any_mask = false;        // some problem iterates on a determinant selection (DavProb::mask)
    int2 *d_urange = nullptr;     // [nunit] first problem, problem count
    long long *d_pidx = nullptr;  // [nprob][kPspMax] P-space determinants of the start block
    int *d_pcount = nullptr;      // [nprob]
    int *d_uhi = nullptr, *d_ulo = nullptr;   // [nunit] sigma flags of the hi / lo plan
};


}  // namespace ifci
