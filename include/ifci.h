/*
 * ifci.h — C ABI of the GB300 (sm_103a) library for the iFCI increment CI solve.
 *
 * Method (arXiv 2307.10675, Methods, "Incremental Full Configuration
 * Interaction", Eqs. 1-5): the correlation energy is expanded over bodies
 * (localized occupied orbitals), E_c = sum_i eps_i + sum_{i>j} eps_ij + ...,
 * with eps_X = E_c(X) - sum of the increments of every non-empty proper
 * subset of X.  E_c(X) = E_X - E_0 where E_X is the lowest singlet CI energy
 * with only the orbitals of body set X correlated (the other bodies' bonding
 * orbitals frozen doubly occupied, their virtuals removed) and E_0 is the
 * energy of the single reference determinant (Methods, last paragraph).
 * The paper solves each E_X with HBCI; this library solves it exactly
 * (determinant FCI + Davidson), whose cost is the sigma build sigma = H c.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an int status (ifci_status_t below).  On failure
 *   ifci_last_error_string(handle) describes the most recent error.
 * - "device" pointers are CUDA global memory on the handle's device, owned
 *   by the caller; the library never frees them.  "host" pointers are plain
 *   CPU memory.  Scratch memory comes only from the handle's workspace.
 * - Asynchronous calls are ordered on the cudaStream_t argument (0 = legacy
 *   default stream).  Calls documented as synchronous return after their
 *   results are written.
 * - Orbital pair index: pair(p,q) = P(P+1)/2 + Q with P = max(p,q),
 *   Q = min(p,q); npair = n(n+1)/2.  Packed two-electron integrals are the
 *   symmetric npair x npair row-major matrix V[pair(pq)][pair(rs)] = (pq|rs)
 *   (chemist notation, real orbitals).
 * - Strings: the nstr = C(norb, nelec_spin) occupation bit masks of one
 *   spin, ordered by increasing integer value (bit p = orbital p).  A CI
 *   vector is the row-major nstr x nstr matrix c[I_alpha][I_beta] of the
 *   determinants |I_alpha I_beta> = A+(I_alpha) B+(I_beta)|0>.
 * - Limits: norb <= 31 (pair index fits 9 bits), nstr < 2^22.
 */
#ifndef IFCI_H
#define IFCI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ifci_stream_t; /* same object as cudaStream_t */

typedef enum {
    IFCI_OK = 0,
    IFCI_ERR_INVALID_ARG = 1,   /* bad size, pointer or option; nothing was launched */
    IFCI_ERR_OOM = 2,           /* workspace could not grow */
    IFCI_ERR_CUDA = 3,          /* a CUDA runtime call failed (message has the CUDA error) */
    IFCI_ERR_NOT_CONVERGED = 4, /* at least one problem hit max_iter; per-problem status says which */
    IFCI_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out */
    IFCI_ERR_UNSUPPORTED = 6,   /* precision or size this build does not provide */
    IFCI_SCREENED = 7           /* per-set status only: the body set was screened out
                                   (ifci_davidson_opts_t.cnb_threshold) and not solved */
} ifci_status_t;

typedef enum {
    IFCI_FP64 = 0, /* every step in FP64 */
    IFCI_FP32 = 1, /* sigma contraction with FP32 inputs, FP32 accumulation */
    IFCI_TF32 = 2, /* sigma contraction on tensor cores, TF32 inputs (rounded with
                      cvt.rna, to nearest, ties away from zero), FP32 accumulation */
    IFCI_BF16 = 3, /* sigma contraction on tensor cores, BF16 inputs, FP32 accumulation */
    IFCI_FP64E = 4 /* sigma contraction to ~FP64 accuracy on FP16 tensor cores: both
                      operands split into 5 slices of 8-bit integers, the 15 leading
                      slice products accumulated exactly in FP32 per scale level,
                      levels combined in int64 (relative error ~2^-38 of max|W||D|) */
} ifci_precision_t;

/* Flag OR-ed into ifci_sigma's precision: the caller asserts that c is
 * spin-flip symmetric, c[Ia][Ib] = c[Ib][Ia] (the singlet sector the Davidson
 * solver works in).  The tensor-core precisions (BF16, TF32, FP64E) then gather the
 * alpha excitations only and return S + S^T, S the sigma of the alpha-only
 * intermediate, which equals H c for such c (a restatement of the sigma
 * build, not a step of the paper).  Ignored by FP64 and FP32, and by
 * spaces with 2 nstr^2 >= 2^31.  For a c that is not symmetric the result is
 * not H c: do not set the flag there. */
#define IFCI_SIGMA_SPIN_SYMMETRIC 0x100

typedef struct ifci_handle_s *ifci_handle_t;

/* ---------------------------------------------------------------- handle */

/* Creates a handle bound to CUDA device `device` with `workspace_bytes` of
 * scratch reserved up front (0 = none).  Calls grow the workspace when they
 * need more.  Not thread-safe: one host thread per handle at a time. */
int ifci_handle_create(ifci_handle_t *handle, size_t workspace_bytes, int device);
int ifci_handle_destroy(ifci_handle_t handle);
/* Message of the most recent failed call on this handle ("" if none).  The
 * string stays valid until the next call on the handle. */
const char *ifci_last_error_string(ifci_handle_t handle);
/* Bytes of workspace currently held by the handle. */
size_t ifci_workspace_bytes(ifci_handle_t handle);
/* Number of kernel launches this handle has issued since creation. */
long long ifci_kernel_launches(ifci_handle_t handle);

/* ifci_wait_selftest — makes one bounded device wait run out on purpose (a
 * CTA waits for an mbarrier arrival that nothing makes, for limit_cycles SM
 * clocks, 1 .. 4e9) and returns IFCI_ERR_TIMEOUT exactly as a timed-out wait
 * inside the contraction kernels does; the CUDA context stays usable and the
 * handle's error flag is cleared.  No paper counterpart: it exercises the
 * library's failure detection without a GPU fault.  Synchronous. */
int ifci_wait_selftest(ifci_handle_t handle, long long limit_cycles, ifci_stream_t stream);

/* Per-kernel-class timing with CUDA events recorded on the launching stream
 * around every kernel the library issues (no paper counterpart; it serves
 * the roofline measurement).  enable != 0 turns it on and zeroes the totals.
 * Classes: 0 sigma gather (and quantisation), 1 sigma contraction (FP64,
 * FP32, BF16, TF32), 2 sigma scatter, 3 Davidson vector kernels, 4 other,
 * 5 FP64-emulating tensor-core contraction, 6 Davidson set-up (integral
 * folds and images, diagonals, start vectors), 7 P-space eigensolves of the
 * start.  ifci_profile_read synchronises the
 * recorded events and returns the accumulated milliseconds and launches. */
int ifci_profile_enable(ifci_handle_t handle, int enable);
int ifci_profile_read(ifci_handle_t handle, int kind, double *ms, long long *launches);

/* ---------------------------------------------------------------- strings */

/* Host-only.  nstr = C(norb, nelec_spin); nexc = excitations per string =
 * nelec_spin * (norb - nelec_spin + 1) (one per occupied orbital for the
 * diagonal E_pp, one per occupied/empty orbital pair). */
int ifci_string_counts(int norb, int nelec_spin, int *nstr, int *nexc);

/* ifci_build_strings — occupation strings and single-excitation table
 * (the alpha/beta string layer of the determinant CI that solves E_X).
 *   strings : device uint64[nstr], output, ascending bit masks.
 *   exc     : device int32[nstr * nexc], output.  Row I lists, in ascending
 *             pair order, every nonzero E_pq |I> = s |J> with p,q such that
 *             p == q (q occupied) or exactly one of p,q occupied; entry =
 *             (J << 10) | (pair(p,q) << 1) | (s < 0).
 * Asynchronous on `stream`.  Errors: INVALID_ARG for sizes out of range. */
int ifci_build_strings(ifci_handle_t handle, int norb, int nelec_spin,
                       uint64_t *strings, int32_t *exc, ifci_stream_t stream);

typedef struct {
    int norb, nelec_spin, nstr, nexc;
    const uint64_t *strings;  /* device, from ifci_build_strings */
    const int32_t *exc;       /* device, from ifci_build_strings */
} ifci_strings_t;

/* ---------------------------------------------------------------- Hamiltonian pieces */

/* ifci_sigma — sigma = H c for one CI space (the per-increment hot loop).
 *   H = sum_pq h1_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps)
 * with E_pq the spin-summed excitation operators, no constant term.
 *   h1    : device double[norb*norb], symmetric one-electron integrals.
 *   eri   : device double[npair*npair], packed (pq|rs).
 *   c     : device double[nstr*nstr], input vector.
 *   sigma : device double[nstr*nstr], output (must not alias c).
 *   precision : ifci_precision_t of the contraction (FP64 exact path;
 *               the others round the contraction inputs, FP32 accumulate).
 * Sizes: BF16 and TF32 take npair <= 256 (norb <= 22), FP64E npair <= 304
 * (norb <= 24; above 204 pairs in K chunks of 192 whose exact int64 partial
 * sums are added), else UNSUPPORTED.  The intermediates take
 * 2 * npair * nstr^2 elements of the precision's storage type; a
 * spin-symmetric FP64E call above 2^31 G elements runs in row slabs of at
 * most 2^31 (16 GB), the scatter adding each slab's contribution into an
 * int64 accumulator, with the same result bit for bit.  Workspace beyond the
 * device's memory fails with OOM.
 * Asynchronous on `stream`; uses handle workspace (grows it if needed). */
int ifci_sigma(ifci_handle_t handle, const ifci_strings_t *str,
               const double *h1, const double *eri, const double *c, double *sigma,
               int precision, ifci_stream_t stream);

/* ifci_sigma_noalloc — the FP64 sigma = H c of ifci_sigma, for callers that
 * cannot allocate device memory: a host program whose memory manager owns all
 * of the GPU's memory (a caching allocator that reserved it up front), or a
 * latency-bound caller that cannot accept cudaMalloc's implicit device
 * synchronisation.  The paper has no counterpart; it exists for such callers.
 * No handle: all scratch (folded integrals, the intermediates D and G, work
 * lists) lives in one file-scope device array of ifci_sigma_noalloc_max_bytes()
 * = 16 MiB, which every GPU that loads the library holds until the process
 * exits.  The call makes no cudaMalloc/cudaFree and calls no allocating
 * library routine.
 *   Arguments and layout as for ifci_sigma (current CUDA device; FP64 only).
 *   Returns INVALID_ARG, without launching anything, when the problem's
 *   scratch (8*npair^2 + 16*npair*nstr^2 bytes plus small work lists) exceeds
 *   the array; CUDA_ERR on a CUDA failure.
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress); make that first call before any
 * stream capture.  Under CUDA's lazy module loading (the default) that first
 * call, or the library's first kernel launch on the device, also loads the
 * library's device code and the array itself, which takes device memory:
 * make the first call on each device before the caller's memory manager
 * reserves the device's memory (or load modules eagerly,
 * CUDA_MODULE_LOADING=EAGER); later calls need no device memory at all.
 * Every call shares the array and each call overwrites what it reads, so
 * nothing carries over between calls — but calls that overlap on the GPU
 * (other streams, other host threads) race on the array. */
size_t ifci_sigma_noalloc_max_bytes(void);
int ifci_sigma_noalloc(const ifci_strings_t *str, const double *h1, const double *eri,
                       const double *c, double *sigma, ifci_stream_t stream);

/* ifci_h_elements — single matrix elements <I|H|J> of the same H (no
 * constant) between determinants, by the Slater–Condon rules on the string
 * bit masks (the Davidson solver uses them for its start vectors: the lowest
 * eigenvector of H among the lowest-diagonal determinants).  The paper has no
 * separate call for this; it is exposed so that the rules can be checked
 * element by element.
 *   bra, ket : device int64[count], determinant indices I = I_a * nstr + I_b.
 *   out      : device double[count].
 * Asynchronous on `stream`; INVALID_ARG for an inconsistent string table. */
int ifci_h_elements(ifci_handle_t handle, const ifci_strings_t *str, const double *h1, const double *eri,
                    long long count, const long long *bra, const long long *ket, double *out,
                    ifci_stream_t stream);

/* ifci_hdiag — diagonal <I|H|I> of the same H (no constant), for the
 * Davidson preconditioner.  hd: device double[nstr*nstr].  Asynchronous. */
int ifci_hdiag(ifci_handle_t handle, const ifci_strings_t *str,
               const double *h1, const double *eri, double *hd, ifci_stream_t stream);

/* ---------------------------------------------------------------- systems */

typedef struct {
    int nbody;               /* number of bodies N */
    const int *body_offset;  /* host int[nbody+1]; body b owns orbitals
                                [off[b], off[b+1]); its first orbital is its
                                bonding (reference-occupied) orbital */
    int norb;                /* total orbitals = off[nbody] */
    const double *h;         /* double[norb*norb] one-electron integrals */
    const double *eri;       /* double[npair*npair] packed (pq|rs) */
    int on_host;             /* 1: h and eri are host pointers (copied in by
                                the call), 0: device pointers */
} ifci_system_t;

/* ifci_frozen_core — the effective CI problem of body set X (Methods,
 * definition of E_c(X)): core C = bonding orbitals of bodies not in X,
 * active A = orbitals of the bodies in X (ascending global index).
 *   E_core = sum_c 2 h_cc + sum_{c,d} [2 (cc|dd) - (cd|dc)]
 *   h1_pq  = h_pq + sum_c [2 (pq|cc) - (pc|cq)]           (p, q in A)
 *   eri_x  = (pq|rs) restricted to A, packed over A's local pair index.
 * bodies: host int[nx], distinct, ascending.  h1: device double[nA*nA];
 * eri_x: device double[npairA^2]; e_core: host double*.  Synchronous. */
int ifci_frozen_core(ifci_handle_t handle, const ifci_system_t *sys, int nx, const int *bodies,
                     double *h1, double *eri_x, double *e_core, ifci_stream_t stream);

/* ---------------------------------------------------------------- Davidson */

typedef struct {
    int norb, nelec_spin;
    const double *h1;   /* device double[norb*norb] */
    const double *eri;  /* device double[npair*npair] packed */
    double e_core;      /* constant added to the eigenvalue */
    double *c_out;      /* device double[nstr*nstr] converged vector, or NULL */
} ifci_problem_t;

typedef struct {
    int precision;       /* ifci_precision_t of the bulk sigma contraction */
    int max_iter;        /* Davidson iterations per problem (default 100) */
    int max_space;       /* subspace size before a restart, 3..24 (default 12) */
    double e_tol;        /* convergence: |E_k - E_{k-1}| < e_tol (default 1e-10 Eh) */
    double r_tol;        /* and ||H x - E x||_2 < r_tol (default 1e-6) */
    int refine;          /* >= 0: ifci_increments keeps the converged vectors in the handle
                            for ifci_rdm_backward; < 0: it does not (default 1).  Mixed
                            precision always finishes on exact sigmas. */
    int hi_precision;    /* mixed mode: sigma of restart vectors, IFCI_FP64 or IFCI_FP64E
                            (default IFCI_FP64E) */
    long long det_budget;/* D elements (npair x determinants) per sigma wave; 0 = 2^31.
                            A problem above it alone runs in row slabs of G on the
                            FP64E path (bit-identical result); on the other paths it
                            fails with OOM */
    int graph_iters;     /* > 0: Davidson iterations are captured in blocks of this
                            many into one CUDA graph, replayed on a stream of the
                            handle (event-ordered with `stream`); 0 = launched one
                            by one (default).  Ignored while profiling is on.
                            Results are identical either way. */
    int sector_passes;   /* 2: problems whose start matrix (the P-space of the lowest
                            -diagonal pair functions) splits into decoupled blocks with a
                            second block within 0.3 Eh of the lowest are solved again
                            from that block's lowest vector, and the lower result (energy
                            and vector) is kept; 0 or 1: one pass (default 0). */
    double decouple_tol; /* > 0: orbitals that no integral couples above this (|h_pq|, and
                            max_rs |(pq|rs)| for p, q in different groups) split a problem into
                            groups; H without those integrals conserves the alpha and beta
                            electron counts of every group, and each such block is solved as
                            its own Davidson problem (all blocks of a space share one sigma
                            per iteration); the lowest block's vector then starts a Davidson
                            iteration with the full H.  The lowest eigenvalue over decoupled
                            sectors is thereby found by construction.  0: off.
                            (default 1e-5) */
    double cnb_threshold;/* ifci_increments / ifci_rdm_backward only.  > 0: connected n-body
                            screening of the body sets of 3 or more bodies (Methods, screening
                            paragraph, C = 10^-4.6 Ha there; the exact rule is in the paper's
                            Supplementary Information, not available): a set is solved only
                            when its bodies are connected through pairs {a, b} of it with
                            |eps_ab| >= cnb_threshold; a screened set has eps_X = 0 in Eqs.
                            2-5 (which are then taken recursively, screened increments
                            counting as zero), e_x = NaN and status IFCI_SCREENED.
                            0: every set is solved (default 0). */
    int hbci_max_rounds; /* ifci_increments only.  > 0: every E_X is the HBCI energy
                            E_var + E_PT2 of ifci_hbci_batched (Methods, HBCI paragraph),
                            from the reference determinant of X, with at most this many
                            variational steps; ifci_rdm_backward then returns UNSUPPORTED.
                            0: exact CI (default 0). */
    double hbci_eps1;    /* HBCI selection threshold (default 1e-3 Eh, the paper's) */
    double hbci_eps2;    /* HBCI PT2 screening threshold (default 1e-6 Eh, the paper's) */
} ifci_davidson_opts_t;

/* Fills opts with the defaults listed above (precision IFCI_FP64). */
void ifci_davidson_default_opts(ifci_davidson_opts_t *opts);

/* ifci_davidson_batched — lowest singlet eigenpair of each problem's
 * H + e_core (Davidson in the spin-flip-even sector c = c^T, which holds
 * S = 0, 2, ...; diagonal preconditioner; classical Gram-Schmidt with a
 * second pass when the first removes more than half of the correction).
 * Start: the lowest eigenvectors of H among the 64 lowest-diagonal pair
 * functions (one per decoupled block of that small matrix first) plus a
 * random vector orthogonal to them; thick restarts keep the four lowest Ritz
 * vectors; Ritz roots within 0.3 Eh of the lowest are corrected in turn
 * until resolved.  When H splits into decoupled sectors (charge
 * distributions over bodies that no integral above decouple_tol couples),
 * every sector block is solved as its own problem and the lowest kept
 * (ifci_davidson_opts_t.decouple_tol), so the lowest eigenvalue over the
 * sectors is found by construction.  Mixed precision (precision = BF16/TF32/FP32)
 * runs a low-precision phase, then rebuilds exact sigmas (hi_precision) of
 * its kept Ritz vectors and finishes exactly; convergence is only judged on
 * exact sigmas.
 *   energies : host double[nprob], eigenvalues including e_core.
 *   iters    : host int[nprob] or NULL, sigma builds per problem.
 *   status   : host int[nprob] or NULL, IFCI_OK or IFCI_ERR_NOT_CONVERGED.
 * Synchronous.  Returns NOT_CONVERGED if any problem did not converge. */
int ifci_davidson_batched(ifci_handle_t handle, int nprob, const ifci_problem_t *probs,
                          const ifci_davidson_opts_t *opts, double *energies, int *iters,
                          int *status, ifci_stream_t stream);

/* ---------------------------------------------------------------- HBCI */

typedef struct {
    double eps1;      /* variational selection threshold (Eh); the paper uses 1e-3 */
    double eps2;      /* EN-PT2 screening threshold (Eh); the paper uses 1e-6 */
    int max_rounds;   /* variational steps at most (one Davidson solve each), >= 1 */
} ifci_hbci_opts_t;

/* ifci_hbci_batched — heat-bath selected CI with an Epstein–Nesbet PT2
 * correction for each problem (Methods, HBCI paragraph: the solver the paper
 * runs for every increment).  Per problem:
 *   1. S = {start_det[i]} (a closed-shell determinant I = Ia * nstr + Ia,
 *      normally the reference with every bonding orbital doubly occupied);
 *   2. (E_var, c) = lowest eigenpair of H + e_core on S in the spin-flip-even
 *      sector (the batched Davidson of ifci_davidson_batched with `dopts`,
 *      seeded from the previous c, sigma kept on S; decouple_tol ignored);
 *   3. every determinant a outside S with max_{i in S} |<a|H|i> c_i| > eps1
 *      joins S with its spin-flip image; back to 2 until none joins or
 *      max_rounds variational steps were taken;
 *   4. E_PT2 = sum_{a not in S} (sum_{i in S, |<a|H|i> c_i| > eps2}
 *      <a|H|i> c_i)^2 / (E_var - <a|H|a> - e_core).
 * S is a byte mask over the problem's determinant index and the PT2
 * numerators an FP64 array over it (nstr^2 * 18 bytes of device memory per
 * problem besides the Davidson's); norb <= 32, nelec_spin <= 7.
 *   start_det : host int64[nprob].
 *   e_var, e_pt2 : host double[nprob] (E_HBCI = e_var + e_pt2).
 *   nsel   : host int64[nprob] or NULL, |S| at the end.
 *   rounds : host int[nprob] or NULL, variational steps taken.
 *   status : host int[nprob] or NULL, IFCI_OK or IFCI_ERR_NOT_CONVERGED
 *            (some Davidson solve of the problem did not converge).
 *   c_out of a problem (optional): the final c.
 * Synchronous.  INVALID_ARG for a start determinant that is not closed-shell
 * or negative thresholds; UNSUPPORTED beyond the sizes above. */
int ifci_hbci_batched(ifci_handle_t handle, int nprob, const ifci_problem_t *probs,
                      const long long *start_det, const ifci_davidson_opts_t *dopts,
                      const ifci_hbci_opts_t *hopts, double *e_var, double *e_pt2,
                      long long *nsel, int *rounds, int *status, ifci_stream_t stream);

/* ---------------------------------------------------------------- increments */

/* Host-only: number of body sets of size 1..max_order (their order, used by
 * every per-set array: by size, then lexicographic in body index). */
int ifci_num_subsets(int nbody, int max_order, long long *count);

/* ifci_increments — the iFCI expansion truncated at max_order (Eqs. 1-5).
 *   e0      : host double*, reference energy E_0.
 *   e_x     : host double[nsub] or NULL, E_X per body set (NaN if screened;
 *             E_var + E_PT2 with opts->hbci_max_rounds > 0).
 *   eps     : host double[nsub], increments eps_X.
 *   e_total : host double*, E_0 + sum eps_X.
 *   iters   : host int[nsub] or NULL, sigma builds per set (HBCI: variational steps).
 *   status  : host int[nsub] or NULL, per-set Davidson status (IFCI_SCREENED for a
 *             set left out by opts->cnb_threshold).
 * Keeps the converged vectors in the handle when opts->refine >= 0 so that
 * ifci_rdm_backward can reuse them.  Synchronous. */
int ifci_increments(ifci_handle_t handle, const ifci_system_t *sys, int max_order,
                    const ifci_davidson_opts_t *opts, double *e0, double *e_x, double *eps,
                    double *e_total, int *iters, int *status, ifci_stream_t stream);

/* ifci_rdm_backward — gradient of E_iFCI (truncated at max_order) with
 * respect to the inputs h and V by Hellmann–Feynman on every E_Y:
 *   dE/dh_pq    = grad_out * sum_Y w_Y gamma^Y_pq + (1 - sum w) gamma^0_pq
 *   dE/dV[A][B] = grad_out * 1/2 sum over ordered (p,q) in A, (r,s) in B of
 *                 [sum_Y w_Y Gamma^Y_pqrs + (1 - sum w) Gamma^0_pqrs]
 * with w_Y = (-1)^(n-|Y|) C(N-|Y|-1, n-|Y|), gamma/Gamma the spin-summed
 * full-space 1-/2-RDMs of E_Y's vector.  Under connected n-body screening
 * (opts->cnb_threshold > 0) w_Y is the derivative of the screened total
 * with respect to E_Y at the inclusion pattern of the forward call (the
 * pattern itself is held fixed).  dh: device double[norb*norb];
 * deri: device double[npair*npair]; both overwritten.
 * recompute_vectors = 0 reuses the vectors of the last ifci_increments on
 * this handle for the same system (INVALID_ARG if there are none).
 * Synchronous. */
int ifci_rdm_backward(ifci_handle_t handle, const ifci_system_t *sys, int max_order,
                      const ifci_davidson_opts_t *opts, double grad_out,
                      double *dh, double *deri, int recompute_vectors, ifci_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* IFCI_H */
