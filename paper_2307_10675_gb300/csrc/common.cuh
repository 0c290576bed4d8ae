// Internal helpers of the iFCI GB300 library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>
#include <vector>

#include "../../include/ifci.h"

struct ifci_handle_s {
    int device = 0;
    // per-kernel-class CUDA-event timing (ifci_profile_enable)
    bool prof = false;
    struct ProfRec { cudaEvent_t a, b; int kind; };
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[8] = {0};
    long long prof_count[8] = {0};
    char *ws = nullptr;          // workspace base (device)
    size_t ws_bytes = 0;         // capacity
    size_t ws_top = 0;           // bump pointer
    // the Davidson solver's own workspace, swapped in for the duration of a
    // solve (DavArena) so that it can grow after the caller carved its part
    char *ws_alt = nullptr;
    size_t ws_alt_bytes = 0, ws_alt_top = 0;
    std::string last_error;
    long long launches = 0;
    int *d_err = nullptr;        // device flag set by kernels whose bounded waits ran out
    int *d_counter = nullptr;    // tile counter of the dynamically scheduled kernels (reset per launch)
    // vectors kept by ifci_increments for ifci_rdm_backward
    struct Kept {
        bool valid = false;
        int nbody = 0, max_order = 0, norb = 0;
        std::vector<int> body_offset;
        const void *h_ptr = nullptr, *eri_ptr = nullptr;
        double *vec = nullptr;               // device, all vectors back to back
        size_t vec_bytes = 0;
        std::vector<long long> vec_off;      // per subset offset (doubles)
        bool screened = false;               // connected n-body screening was applied
        std::vector<char> included;          // per subset: solved (1) or screened out (0)
    } kept;
};

namespace ifci {

constexpr int kPairBits = 9;       // pair index < 512  => norb <= 31
constexpr int kBlk16 = 16;         // 16-pair blocks of the tensor-core paths (npair <= 256)
constexpr int kBlk16Stride = 20;   // bytes per string in the block-offset table (19 blocks: npair <= 304)
constexpr int kMaxNorb = 31;
constexpr int kMaxStr = 1 << 22;

__host__ __device__ inline int pair_of(int p, int q) {
    int P = p > q ? p : q, Q = p > q ? q : p;
    return P * (P + 1) / 2 + Q;
}
__host__ __device__ inline int exc_J(int32_t e) { return (int)((uint32_t)e >> 10); }
__host__ __device__ inline int exc_pair(int32_t e) { return (e >> 1) & 511; }
__host__ __device__ inline double exc_sign(int32_t e) { return (e & 1) ? -1.0 : 1.0; }

long long binom(int n, int k);

// error bookkeeping ------------------------------------------------------
int set_error(ifci_handle_t h, int code, const char *fmt, ...);

#define IFCI_CUDA_TRY(h, expr)                                                        \
    do {                                                                              \
        cudaError_t _e = (expr);                                                      \
        if (_e != cudaSuccess)                                                        \
            return ifci::set_error((h), IFCI_ERR_CUDA, "%s:%d %s: %s", __FILE__,      \
                                   __LINE__, #expr, cudaGetErrorString(_e));          \
    } while (0)

#define IFCI_LAUNCH_CHECK(h)                                                          \
    do {                                                                              \
        (h)->launches++;                                                              \
        cudaError_t _e = cudaGetLastError();                                          \
        if (_e != cudaSuccess)                                                        \
            return ifci::set_error((h), IFCI_ERR_CUDA, "%s:%d launch: %s", __FILE__,  \
                                   __LINE__, cudaGetErrorString(_e));                 \
    } while (0)

#define IFCI_TRY(expr)                  \
    do {                                \
        int _s = (expr);                \
        if (_s != IFCI_OK) return _s;   \
    } while (0)

// profiling ---------------------------------------------------------------
enum ProfKind { PK_GATHER = 0, PK_CONTRACT = 1, PK_SCATTER = 2, PK_VECTOR = 3, PK_OTHER = 4, PK_CONTRACT_HI = 5,
                PK_SETUP = 6, PK_PSPACE = 7 };
void prof_begin(ifci_handle_t h, cudaStream_t s, int kind);
void prof_end(ifci_handle_t h, cudaStream_t s);
void prof_collect(ifci_handle_t h);   // adds finished event pairs to the totals (synchronises them)

struct ProfScope {
    ifci_handle_t h;
    cudaStream_t s;
    ProfScope(ifci_handle_t h_, cudaStream_t s_, int kind) : h(h_), s(s_) {
        if (h->prof) prof_begin(h, s, kind);
    }
    ~ProfScope() {
        if (h->prof) prof_end(h, s);
    }
};

// workspace --------------------------------------------------------------
// Calls reserve what they need up front (ws_reserve), then carve pieces with
// ws_take in the same order.  Growing synchronises the device first.
int ws_reserve(ifci_handle_t h, size_t bytes);
void ws_reset(ifci_handle_t h);
template <typename T>
T *ws_take(ifci_handle_t h, size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (h->ws_top + bytes > h->ws_bytes) return nullptr;
    T *p = reinterpret_cast<T *>(h->ws + h->ws_top);
    h->ws_top += bytes;
    return p;
}
inline size_t ws_round(size_t bytes) { return (bytes + 255) & ~size_t(255); }

// Makes the handle's Davidson workspace the current one (ws_reserve, ws_take)
// for its lifetime; the caller's workspace and the pointers into it stay valid.
struct DavArena {
    ifci_handle_t h;
    explicit DavArena(ifci_handle_t h_) : h(h_) { swap(); }
    ~DavArena() { swap(); }
    DavArena(const DavArena &) = delete;
    DavArena &operator=(const DavArena &) = delete;
    void swap() {
        char *b = h->ws; h->ws = h->ws_alt; h->ws_alt = b;
        size_t t = h->ws_bytes; h->ws_bytes = h->ws_alt_bytes; h->ws_alt_bytes = t;
        t = h->ws_top; h->ws_top = h->ws_alt_top; h->ws_alt_top = t;
    }
};

inline cudaStream_t as_cuda(ifci_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

int device_sm_count(int device);
// Grid of a grid-stride kernel over n blocks of work: at most per_sm
// resident blocks per SM (at least 1 block).
inline int stride_grid(int device, long long n, int per_sm) {
    const long long g = (long long)device_sm_count(device) * per_sm;
    return (int)(n < 1 ? 1 : (n < g ? n : g));
}

// The dynamic shared memory a kernel may use is a per-device attribute: each
// caller keeps one of these per kernel and raises the attribute on a device
// the first time that device needs more than it was opened up to.
constexpr int kMaxDevices = 64;
struct SmemOptIn {
    int bytes[kMaxDevices] = {};
};
template <typename K>
inline cudaError_t ensure_smem(SmemOptIn &opt, int device, K kernel, int bytes) {
    if (device < 0 || device >= kMaxDevices) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (bytes <= opt.bytes[device]) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) opt.bytes[device] = bytes;
    return e;
}
int launch_exc_blocks(ifci_handle_t h, int nstr, int nexc, const int32_t *exc, uint8_t *blk, cudaStream_t s);
// row stride (int32 entries) of the dense pair map
__host__ __device__ inline int pmap_ld(int np) { return (np + 15) / 16 * 16; }
// pair map of the spin-flip-symmetric tensor-core gathers (needs 2 nstr^2 < 2^31)
int launch_pair_map(ifci_handle_t h, int nstr, int nexc, int np, const int32_t *exc, int32_t *pmap, cudaStream_t s);

}  // namespace ifci
