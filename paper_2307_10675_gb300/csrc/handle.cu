// Handle, workspace and error reporting of the C ABI.
#include <stdarg.h>
#include <string.h>

#include "common.cuh"

namespace ifci {

long long binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    long long r = 1;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

int set_error(ifci_handle_t h, int code, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->last_error = buf;
    return code;
}

int ws_reserve(ifci_handle_t h, size_t bytes) {
    h->ws_top = 0;
    if (bytes <= h->ws_bytes) return IFCI_OK;
    // the old buffer may still be read by work in flight on any stream
    IFCI_CUDA_TRY(h, cudaDeviceSynchronize());
    if (h->ws) IFCI_CUDA_TRY(h, cudaFree(h->ws));
    h->ws = nullptr;
    h->ws_bytes = 0;
    size_t want = bytes + bytes / 8;
    cudaError_t e = cudaMalloc(&h->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&h->ws, bytes);
        want = bytes;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->ws = nullptr;
        return set_error(h, IFCI_ERR_OOM, "workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
    h->ws_bytes = want;
    return IFCI_OK;
}

void ws_reset(ifci_handle_t h) { h->ws_top = 0; }

static cudaEvent_t prof_event(ifci_handle_t h) {
    if (!h->prof_pool.empty()) {
        cudaEvent_t e = h->prof_pool.back();
        h->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(ifci_handle_t h, cudaStream_t s, int kind) {
    ifci_handle_s::ProfRec r;
    r.a = prof_event(h);
    r.b = nullptr;
    r.kind = kind;
    cudaEventRecord(r.a, s);
    h->prof_pending.push_back(r);
}

void prof_end(ifci_handle_t h, cudaStream_t s) {
    if (h->prof_pending.empty()) return;
    auto &r = h->prof_pending.back();
    if (r.b) return;
    r.b = prof_event(h);
    cudaEventRecord(r.b, s);
}

void prof_collect(ifci_handle_t h) {
    for (auto &r : h->prof_pending) {
        if (!r.b) continue;
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            h->prof_ms[r.kind] += ms;
            h->prof_count[r.kind] += 1;
        }
        h->prof_pool.push_back(r.a);
        h->prof_pool.push_back(r.b);
    }
    h->prof_pending.clear();
    cudaGetLastError();
}

int device_sm_count(int device) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
    return n > 0 ? n : 1;
}

}  // namespace ifci

extern "C" {

int ifci_handle_create(ifci_handle_t *handle, size_t workspace_bytes, int device) {
    if (!handle) return IFCI_ERR_INVALID_ARG;
    *handle = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return IFCI_ERR_INVALID_ARG;
    }
    ifci_handle_t h = new ifci_handle_s();
    h->device = device;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    int st = IFCI_OK;
    if (cudaMalloc(&h->d_err, 256) != cudaSuccess || cudaMemset(h->d_err, 0, 256) != cudaSuccess ||
        cudaMalloc(&h->d_counter, 256) != cudaSuccess || cudaMemset(h->d_counter, 0, 256) != cudaSuccess) {
        cudaGetLastError();
        st = IFCI_ERR_CUDA;
    }
    if (st == IFCI_OK && workspace_bytes) st = ifci::ws_reserve(h, workspace_bytes);
    cudaSetDevice(prev);
    if (st != IFCI_OK) {
        if (h->d_err) cudaFree(h->d_err);
        if (h->d_counter) cudaFree(h->d_counter);
        if (h->ws) cudaFree(h->ws);
        delete h;
        return st;
    }
    *handle = h;
    return IFCI_OK;
}

int ifci_handle_destroy(ifci_handle_t h) {
    if (!h) return IFCI_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    ifci::prof_collect(h);
    for (cudaEvent_t e : h->prof_pool) cudaEventDestroy(e);
    if (h->ws) cudaFree(h->ws);
    if (h->ws_alt) cudaFree(h->ws_alt);
    if (h->kept.vec) cudaFree(h->kept.vec);
    if (h->d_err) cudaFree(h->d_err);
    if (h->d_counter) cudaFree(h->d_counter);
    cudaSetDevice(prev);
    delete h;
    return IFCI_OK;
}

const char *ifci_last_error_string(ifci_handle_t h) { return h ? h->last_error.c_str() : "null handle"; }

size_t ifci_workspace_bytes(ifci_handle_t h) { return h ? h->ws_bytes + h->ws_alt_bytes : 0; }

long long ifci_kernel_launches(ifci_handle_t h) { return h ? h->launches : 0; }

int ifci_profile_enable(ifci_handle_t h, int enable) {
    if (!h) return IFCI_ERR_INVALID_ARG;
    ifci::prof_collect(h);
    h->prof = enable != 0;
    for (int k = 0; k < 8; k++) {
        h->prof_ms[k] = 0.0;
        h->prof_count[k] = 0;
    }
    return IFCI_OK;
}

int ifci_profile_read(ifci_handle_t h, int kind, double *ms, long long *launches) {
    if (!h || kind < 0 || kind >= 8) return IFCI_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    ifci::prof_collect(h);
    cudaSetDevice(prev);
    if (ms) *ms = h->prof_ms[kind];
    if (launches) *launches = h->prof_count[kind];
    return IFCI_OK;
}

}  // extern "C"
