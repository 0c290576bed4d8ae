// ifci_sigma_noalloc: the FP64 sigma build of ifci_sigma with all of its
// scratch memory in one fixed, file-scope device array, for callers that may
// not allocate device memory themselves (see include/ifci.h).
#include <atomic>

#include "hamiltonian.cuh"
#include "sigma.cuh"

namespace ifci {

cudaError_t launch_sigma_fp64_raw(const SigmaProb *d_probs, const WorkItem *d_items, int nitem,
                                  const WorkItem *d_tiles, int ntile, double *D, double *G, cudaStream_t s);
cudaError_t launch_fold_raw(const FoldDesc *d_desc, int max_np, cudaStream_t s);

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB on every device that loads the library
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
// device address of g_static_scratch, per device (written once per device;
// host threads may race on the first call, and each stores the same address)
std::atomic<void *> g_scratch_addr[kMaxDevices];

// the two descriptors of the call, passed by value so that no host buffer
// outlives the call
__global__ void write_desc_kernel(FoldDesc *fd, FoldDesc f, SigmaProb *pd, SigmaProb p) {
    *fd = f;
    *pd = p;
}

// Work lists of the single problem: gather/scatter items and 64 x 64 contraction tiles.
__global__ void fill_work_kernel(WorkItem *items, int nitem, WorkItem *tiles, int ntile, int np, long long ndet) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nitem) items[i] = WorkItem{0, 0, (long long)i * kGatherChunk};
    if (i < ntile) {
        long long ntn = (ndet + kGemmTN - 1) / kGemmTN;
        int mt = (int)(i / ntn);
        long long nt = i % ntn;
        tiles[i] = WorkItem{0, mt * kGemmTM, nt * kGemmTN};
    }
}

}  // namespace
}  // namespace ifci

extern "C" size_t ifci_sigma_noalloc_max_bytes(void) { return ifci::kStaticScratchBytes; }

extern "C" int ifci_sigma_noalloc(const ifci_strings_t *str, const double *h1, const double *eri, const double *c,
                                  double *sigma, ifci_stream_t stream) {
    using namespace ifci;
    if (!str || !h1 || !eri || !c || !sigma || !str->exc || c == sigma) return IFCI_ERR_INVALID_ARG;
    int nstr = 0, nexc = 0;
    if (ifci_string_counts(str->norb, str->nelec_spin, &nstr, &nexc) != IFCI_OK || nstr != str->nstr ||
        nexc != str->nexc || str->nelec_spin < 1)
        return IFCI_ERR_INVALID_ARG;
    const int n = str->norb, np = n * (n + 1) / 2;
    const long long ndet = (long long)nstr * nstr;
    const int nitem = (int)((ndet + kGatherChunk - 1) / kGatherChunk);
    const int ntile = (int)(((np + kGemmTM - 1) / kGemmTM) * ((ndet + kGemmTN - 1) / kGemmTN));
    const size_t need = ws_round(sizeof(FoldDesc)) + ws_round(sizeof(SigmaProb)) + ws_round((size_t)np * np * 8) +
                        2 * ws_round((size_t)np * ndet * 8) + ws_round((size_t)nitem * sizeof(WorkItem)) +
                        ws_round((size_t)ntile * sizeof(WorkItem));
    if (need > kStaticScratchBytes) return IFCI_ERR_INVALID_ARG;   // larger than the fixed scratch array

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return IFCI_ERR_CUDA;
    void *addr = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!addr) {
        // once per device, with that device current: the host-side symbol is
        // only a stand-in, the kernels need the device address
        if (cudaGetSymbolAddress(&addr, g_static_scratch) != cudaSuccess || !addr) {
            cudaGetLastError();
            return IFCI_ERR_CUDA;
        }
        g_scratch_addr[dev].store(addr, std::memory_order_release);
    }
    char *base = static_cast<char *>(addr);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base + off;
        off += ws_round(bytes);
        return p;
    };
    auto *fd = reinterpret_cast<FoldDesc *>(take(sizeof(FoldDesc)));
    auto *pd = reinterpret_cast<SigmaProb *>(take(sizeof(SigmaProb)));
    auto *W = reinterpret_cast<double *>(take((size_t)np * np * 8));
    auto *D = reinterpret_cast<double *>(take((size_t)np * ndet * 8));
    auto *G = reinterpret_cast<double *>(take((size_t)np * ndet * 8));
    auto *items = reinterpret_cast<WorkItem *>(take((size_t)nitem * sizeof(WorkItem)));
    auto *tiles = reinterpret_cast<WorkItem *>(take((size_t)ntile * sizeof(WorkItem)));

    cudaStream_t s = as_cuda(stream);
    FoldDesc f{n, 2 * str->nelec_spin, np, h1, eri, W};
    SigmaProb p{};
    p.n = n; p.nstr = nstr; p.nexc = nexc; p.np = np; p.ld = np;
    p.ndet = ndet; p.stride = ndet; p.exc = str->exc; p.W = W;
    p.cbase = c; p.sbase = sigma; p.doff = 0;
    // every scratch byte used below is written before it is read: nothing needs clearing
    write_desc_kernel<<<1, 1, 0, s>>>(fd, f, pd, p);
    if (cudaGetLastError() != cudaSuccess) return IFCI_ERR_CUDA;
    if (launch_fold_raw(fd, np, s) != cudaSuccess) return IFCI_ERR_CUDA;
    int nfill = nitem > ntile ? nitem : ntile;
    fill_work_kernel<<<(nfill + 255) / 256, 256, 0, s>>>(items, nitem, tiles, ntile, np, ndet);
    if (cudaGetLastError() != cudaSuccess) return IFCI_ERR_CUDA;
    if (launch_sigma_fp64_raw(pd, items, nitem, tiles, ntile, D, G, s) != cudaSuccess) return IFCI_ERR_CUDA;
    return IFCI_OK;
}
