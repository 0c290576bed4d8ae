// Self-test of the bounded device waits (failure detection without a fault).
//
// Every spin-wait of the library's kernels (mbarrier phases of the
// tensor-core contractions) gives up after a cycle limit, sets the handle's
// device error flag and returns; the host then reports IFCI_ERR_TIMEOUT and
// the CUDA context stays usable.  This entry makes one such wait run out on
// purpose: one CTA waits on an mbarrier that expects an arrival nothing
// makes, with a short limit.
#include "common.cuh"
#include "tcgen05.cuh"

namespace ifci {
namespace {

__global__ void wait_selftest_kernel(long long limit_cycles, int *__restrict__ err) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = tc::smem_u32(&bar);
    if (threadIdx.x == 0) {
        tc::mbar_init(b, 1);   // one arrival expected, none is ever made
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool done = false;
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        while (!done) {
            uint32_t ok;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(ok)
                : "r"(b), "r"(0u)
                : "memory");
            if (ok) done = true;
            else if (clock64() - t0 > limit_cycles) break;
        }
        if (!done) atomicExch(err, 1);
    }
    __syncthreads();
}

}  // namespace
}  // namespace ifci

extern "C" int ifci_wait_selftest(ifci_handle_t h, long long limit_cycles, ifci_stream_t stream) {
    using namespace ifci;
    if (!h || !h->d_err) return IFCI_ERR_INVALID_ARG;
    if (limit_cycles < 1 || limit_cycles > 4000000000ll)
        return set_error(h, IFCI_ERR_INVALID_ARG, "wait_selftest: limit %lld cycles", limit_cycles);
    IFCI_CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = as_cuda(stream);
    wait_selftest_kernel<<<1, 32, 0, s>>>(limit_cycles, h->d_err);
    IFCI_LAUNCH_CHECK(h);
    int flag = 0;
    IFCI_CUDA_TRY(h, cudaMemcpyAsync(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));
    if (flag) {
        IFCI_CUDA_TRY(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
        IFCI_CUDA_TRY(h, cudaStreamSynchronize(s));
        return set_error(h, IFCI_ERR_TIMEOUT, "wait_selftest: the bounded wait ran out as intended");
    }
    return IFCI_OK;
}
