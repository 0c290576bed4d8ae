// Tensor-core (tcgen05) contraction G = W D for the BF16 and TF32 paths.
#include "sigma.cuh"

namespace ifci {

int tc_supported(int precision) { return 0; }
int tc_operand_bytes(int np, int precision) { return 256; }
int launch_tc_pack_w(ifci_handle_t h, int nprob, const SigmaProb *d_probs, int precision, cudaStream_t s) {
    return set_error(h, IFCI_ERR_UNSUPPORTED, "tensor-core path not built");
}
int launch_tc_contract(ifci_handle_t h, const SigmaPlan &plan, const SigmaWave &w, int precision, const void *D,
                       void *G, cudaStream_t s) {
    return set_error(h, IFCI_ERR_UNSUPPORTED, "tensor-core path not built");
}

}  // namespace ifci
