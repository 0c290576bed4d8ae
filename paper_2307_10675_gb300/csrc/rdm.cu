// 1-/2-RDM backward pass of the iFCI energy (Hellmann–Feynman per body set).
#include "dav_driver.cuh"

extern "C" int ifci_rdm_backward(ifci_handle_t h, const ifci_system_t *sys, int max_order,
                                 const ifci_davidson_opts_t *opts, double grad_out, double *dh, double *deri,
                                 int recompute_vectors, ifci_stream_t stream) {
    return ifci::set_error(h, IFCI_ERR_UNSUPPORTED, "rdm_backward: not built yet");
}
