"""GB300 (sm_103a) library for the iFCI increment CI solve of arXiv 2307.10675.

The compute path is the CUDA library ``_build/libifci.so`` (C ABI in
``include/ifci.h``); this package only marshals arguments to it.
"""
from .api import (  # noqa: F401
    IFCI_BF16, IFCI_FP32, IFCI_FP64, IFCI_FP64E, IFCI_TF32, IFCI_SCREENED, PRECISIONS,
    CIProblem, Handle, IfciEnergy, IfciError, StringTables, SystemArrays, ifci_energy,
    body_subsets, davidson_opts,
    ifci_build_strings, ifci_davidson_batched, ifci_frozen_core, ifci_h_elements, ifci_hdiag, ifci_increments,
    ifci_num_subsets, ifci_rdm_backward, ifci_sigma, ifci_sigma_noalloc, ifci_sigma_noalloc_max_bytes,
    ifci_wait_selftest,
    ifci_string_counts, ifci_hbci_batched, reference_determinant,
)
