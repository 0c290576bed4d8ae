"""CPU-side checks of the C-ABI library: it builds, loads, exports every
declared entry point, and its host-only counting functions are right."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "ifci.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*|size_t|long long)\s*\*?\s*(ifci_\w+)\s*\(",
                                 src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["ifci_build_strings", "ifci_sigma", "ifci_davidson_batched", "ifci_increments",
                     "ifci_rdm_backward", "ifci_handle_create", "ifci_handle_destroy"]:
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2307_10675_gb300 import _capi
    lib = _capi.load()
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert set(_capi.EXPORTS) <= set(_declared_functions())


@pytest.mark.parametrize("norb,m", [(2, 1), (6, 3), (14, 7), (18, 3), (31, 1)])
def test_string_counts(norb, m):
    from paper_2307_10675_gb300 import ifci_string_counts
    nstr, nexc = ifci_string_counts(norb, m)
    assert nstr == math.comb(norb, m)
    assert nexc == m * (norb - m + 1)


def test_string_counts_reject_out_of_range():
    from paper_2307_10675_gb300 import IfciError, ifci_string_counts
    for args in [(32, 3), (0, 0), (5, 6), (-1, 0)]:
        with pytest.raises(IfciError):
            ifci_string_counts(*args)


@pytest.mark.parametrize("nbody,order", [(4, 2), (24, 3), (40, 3), (21, 4)])
def test_num_subsets_and_order(nbody, order):
    from paper_2307_10675_gb300 import body_subsets, ifci_num_subsets
    n = ifci_num_subsets(nbody, order)
    assert n == sum(math.comb(nbody, k) for k in range(1, order + 1))
    if nbody <= 24:
        assert len(body_subsets(nbody, order)) == n


def test_handle_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2307_10675_gb300 import Handle, IfciError
    with pytest.raises(IfciError):
        Handle(0, 0)
