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


def _header_struct_fields(name):
    src = open(os.path.join(ROOT, "include", "ifci.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        parts = [p.strip() for p in decl.split(",") if p.strip()]
        if not parts:
            continue
        fields.append(parts[0].split()[-1].lstrip("*").split("[")[0])
        fields += [p.lstrip("*").split("[")[0].strip() for p in parts[1:]]
    return fields


@pytest.mark.parametrize("cname,pyname", [("ifci_davidson_opts_t", "DavidsonOpts"), ("ifci_problem_t", "Problem"),
                                           ("ifci_system_t", "System"), ("ifci_strings_t", "Strings"),
                                           ("ifci_hbci_opts_t", "HbciOpts")])
def test_binding_structs_follow_the_header(cname, pyname):
    """The ctypes mirrors list the header's fields in the header's order."""
    from paper_2307_10675_gb300 import _capi
    fields = [f[0] for f in getattr(_capi, pyname)._fields_]
    assert fields == _header_struct_fields(cname)


def test_davidson_default_opts_from_the_library():
    from paper_2307_10675_gb300 import _capi
    o = _capi.DavidsonOpts()
    _capi.load().ifci_davidson_default_opts(ctypes.byref(o))
    assert (o.precision, o.max_iter, o.max_space) == (_capi.IFCI_FP64, 100, 12)
    assert (o.e_tol, o.r_tol) == (1e-10, 1e-6)
    assert o.hi_precision == _capi.IFCI_FP64E
    assert o.det_budget == 0 and o.graph_iters == 0
    assert o.sector_passes == 0 and o.decouple_tol == 1e-5
    assert o.cnb_threshold == 0.0
    assert (o.hbci_max_rounds, o.hbci_eps1, o.hbci_eps2) == (0, 1e-3, 1e-6)


def test_sigma_flag_matches_the_header():
    from paper_2307_10675_gb300 import _capi
    src = open(os.path.join(ROOT, "include", "ifci.h")).read()
    m = re.search(r"#define\s+IFCI_SIGMA_SPIN_SYMMETRIC\s+(0x[0-9a-fA-F]+|\d+)", src)
    assert m and int(m.group(1), 0) == _capi.IFCI_SIGMA_SPIN_SYMMETRIC
