"""ifci_sigma_noalloc: the sigma entry point for callers that cannot allocate
device memory (its scratch is one fixed device array inside the library).

Checked through the C ABI against ifci_sigma on two calls in a row, with the
FP64 tolerance of the other sigma tests.  This file is collected last so that
a run stopping at the first failure has run every other test already; it
sets up everything it needs itself, so it also passes alone in a fresh process.
"""
import math

import numpy as np
import pytest
import torch

from synth import chain_4x2, chain_24_uneven, random_ci_vector

import paper_2307_10675_gb300 as ifci

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _problem(handle, chain, X):
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    h1, eri, _ = ifci.ifci_frozen_core(handle, sysa, X)
    t = ifci.ifci_build_strings(handle, h1.shape[0], len(X))
    return t, h1, eri


def test_noalloc_sigma_matches_ifci_sigma_on_consecutive_calls():
    torch.cuda.set_device(DEV)
    with ifci.Handle(0, 0) as h:
        t, h1, eri = _problem(h, chain_4x2(), (0, 1, 2, 3))          # CAS(8e,8o), 4900 dets
        assert 8 * 36 * 36 + 16 * 36 * t.nstr ** 2 < ifci.ifci_sigma_noalloc_max_bytes()
        outs = []
        for seed in (5, 6):                                          # two calls in a row
            c = torch.tensor(random_ci_vector(t.nstr, t.nstr, seed=seed), device=DEV)
            ref = ifci.ifci_sigma(h, t, h1, eri, c)
            got = torch.full_like(c, float("nan"))
            assert ifci.ifci_sigma_noalloc(t, h1, eri, c, got) == 0
            torch.cuda.synchronize()
            np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=1e-10)
            outs.append(got.cpu().numpy())
        assert not np.allclose(outs[0], outs[1])


def test_noalloc_sigma_second_shape_after_first():
    """A different (smaller) problem right after a larger one uses the same array."""
    with ifci.Handle(0, 0) as h:
        for X in [(0, 1), (8, 11, 12)]:
            t, h1, eri = _problem(h, chain_24_uneven(), X)
            c = torch.tensor(random_ci_vector(t.nstr, t.nstr, seed=9), device=DEV)
            ref = ifci.ifci_sigma(h, t, h1, eri, c)
            got = torch.empty_like(c)
            assert ifci.ifci_sigma_noalloc(t, h1, eri, c, got) == 0
            torch.cuda.synchronize()
            np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=1e-10)


def test_noalloc_sigma_rejects_problems_beyond_the_array():
    with ifci.Handle(0, 0) as h:
        chain = chain_24_uneven()
        six = tuple(b for b, s in enumerate(chain.body_sizes) if s == 6)[:3]   # CAS(6e,18o)
        t, h1, eri = _problem(h, chain, six)
        need = 16 * 171 * t.nstr ** 2
        assert need > ifci.ifci_sigma_noalloc_max_bytes()
        c = torch.zeros(t.nstr * t.nstr, dtype=torch.float64, device=DEV)
        out = torch.zeros_like(c)
        assert ifci.ifci_sigma_noalloc(t, h1, eri, c, out) == 1      # IFCI_ERR_INVALID_ARG


def test_noalloc_sigma_allocates_nothing_once_set_up():
    """After one call on the device (which loads the library's device code and
    the fixed array), later calls succeed while the caller's allocator holds
    nearly all free device memory, and leave the free memory unchanged."""
    torch.cuda.set_device(DEV)
    with ifci.Handle(0, 0) as h:
        t, h1, eri = _problem(h, chain_4x2(), (0, 1, 2))
        c = torch.tensor(random_ci_vector(t.nstr, t.nstr, seed=3), device=DEV)
        ref = ifci.ifci_sigma(h, t, h1, eri, c)
        out = torch.empty_like(c)
        assert ifci.ifci_sigma_noalloc(t, h1, eri, c, out) == 0      # set-up call
        torch.cuda.synchronize()
        free, _ = torch.cuda.mem_get_info()
        got = torch.full_like(c, float("nan"))
        hold = torch.empty(max(0, free - (512 << 20)), dtype=torch.uint8, device=DEV)   # leave 512 MiB
        try:
            torch.cuda.synchronize()
            before, _ = torch.cuda.mem_get_info()
            assert ifci.ifci_sigma_noalloc(t, h1, eri, c, got) == 0
            torch.cuda.synchronize()
            after, _ = torch.cuda.mem_get_info()
            assert after == before
            np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=1e-10)
        finally:
            del hold
            torch.cuda.empty_cache()
