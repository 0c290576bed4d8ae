"""Connected n-body screening (ifci_davidson_opts_t.cnb_threshold; Methods,
screening paragraph) through the C ABI.

* 4 x 2 chain to 4 bodies with a threshold that keeps the three largest pair
  increments: the kept sets, their increments and the total equal the
  oracle's screened expansion.
* 40-body chain to 3 bodies at the paper's C = 10^-4.6 Ha: the kept 3-body
  sets are exactly those whose pair graph (|eps_ab| >= C, from the call's
  own pair increments) is connected; a kept set's energy equals the
  unscreened run's; screened sets report IFCI_SCREENED and NaN.
* The gradient of the screened total (inclusion pattern fixed) obeys
  Euler's identity, sum h dE/dh + sum V dE/dV = E_total.
"""
import itertools

import numpy as np
import pytest
import torch

from oracle import fci
from synth import chain_4x2, chain_24_uneven, chain_40_uneven

import paper_2307_10675_gb300 as ifci

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
C_PAPER = 10 ** -4.6


def _system(chain):
    return ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))


def _connected(X, pair_eps, C):
    seen, stack = {X[0]}, [X[0]]
    while stack:
        a = stack.pop()
        for b in X:
            if b not in seen and abs(pair_eps[tuple(sorted((a, b)))]) >= C:
                seen.add(b)
                stack.append(b)
    return len(seen) == len(X)


@pytest.mark.parametrize("prec", ["fp64", "fp64e"])
def test_screened_expansion_matches_the_oracle(prec):
    s = chain_4x2()
    _, _, eps_full, _ = fci.ifci_energies(s, 4)
    mags = sorted(abs(v) for X, v in eps_full.items() if len(X) == 2)
    C = 0.5 * (mags[2] + mags[3])
    e0, ex, eps, total = fci.ifci_energies(s, 4, cnb=C)
    with ifci.Handle(0, 0) as h:
        out = ifci.ifci_increments(h, _system(s), 4, ifci.davidson_opts(prec, r_tol=1e-8, e_tol=1e-12,
                                                                          cnb_threshold=C))
    subs = ifci.body_subsets(4, 4)
    for i, X in enumerate(subs):
        if X in ex:
            assert out["status"][i] == 0
            assert out["e_x"][i] == pytest.approx(ex[X], abs=1e-8), X
        else:
            assert out["status"][i] == ifci.IFCI_SCREENED and np.isnan(out["e_x"][i]), X
        assert out["eps"][i] == pytest.approx(eps[X], abs=1e-8), X
    assert out["e_total"] == pytest.approx(total, abs=1e-8)


def test_paper_threshold_on_the_40_body_chain():
    chain = chain_40_uneven()
    opts = dict(r_tol=1e-7, e_tol=1e-11, max_iter=300)
    with ifci.Handle(0, 0) as h:
        sysd = _system(chain)
        full = ifci.ifci_increments(h, sysd, 3, ifci.davidson_opts("fp64e", **opts))
        scr = ifci.ifci_increments(h, sysd, 3, ifci.davidson_opts("fp64e", cnb_threshold=C_PAPER, **opts))
    subs = ifci.body_subsets(40, 3)
    pair_eps = {X: scr["eps"][i] for i, X in enumerate(subs) if len(X) == 2}
    nkept = 0
    for i, X in enumerate(subs):
        if len(X) < 3:
            assert scr["status"][i] == 0
            assert scr["e_x"][i] == full["e_x"][i]
            continue
        keep = _connected(X, pair_eps, C_PAPER)
        margin = min(abs(abs(pair_eps[p]) - C_PAPER) for p in itertools.combinations(X, 2))
        if margin < 1e-9:
            continue                                   # a pair on the threshold: either choice is valid
        if keep:
            nkept += 1
            assert scr["status"][i] == 0
            assert scr["e_x"][i] == pytest.approx(full["e_x"][i], abs=1e-9), X
        else:
            assert scr["status"][i] == ifci.IFCI_SCREENED and np.isnan(scr["e_x"][i]) and scr["eps"][i] == 0.0
    assert 0 < nkept < 9880
    assert scr["e_total"] == pytest.approx(scr["e0"] + float(np.sum(scr["eps"])), abs=1e-9)


def test_screened_gradient_obeys_euler_identity():
    chain = chain_24_uneven()
    with ifci.Handle(0, 0) as h:
        sysd = _system(chain)
        opts = ifci.davidson_opts("fp64e", r_tol=1e-7, e_tol=1e-11, cnb_threshold=C_PAPER)
        out = ifci.ifci_increments(h, sysd, 3, opts)
        assert np.any(out["status"] == ifci.IFCI_SCREENED)
        dh, dV = ifci.ifci_rdm_backward(h, sysd, 3, 1.0, opts)
        torch.cuda.synchronize()
    euler = float(np.sum(chain.h * dh.cpu().numpy()) + np.sum(chain.eri_packed() * dV.cpu().numpy()))
    assert euler == pytest.approx(out["e_total"], abs=1e-7)
