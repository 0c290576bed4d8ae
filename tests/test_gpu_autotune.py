"""The autotuner of the batched solve's launch parameters (max_space,
det_budget, graph_iters): every candidate it times reproduces the first
candidate's energies, the choice is one of the timed candidates, and a
second call reads it back from the cache file."""
import os

import pytest
import torch

from synth import chain_24_uneven

import paper_2307_10675_gb300 as ifci
from paper_2307_10675_gb300 import autotune

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def test_autotune_chooses_a_timed_candidate_and_caches_it(tmp_path):
    chain = chain_24_uneven()
    sysd = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    sets = [(0, 1), (3, 4, 5), (8, 11, 12), (2, 9, 20)]
    cache = os.path.join(tmp_path, "tune.json")
    grid = {"max_space": [12, 8], "det_budget": [1 << 28, 1 << 31], "graph_iters": [0, 4]}
    with ifci.Handle(0, 0) as h:
        a = autotune.autotune(h, sysd, sets, "fp64e", grid=grid, cache=cache)
        b = autotune.autotune(h, sysd, sets, "fp64e", grid=grid, cache=cache)
    assert not a["cached"] and b["cached"] and a["params"] == b["params"]
    timed = [c["params"] for c in a["table"]]
    assert a["params"] in timed
    assert all(c["accepted"] for c in a["table"])
    assert max(c["max_abs_energy_deviation"] for c in a["table"]) < 1e-8
