"""Host-side arithmetic of bench.py (no GPU): work models and the per-class
roofline summary it prints."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from synth import chain_24_uneven  # noqa: E402


def test_cost_model_counts():
    nd, fl = bench.cost_of(18, 3)
    assert nd == 665856 and fl == 2.0 * 665856 * 171 ** 2
    # executed FP16 work of one CAS(6e,18o) sigma: 15 products, 5202 row tiles, N padded to 96 + 80, K to 176
    assert bench.executed_oz_flops(18, 3) == 15.0 * 2.0 * (816 * 7) * 128 * (96 + 80) * 176


def test_class_rooflines_fields_and_scaling():
    subs = bench.subset_sizes(chain_24_uneven(), 3)
    iters = np.full(len(subs), 20, dtype=np.int32)
    out = bench.class_rooflines(subs, iters, {"scatter": 500.0, "gather": 100.0, "vector": 1300.0}, 1,
                                6791.4, 1.10)
    assert set(out) == {"scatter", "davidson_vectors"}
    assert out["scatter"]["bound"] == "hbm" and 0 < out["scatter"]["frac"] < 10
    v = out["davidson_vectors"]
    assert v["bound"] == "fp64_alu" and v["achieved"] > 0 and 0 < v["hbm_frac"] < 10
    # twice the time, half the rate
    out2 = bench.class_rooflines(subs, iters, {"scatter": 1000.0, "gather": 200.0, "vector": 2600.0}, 1,
                                 6791.4, 1.10)
    assert math.isclose(out2["scatter"]["achieved"] * 2, out["scatter"]["achieved"])
    assert math.isclose(out2["davidson_vectors"]["achieved"] * 2, v["achieved"])
    assert bench.class_rooflines(subs, iters, {}, 1, 6791.4, 1.10) == {}


def test_contracted_pairs_of_decoupled_groups():
    """Three bodies far apart contract only their own pairs; three adjacent
    bodies contract every pair of their union."""
    from synth import chain_40_uneven
    c = chain_40_uneven()
    C = bench.body_coupling(c)
    s = c.body_sizes
    far = (0, 19, 39)
    assert bench.contracted_pairs(far, s, C) == sum(s[b] * (s[b] + 1) // 2 for b in far)
    near = (10, 11, 12)
    n = sum(s[b] for b in near)
    assert bench.contracted_pairs(near, s, C) == n * (n + 1) // 2
