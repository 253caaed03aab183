"""The stored full-size results (tests/golden/full_size_digests.json) against
the oracle itself, on the cases it finishes in seconds.

The GPU parity tests compare the CUDA path with these stored digests; this
test checks on the CPU that the file still holds what its generating script
(make_full_size_digests.py, which calls only the oracle) gives: the same
input recipe, thinned image digest, lowering count and last changing phase."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_1603_09180_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "full_size_digests.json")) as f:
    CASES = json.load(f)["cases"]


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def cheapest(n):
    cost = lambda r: r["h"] * r["w"] * max(1, r["rounds"])
    return sorted(CASES, key=lambda k: cost(CASES[k]))[:n]


@pytest.mark.parametrize("name", cheapest(6) + ["batch_512_u8_s0_l0"])
def test_stored_case_matches_the_oracle(name):
    r = CASES[name]
    img = synth.value_noise_image(r["h"], r["w"], r["dtype"], seed=r["seed"], vmax=r["vmax"])
    assert digest(img) == r["input_sha256"]
    out, st = oracle.thin(img, r["lam"])
    assert digest(out) == r["sha256"]
    assert st["lowered"] == r["lowered"] and st["last_change_phase"] == r["last_change_phase"]
    assert st["converged"] == 1


def test_every_workload_is_covered():
    kinds = {}
    for k in CASES:
        kinds[k.split("_")[0]] = kinds.get(k.split("_")[0], 0) + 1
    assert kinds == {"single": 1, "batch": 192, "large": 4, "uneven": 1024}
    for k, r in CASES.items():
        assert len(r["sha256"]) == 64 and r["lowered"] >= 0 and r["rounds"] >= 1, k
