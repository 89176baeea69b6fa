"""The stored oracle map digests (tests/golden/map_digests.json) are well formed and reproducible: the
4x5 case, cheap on the CPU, is recomputed with the oracle and must give the same digests."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "map_digests.json")
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_map_digests as mk  # noqa: E402


def test_digest_file_is_well_formed():
    with open(GOLDEN) as f:
        data = json.load(f)
    assert "_source" in data
    for name, case in data.items():
        if name.startswith("_"):
            continue
        n = case["count"]
        chunks = (n + (1 << case["chunk_bits"]) - 1) >> case["chunk_bits"]
        assert len(case["phen"]) == len(case["aux"]) == chunks, name
        d = case["designability"]
        assert 0 <= d["minus1"] <= n and d["designable"] <= case["S"]


def test_4x5_digests_recomputed_by_the_oracle():
    with open(GOLDEN) as f:
        case = json.load(f)["4x5"]
    import oracle

    dims, ids, _ = mk.case_ids("4x5")
    phen, aux = oracle.Box(dims).phenotypes(ids, aux=True)
    assert mk.chunk_digests(phen, case["chunk_bits"]) == case["phen"]
    assert mk.chunk_digests(aux, case["chunk_bits"]) == case["aux"]
    assert mk.histogram(phen, case["S"]) == case["designability"]
    assert np.unique(phen).shape[0] > 10
