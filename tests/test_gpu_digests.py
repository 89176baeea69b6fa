"""Whole-map parity at full size: GPU maps compared, chunk by chunk, with digests of the oracle's
maps written by tests/golden/make_map_digests.py (which calls only oracle/).  Covered: every id of
4x5, 5x5 and 2x3x4, a 2^20-id block of 3x3x3, and seeded samples of 3x3x3 and of four 6x6 shards;
phenotypes and the lowest-index minimiser (aux) both, plus the designability of each case."""
import hashlib
import json
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "map_digests.json")
sys.path.insert(0, os.path.join(HERE, "golden"))


@pytest.fixture(scope="module")
def hp():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2008_05612_gb300 as m

    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available for a gpu-marked test")
    return m


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def chunk_digests(a, chunk_bits):
    a = np.ascontiguousarray(a, dtype="<i4")
    step = 1 << chunk_bits
    return [hashlib.sha256(a[i:i + step].tobytes()).hexdigest()[:16] for i in range(0, a.shape[0], step)]


def compare(name, what, got, want_digests, chunk_bits):
    have = chunk_digests(got, chunk_bits)
    bad = [i for i, (a, b) in enumerate(zip(have, want_digests)) if a != b]
    assert len(have) == len(want_digests)
    assert not bad, f"{name} {what}: chunks {bad[:10]} (of 2^{chunk_bits} entries each) differ from the oracle"


CASES = [c for c in ("4x5", "5x5", "2x3x4", "3x3x3blk", "3x3x3smp", "6x6smp")]


@pytest.mark.parametrize("name", CASES)
def test_gpu_map_equals_oracle_digests(hp, name):
    data = golden()
    if name not in data:
        pytest.skip(f"no oracle digest for {name} in {GOLDEN}")
    case = data[name]
    import make_map_digests as mk  # the same id recipes (seeded generators only)

    dims, ids, _ = mk.case_ids(name)
    s = hp.Structs(tuple(dims))
    assert (s.N, s.S, s.S_dir) == (case["N"], case["S"], case["S_dir"])
    n = ids.shape[0]
    if name.endswith("smp"):
        t = torch.from_numpy(ids.view(np.int64)).cuda()
        phen, aux = hp.sequence_scan(s, t, aux=True)
    else:
        begin = int(ids[0])
        assert (ids == np.arange(begin, begin + n, dtype=np.uint64)).all()
        phen = torch.empty(n, dtype=torch.int32, device="cuda")
        aux = torch.empty(n, dtype=torch.int32, device="cuda")
        hp.phenotype_map(s, begin, n, out=phen, aux=aux)
    hist = hp.designability(phen, s.S).cpu().numpy().astype(np.uint64)
    phen, aux = phen.cpu().numpy(), aux.cpu().numpy()
    compare(name, "phenotypes", phen, case["phen"], case["chunk_bits"])
    compare(name, "aux", aux, case["aux"], case["chunk_bits"])
    d = case["designability"]
    assert int(hist[s.S]) == d["minus1"] and int((hist[: s.S] > 0).sum()) == d["designable"]
    assert int(hist[: s.S].max()) == d["max"]
    assert hashlib.sha256(np.ascontiguousarray(hist, dtype="<u8").tobytes()).hexdigest()[:16] == d["sha"]
