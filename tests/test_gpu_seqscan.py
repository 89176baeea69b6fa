"""Per-sequence scan (plain and bound-pruned) against the oracle and the exhaustive kernel (GPU)."""
import numpy as np
import pytest

from paper_2008_05612_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hp():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2008_05612_gb300 as m

    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available for a gpu-marked test")
    return m


def conformations_of_classes(structs, classes, k):
    """[n, k] conformation indices: every conformation of each listed class, padded with -1."""
    _, _, cls = structs.export()
    first = np.searchsorted(cls, np.arange(structs.S))
    out = np.full((len(classes), k), -1, dtype=np.int32)
    for r, row in enumerate(classes):
        j = 0
        for c in row:
            if c < 0:
                continue
            s = first[c]
            while s < structs.S_dir and cls[s] == c and j < k:
                out[r, j] = s
                j += 1
                s += 1
    return out


def ids_tensor(ids):
    return torch.from_numpy(np.asarray(ids, dtype=np.uint64).view(np.int64)).cuda()


def test_plain_scan_full_4x4(hp, obox):
    s = hp.Structs((4, 4))
    ids = np.arange(1 << 16, dtype=np.uint64)
    phen, aux = hp.sequence_scan(s, ids_tensor(ids), aux=True)
    want, want_aux = obox((4, 4)).full_map(aux=True)
    np.testing.assert_array_equal(phen.cpu().numpy(), want)
    np.testing.assert_array_equal(aux.cpu().numpy(), want_aux)


@pytest.mark.parametrize("dims,n", [((3, 3, 3), 1500), ((6, 6), 600), ((2, 3, 4), 800), ((5, 5), 2000)])
def test_plain_and_pruned_scan_sampled(hp, obox, dims, n):
    s = hp.Structs(dims)
    ids = inputs.sample_ids(s.N, n, seed=71)
    want, want_aux = obox(dims).phenotypes(ids, aux=True)
    t = ids_tensor(ids)
    cnt_plain = torch.zeros(2, dtype=torch.int64, device="cuda")
    phen, aux = hp.sequence_scan(s, t, aux=True, counters=cnt_plain)
    np.testing.assert_array_equal(phen.cpu().numpy(), want)
    np.testing.assert_array_equal(aux.cpu().numpy(), want_aux)
    # candidates = the true minimiser's class (best case) and random classes (worst case): both exact
    best = conformations_of_classes(s, want_aux[:, None], 2)
    rnd = conformations_of_classes(s, (inputs.sample_ids(20, n * 3, seed=5) % np.uint64(s.S)).astype(np.int64).reshape(n, 3), 6)
    for cand in (best, rnd):
        cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
        p2, a2 = hp.sequence_scan(s, t, cand=torch.from_numpy(cand).cuda(), aux=True, counters=cnt)
        np.testing.assert_array_equal(p2.cpu().numpy(), want)
        np.testing.assert_array_equal(a2.cpu().numpy(), want_aux)
        assert int(cnt[0]) <= int(cnt_plain[0])
    assert int(cnt_plain[0]) == n * s.S_dir


def test_pruned_scan_matches_exhaustive_block(hp):
    s = hp.Structs((3, 3, 3))
    base = 5 << 22
    block = hp.phenotype_map(s, base, 1 << 16, aux=torch.empty(1 << 16, dtype=torch.int32, device="cuda"))
    ids = np.arange(base, base + (1 << 16), dtype=np.uint64)[::7]
    phen = hp.sequence_scan(s, ids_tensor(ids))
    np.testing.assert_array_equal(phen.cpu().numpy(), block.cpu().numpy()[::7])
