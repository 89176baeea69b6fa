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


@pytest.mark.parametrize("dims,n", [((3, 3), 512), ((4, 4), 1 << 16), ((3, 3, 3), 1200), ((6, 6), 400)])
def test_gap_thresholds_and_gaps(hp, obox, dims, n):
    """Energy-gap thresholds T > 1 (Section 2.1) and the gap E2 - E1 itself (Appendix C returns
    E1 - E2): plain scan exact; pruned scan exact in the phenotype and in the gap clipped at T."""
    s = hp.Structs(dims)
    o = obox(dims)
    ids = np.arange(n, dtype=np.uint64) if n == (1 << s.N) else inputs.sample_ids(s.N, n, seed=23)
    t = ids_tensor(ids)
    _, want_aux, want_gap = o.phenotypes(ids, aux=True, gaps=True)
    rnd = conformations_of_classes(s, (inputs.sample_ids(20, n * 2, seed=9) % np.uint64(s.S)).astype(np.int64).reshape(n, 2), 4)
    best = conformations_of_classes(s, want_aux[:, None], 2)
    for T in (1, 2, 3, 10, 13, 23, 40):
        want = np.where(want_gap >= T, want_aux, -1)  # the oracle's threshold rule, pinned on the CPU
        phen, aux, gap = hp.sequence_scan(s, t, aux=True, gap_threshold=T, gaps=True)
        np.testing.assert_array_equal(phen.cpu().numpy(), want)
        np.testing.assert_array_equal(aux.cpu().numpy(), want_aux)
        np.testing.assert_array_equal(gap.cpu().numpy(), want_gap)
        for cand in (best, rnd):
            cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
            p2, g2 = hp.sequence_scan(s, t, cand=torch.from_numpy(cand).cuda(), gap_threshold=T, gaps=True,
                                      counters=cnt)
            np.testing.assert_array_equal(p2.cpu().numpy(), want)
            np.testing.assert_array_equal(g2.cpu().numpy(), np.minimum(want_gap, T))
            assert int(cnt[0]) <= n * s.S_dir
        # without the gap output the threshold-T phenotypes are the same
        np.testing.assert_array_equal(hp.sequence_scan(s, t, gap_threshold=T).cpu().numpy(), want)


def test_threshold_1_gap_variant_equals_plain_scan(hp):
    s = hp.Structs((3, 3, 3))
    t = ids_tensor(inputs.sample_ids(27, 3000, seed=41))
    p1, a1 = hp.sequence_scan(s, t, aux=True)
    p2, a2, g2 = hp.sequence_scan(s, t, aux=True, gaps=True)
    assert torch.equal(p1, p2) and torch.equal(a1, a2)
    assert torch.equal(p2 >= 0, g2 >= 1)


def test_single_conformation_box_gap(hp):
    s = hp.Structs((2, 2))
    t = ids_tensor(np.arange(16, dtype=np.uint64))
    phen, gap = hp.sequence_scan(s, t, gap_threshold=1000, gaps=True)
    assert (phen == 0).all() and (gap == np.iinfo(np.int32).max).all()


@pytest.mark.parametrize("dims,begin,count", [((4, 4), 0, 1 << 16), ((3, 3, 3), 3 << 20, 1500), ((4, 5), 12345, 777)])
def test_map_at_threshold_above_1(hp, obox, dims, begin, count):
    """hp_phenotype_map with gap_threshold > 1 (the tiled kernel's gap variant) against the oracle:
    one tile (4x4), several tiles and ragged aligned blocks (3x3x3, 4x5), with aux."""
    s = hp.Structs(dims)
    o = obox(dims)
    ids = np.arange(begin, begin + count, dtype=np.uint64)
    _, want_aux, want_gap = o.phenotypes(ids, aux=True, gaps=True)
    for T in (2, 10, 23):
        want = np.where(want_gap >= T, want_aux, -1)
        aux = torch.empty(count, dtype=torch.int32, device="cuda")
        got = hp.phenotype_map(s, begin, count, aux=aux, gap_threshold=T)
        np.testing.assert_array_equal(got.cpu().numpy(), want)
        np.testing.assert_array_equal(aux.cpu().numpy(), want_aux)


@pytest.mark.parametrize("dims,begin,count,sample", [((3, 3, 3), 5 << 22, 1 << 20, 1), ((6, 6), 7 << 30, 1 << 22, 64),
                                                     ((2, 3, 4), 0, 1 << 24, 256)])
def test_tiled_map_thresholds_match_the_scan(hp, dims, begin, count, sample):
    """The tiled map at T > 1 against the per-sequence scan at T (checked against the oracle above)
    on many tiles of conformations: 3x3x3 (404 tiles), 6x6 (224), 2x3x4 (even N, whole space)."""
    s = hp.Structs(dims)
    ids = torch.arange(begin, begin + count, sample, dtype=torch.int64, device="cuda")
    m1 = hp.phenotype_map(s, begin, count)
    for T in (2, 5, 13):
        aux = torch.empty(count, dtype=torch.int32, device="cuda")
        mT = hp.phenotype_map(s, begin, count, aux=aux, gap_threshold=T)
        want, want_aux = hp.sequence_scan(s, ids, aux=True, gap_threshold=T)
        assert torch.equal(mT[::sample], want) and torch.equal(aux[::sample], want_aux)
        assert bool(((mT == -1) | (mT == m1)).all())  # raising T only turns folders into non-folders
        m1 = mT


def test_full_3x3x3_map_at_threshold_3(hp):
    """Whole 3x3x3 space at T = 3: the reversal half enumeration and its mirrored writes."""
    s = hp.Structs((3, 3, 3))
    m = hp.phenotype_map(s, gap_threshold=3)
    ids = torch.from_numpy(inputs.sample_ids(27, 1 << 15, seed=77).view(np.int64)).cuda()
    assert torch.equal(m[ids], hp.sequence_scan(s, ids, gap_threshold=3))
    g = ids
    r = torch.zeros_like(g)
    for i in range(27):
        r |= ((g >> i) & 1) << (26 - i)
    assert torch.equal(m[ids], m[r])
