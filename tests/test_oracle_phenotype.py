"""Pins for the oracle's ground-state search (Section 2.1, Appendix C semantics) and readings."""
import numpy as np
import pytest

import oracle
from paper_2008_05612_gb300 import inputs
from tests import _brute


@pytest.mark.parametrize("dims", [(2, 3), (3, 3), (2, 4), (2, 2, 2)])
def test_full_map_equals_brute_force(obox, dims):
    b = obox(dims)
    want, S = _brute.phenotype_map(dims)
    got = b.full_map()
    assert S == b.S
    np.testing.assert_array_equal(got, want)


def test_2x2_single_structure_always_folds(obox):
    """One fold only: it is always the unique minimum (the plain definition), even at E = 0."""
    b = obox((2, 2))
    assert (b.full_map() == 0).all()


def test_2x3_hand_worked_readings(obox):
    """Hand-derived 2x3 cases.  Conformations: U {(0,5),(1,4)}, zig-zag {(0,3),(2,5)},
    hook K {(0,5),(2,5)} and its reverse K^R {(0,3),(0,5)} (one class).
      h = H at 0 only:   U -10, Z -10, K -10, K^R -20 -> B and C give K's class; A (K only) ties -> -1.
      h = H at 0 and 5:  U -23, Z -20, K -33, K^R -33 -> B: -1 (two conformations tie); C and A: K.
      h = H at 5 only:   U -10, Z -10, K -20, K^R -10 -> K in every reading.
      all P / all H: every fold ties -> -1."""
    b = obox((2, 3))
    _, cls, contacts, _ = b.export()
    sets = [tuple(sorted(map(tuple, c.tolist()))) for c in contacts]
    k = cls[sets.index(((0, 5), (2, 5)))]
    kr = cls[sets.index(((0, 3), (0, 5)))]
    assert k == kr
    seqs = np.array([0b000001, 0b100001, 0b100000, 0, 0b111111], dtype=np.uint64)
    A = b.phenotypes(seqs, reading=oracle.READING_A)
    B = b.phenotypes(seqs, reading=oracle.READING_B)
    C = b.phenotypes(seqs, reading=oracle.READING_C)
    # which orientation is canonical decides reading A for the first case; K^R wins at -20
    assert B.tolist() == [k, -1, k, -1, -1]
    assert C.tolist() == [k, k, k, -1, -1]
    assert A[2] == k and A[3] == -1 and A[4] == -1
    # energy gaps E2 - E1 under B (Appendix C returns their negatives): -20 vs -10, a tie at -33,
    # -20 vs -10, and two all-equal rows; a gap of 10 folds up to threshold 10 and not at 11
    _, gaps = b.phenotypes(seqs, gaps=True)
    assert gaps.tolist() == [10, 0, 10, 0, 0]
    assert b.phenotypes(seqs, gap=10).tolist() == [k, -1, k, -1, -1]
    assert b.phenotypes(seqs, gap=11).tolist() == [-1, -1, -1, -1, -1]


@pytest.mark.parametrize("dims", [(4, 4), (2, 4), (3, 4)])
def test_reversal_invariance(obox, dims):
    """Under reading B, E(h^R, s) = E(h, s^R) and the conformation set is closed under reversal,
    so P(h^R) = P(h) (the map symmetry noted in Appendix B)."""
    b = obox(dims)
    m = b.full_map()
    N = b.N
    g = np.arange(1 << N, dtype=np.int64)
    r = np.zeros_like(g)
    for i in range(N):
        r |= ((g >> i) & 1) << (N - 1 - i)
    np.testing.assert_array_equal(m, m[r])


def test_gap_threshold_monotone(obox):
    """Raising the energy-gap threshold (Section 2.1) can only turn folders into non-folders."""
    b = obox((4, 4))
    m1 = b.full_map(gap=1)
    for T in (2, 5, 10, 23):
        mT = b.full_map(gap=T)
        assert ((mT == -1) | (mT == m1)).all()
        assert (mT >= 0).sum() <= (m1 >= 0).sum()
        m1 = mT


@pytest.mark.parametrize("dims", [(2, 3), (3, 3), (2, 2, 2)])
def test_gaps_and_thresholds_equal_brute_force(obox, dims):
    """E2 - E1 and the phenotype at energy-gap thresholds T > 1 (Section 2.1; Appendix C keeps the
    lowest and second-lowest energy) against the brute force: a genotype folds iff E2 - E1 >= T."""
    b = obox(dims)
    first, want_gaps, S = _brute.gap_map(dims)
    phen, aux, gaps = b.full_map(aux=True, gaps=True)
    assert aux.tolist() == first
    assert gaps.tolist() == want_gaps
    g = np.array(want_gaps)
    for T in (1, 3, 10, 13, 20, 23, 33):
        want = np.where(g >= T, np.array(first), -1)
        np.testing.assert_array_equal(b.full_map(gap=T), want)


def test_single_conformation_gap_is_unbounded(obox):
    b = obox((2, 2))
    phen, gaps = b.full_map(gap=1000, gaps=True)
    assert (phen == 0).all() and (gaps == np.iinfo(np.int32).max).all()


def test_aux_is_lowest_index_minimiser(obox):
    b = obox((4, 4))
    ids = np.arange(1 << 16, dtype=np.uint64)[::97]
    phen, aux = b.phenotypes(ids, aux=True)
    _, cls, _, _ = b.export()
    for g, p, a in zip(ids.tolist()[:200], phen.tolist(), aux.tolist()):
        es = [b.energy(g, s) for s in range(b.S_dir)]
        first = int(np.argmin(es))
        assert a == cls[first]
        if p >= 0:
            assert p == a


def test_3x3x3_folding_fraction_matches_paper(obox):
    """Section 3.2 / Table 4: 4.76% of 3x3x3 HP sequences have a unique ground state (Li et al. 4.75%).
    A seeded sample of 4000 ids must land within 4 binomial standard errors under reading B,
    and reading A (one orientation per class) must not."""
    b = obox((3, 3, 3))
    ids = inputs.sample_ids(27, 4000, seed=3)
    f = float((b.phenotypes(ids, reading=oracle.READING_B) >= 0).mean())
    se = np.sqrt(0.0476 * (1 - 0.0476) / len(ids))
    assert abs(f - 0.0476) < 4 * se
    ids_a = ids[:1500]
    fa = float((b.phenotypes(ids_a, reading=oracle.READING_A) >= 0).mean())
    assert abs(fa - 0.0476) > 6 * np.sqrt(0.0476 * 0.9524 / len(ids_a))
