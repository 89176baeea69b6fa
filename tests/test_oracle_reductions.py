"""Pins for the oracle's map reductions: designability (Section 2.3), Eq. 2 numerators and
robustness / phi_del, and neutral-network components."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2008_05612_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")


def synthetic_map(N, S, seed):
    """A seeded map with neutral plateaus: phenotype from the top bits, holes set to -1."""
    g = np.arange(1 << N, dtype=np.uint64)
    r = inputs.splitmix64(g >> np.uint64(max(N - 6, 0)) ^ np.uint64(seed))
    p = (r % np.uint64(S)).astype(np.int32)
    hole = inputs.splitmix64(g ^ np.uint64(seed * 7 + 1)) % np.uint64(5) == 0
    p[hole] = -1
    return p


def brute_robustness(phen, N, S):
    neutral = np.zeros(S + 1, dtype=np.uint64)
    to_del = np.zeros(S + 1, dtype=np.uint64)
    g = np.arange(1 << N)
    b = np.where(phen < 0, S, phen)
    for i in range(N):
        q = phen[g ^ (1 << i)]
        np.add.at(neutral, b[q == phen], 1)
        np.add.at(to_del, b[q < 0], 1)
    return neutral, to_del


def brute_components(phen, N):
    """Breadth-first search over neutral flips (independent of the oracle's union-find)."""
    label = np.full(1 << N, -1, dtype=np.int64)
    for start in range(1 << N):
        if phen[start] < 0 or label[start] >= 0:
            continue
        comp = [start]
        label[start] = start
        k = 0
        while k < len(comp):
            g = comp[k]
            k += 1
            for i in range(N):
                h = g ^ (1 << i)
                if label[h] < 0 and phen[h] == phen[g]:
                    label[h] = start
                    comp.append(h)
        # start is the smallest id reached first in increasing order
        label[np.array(comp)] = min(comp)
    return label


def test_designability_counts():
    phen = synthetic_map(12, 9, 1)
    h = oracle.designability(phen, 9)
    assert int(h.sum()) == 1 << 12
    assert int(h[9]) == int((phen < 0).sum())
    np.testing.assert_array_equal(h[:9], np.bincount(phen[phen >= 0], minlength=9))


@pytest.mark.parametrize("N,S,seed", [(10, 4, 2), (12, 9, 3)])
def test_robustness_matches_brute(N, S, seed):
    phen = synthetic_map(N, S, seed)
    n, d = oracle.robustness(phen, N, S)
    bn, bd = brute_robustness(phen, N, S)
    np.testing.assert_array_equal(n, bn)
    np.testing.assert_array_equal(d, bd)
    # every neutral edge is counted from both ends
    assert (n % 2 == 0).all()


@pytest.mark.parametrize("N,S,seed", [(10, 4, 2), (12, 9, 3), (11, 2, 4)])
def test_components_match_bfs(N, S, seed):
    phen = synthetic_map(N, S, seed)
    lab, nc = oracle.components(phen, N, S)
    want = brute_components(phen, N)
    np.testing.assert_array_equal(lab, want)
    for p in range(S):
        members = lab[phen == p]
        assert int(nc[p]) == len(np.unique(members))


def test_real_4x4_map_invariants(obox):
    """Sum of designabilities is 2^N; R_p even; neutral + deleterious + other flips = N 2^N;
    component sizes add up to N_p; labels are the smallest member."""
    b = obox((4, 4))
    phen = b.full_map()
    N, S = b.N, b.S
    h = oracle.designability(phen, S)
    assert int(h.sum()) == 1 << N
    n, d = oracle.robustness(phen, N, S)
    bn, bd = brute_robustness(phen, N, S)
    np.testing.assert_array_equal(n, bn)
    np.testing.assert_array_equal(d, bd)
    lab, nc = oracle.components(phen, N, S)
    np.testing.assert_array_equal(lab, brute_components(phen, N))
    assert int(nc.sum()) == len(np.unique(lab[lab >= 0]))
    for p in range(S):
        m = phen == p
        assert int(m.sum()) == int(h[p])
        if m.any():
            assert (lab[m] <= np.nonzero(m)[0]).all()
    other = 0
    g = np.arange(1 << N)
    for i in range(N):
        q = phen[g ^ (1 << i)]
        other += int(((q != phen) & (q >= 0)).sum())
    assert int(n.sum()) + int(d[:S].sum()) + other + int(d[S]) - int(n[S]) == N << N


def test_neighbourhood_rows_sum_to_N_Nq(obox):
    """Eq. 2: the (K-1)L = N neighbours of phenotype q's genotypes split over all p; phi_qq = rho_q."""
    b = obox((4, 4))
    phen = b.full_map()
    h = oracle.designability(phen, b.S)
    n, d = oracle.robustness(phen, b.N, b.S)
    q = int(np.argmax(h[: b.S]))
    row = oracle.neighbourhood(phen, b.N, b.S, q)
    assert int(row.sum()) == b.N * int(h[q])
    assert int(row[q]) == int(n[q]) and int(row[b.S]) == int(d[q])


def test_golden_file_is_well_formed():
    with open(GOLDEN) as f:
        pins = json.load(f)
    assert pins["folds_3x3x3"]["value"] - pins["undesignable_3x3x3"]["value"] == pins["designable_3x3x3"]["value"]
    assert abs(pins["fold_fraction_3x3x3"]["value"] + pins["deleterious_fraction_3x3x3"]["value"] - 1) < 1e-9


def brute_neighbourhood(phen, N, S, q):
    """Eq. 2 numerators of row q by direct counting: for every genotype of phenotype q and every
    single flip, one count at the neighbour's phenotype (index S for -1)."""
    row = np.zeros(S + 1, dtype=np.uint64)
    g = np.nonzero(phen == q)[0]
    for i in range(N):
        p = phen[g ^ (1 << i)]
        np.add.at(row, np.where(p < 0, S, p), 1)
    return row


@pytest.mark.parametrize("N,S,seed", [(10, 4, 2), (12, 9, 3)])
def test_neighbourhood_every_row_matches_brute_force(N, S, seed):
    """Every entry of every row (q = -1 .. S-1), on maps whose rows have many nonzero entries."""
    phen = synthetic_map(N, S, seed)
    for q in range(-1, S):
        np.testing.assert_array_equal(oracle.neighbourhood(phen, N, S, q), brute_neighbourhood(phen, N, S, q))


def test_neighbourhood_every_row_of_the_4x4_map(obox):
    b = obox((4, 4))
    phen = b.full_map()
    for q in range(-1, b.S):
        np.testing.assert_array_equal(oracle.neighbourhood(phen, b.N, b.S, q), brute_neighbourhood(phen, b.N, b.S, q))
