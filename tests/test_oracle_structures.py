"""Pins for the oracle's fold-library enumeration (Section 2.1; counts in Section 3.2 and Appendix C)."""
import numpy as np
import pytest

import oracle
from tests import _brute

TINY = [(2, 2), (2, 3), (3, 3), (2, 4), (3, 4), (2, 2, 2)]


def box_edges(dims):
    full = tuple(dims) + (1,) * (3 - len(dims))
    n = full[0] * full[1] * full[2]
    e = 0
    for k in range(3):
        e += (full[k] - 1) * n // full[k]
    return e


@pytest.mark.parametrize("dims", TINY)
def test_matches_brute_force_library(obox, dims):
    """Same conformations, same order, same classes as an independent brute force."""
    b = obox(dims)
    order, cls, S = _brute.library(dims)
    coords, ccls, _, _ = b.export()
    assert b.S_dir == len(order)
    assert b.S == S
    assert [tuple(int(v) for v in row) for row in coords] == [tuple(c) for c in order]
    assert list(ccls) == cls
    assert b.n_paths == len(_brute.hamiltonian_paths(dims))


def test_3x3x3_class_count_is_papers(obox):
    """Section 3.2: 51,704 compact folds on the 3x3x3 lattice."""
    b = obox((3, 3, 3))
    assert b.S == 51704
    assert b.nsym == 48


def test_6x6_directed_count_is_papers_n_fold(obox):
    """Appendix C: N_FOLD = 57337 folds for the 6x6 lattice = conformations modulo the 8 square symmetries."""
    b = obox((6, 6))
    assert b.S_dir == 57337
    assert b.nsym == 8


@pytest.mark.parametrize("dims", [(2, 2), (2, 3), (3, 3), (2, 4), (4, 4), (4, 5), (5, 5), (2, 3, 4), (6, 6), (3, 3, 3)])
def test_burnside_and_free_action(obox, dims):
    """Directed paths have trivial stabilisers, so S_dir = #paths / |G|; the class count follows
    Burnside over G x {identity, reversal}: S = (#paths + sum_g Fix(g o reversal)) / (2|G|)."""
    b = obox(dims)
    assert b.S_dir * b.nsym == b.n_paths
    assert (b.n_paths + b.fix_rev) % (2 * b.nsym) == 0
    assert b.S == (b.n_paths + b.fix_rev) // (2 * b.nsym)
    assert b.S <= b.S_dir <= 2 * b.S


@pytest.mark.parametrize("dims", [(2, 3), (3, 3), (4, 4), (4, 5), (5, 5), (2, 3, 4)])
def test_every_walk_is_compact_with_C_contacts(obox, dims):
    """Every Hamiltonian path uses N-1 lattice edges as bonds; all other box edges are contacts."""
    b = obox(dims)
    coords, _, contacts, cnt = b.export()
    C = box_edges(dims) - (b.N - 1)
    assert b.C == C
    assert (cnt == C).all()
    full = tuple(dims) + (1,) * (3 - len(dims))
    xyz = np.array(_brute.sites(dims))
    # each conformation visits every site once, consecutive residues adjacent
    for row in coords[:: max(1, b.S_dir // 200)]:
        assert sorted(row.tolist()) == list(range(b.N))
        d = np.abs(xyz[row[1:]] - xyz[row[:-1]]).sum(1)
        assert (d == 1).all()
    del full


@pytest.mark.parametrize("dims", [(3, 3), (5, 5), (3, 3, 3)])
def test_odd_box_ends_on_majority_colour(obox, dims):
    """With an odd number of sites the path alternates colours and both ends lie on the majority colour."""
    b = obox(dims)
    coords, _, _, _ = b.export()
    xyz = np.array(_brute.sites(dims))
    colour = xyz.sum(1) % 2
    assert (colour[coords[:, 0]] == 0).all() and (colour[coords[:, -1]] == 0).all()


@pytest.mark.parametrize("dims", [(4, 4), (5, 5), (2, 3, 4)])
def test_class_reps_sorted_and_minimal(obox, dims):
    """Class ids rank the representatives; each is the smallest image over G and reversal."""
    b = obox(dims)
    reps = b.class_reps()
    assert all(tuple(reps[i]) < tuple(reps[i + 1]) for i in range(b.S - 1))
    G = _brute.group(dims)
    pts = _brute.sites(dims)
    for r in reps[:: max(1, b.S // 50)]:
        c = [pts[s] for s in r]
        imgs = []
        for seq in (c, c[::-1]):
            imgs += [tuple(_brute.site_id(g(x), dims) for x in seq) for g in G]
        assert min(imgs) == tuple(int(v) for v in r)


def test_2x3_hand_worked_conformations(obox):
    """The 2x3 box: four conformations in three classes (hand-derived from Section 2.1's definition).
    Picture the box 3 wide and 2 high: top row a b c, bottom row d e f.  Contact sets are residue pairs,
    so they do not depend on how the box is oriented or numbered.  U-turn a b c f e d: contacts (0,5),(1,4); the zig-zag a d e b c f: (0,3),(2,5);
    the hook a d e f c b and its reverse: (0,5),(2,5) and (0,3),(0,5)."""
    b = obox((2, 3))
    assert (b.S, b.S_dir, b.C) == (3, 4, 2)
    _, cls, contacts, _ = b.export()
    sets = sorted(tuple(sorted(map(tuple, c.tolist()))) for c in contacts)
    assert sets == sorted([((0, 5), (1, 4)), ((0, 3), (2, 5)), ((0, 5), (2, 5)), ((0, 3), (0, 5))])
    # exactly one class holds two orientations
    assert sorted(np.bincount(cls).tolist()) == [1, 1, 2]
