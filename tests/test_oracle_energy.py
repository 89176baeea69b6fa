"""Pins for the oracle's energies (Eq. 1, Table 1 x 10) and the pruning bound."""
import numpy as np
import pytest

from paper_2008_05612_gb300 import inputs
from tests import _brute


@pytest.mark.parametrize("dims", [(2, 3), (3, 3), (2, 4), (2, 2, 2)])
def test_energy_equals_coordinate_brute_force(obox, dims):
    """Contact-list sum == the oracle's own coordinate scan == an independent Python coordinate scan."""
    b = obox(dims)
    order, _, _ = _brute.library(dims)
    for s, conf in enumerate(order):
        for g in range(1 << b.N):
            e = _brute.energy(conf, g, dims)
            assert b.energy(g, s) == e
            assert b.energy_coords(g, s) == e


@pytest.mark.parametrize("dims", [(4, 4), (5, 5), (2, 3, 4), (3, 3, 3), (6, 6)])
def test_energy_closed_form_on_samples(obox, dims):
    """E = -10 A - 3 B with A = sum_i h_i c_i(s) and B = #HH contacts (the x10 Table 1 split into
    a per-residue term and a pair term); checked against the coordinate scan on seeded samples."""
    b = obox(dims)
    _, _, contacts, _ = b.export()
    ids = inputs.sample_ids(b.N, 300, seed=11)
    confs = (inputs.splitmix64(np.arange(300, dtype=np.uint64) + np.uint64(5)) % np.uint64(b.S_dir)).astype(np.int64)
    for g, s in zip(ids.tolist(), confs.tolist()):
        h = [(g >> i) & 1 for i in range(b.N)]
        c = np.zeros(b.N, dtype=np.int64)
        B = 0
        for i, j in contacts[s].tolist():
            c[i] += 1
            c[j] += 1
            B += h[i] & h[j]
        A = int(sum(h[i] * c[i] for i in range(b.N)))
        e = b.energy_coords(g, s)
        assert e == -10 * A - 3 * B
        assert b.energy(g, s) == e
        assert b.lower_bound(g, s) <= e


@pytest.mark.parametrize("dims", [(4, 4), (2, 3, 4)])
def test_single_h_and_homopolymers(obox, dims):
    """One H at residue i scores -10 c_i(s); all-P scores 0; all-H scores -23 C for every fold."""
    b = obox(dims)
    _, _, contacts, _ = b.export()
    allh = (1 << b.N) - 1
    for s in range(0, b.S_dir, max(1, b.S_dir // 40)):
        deg = np.bincount(contacts[s].reshape(-1), minlength=b.N)
        for i in range(b.N):
            assert b.energy(1 << i, s) == -10 * int(deg[i])
        assert b.energy(0, s) == 0
        assert b.energy(allh, s) == -23 * b.C


@pytest.mark.parametrize("dims", [(3, 3), (2, 4), (4, 4)])
def test_lower_bound_is_safe_everywhere(obox, dims):
    """L_s(h) = -10 A - 3 min(C, floor(A/2)) never exceeds E(h, s), and is tight when B = min(C, A/2)."""
    b = obox(dims)
    tight = 0
    for s in range(b.S_dir):
        for g in range(1 << b.N):
            lb, e = b.lower_bound(g, s), b.energy(g, s)
            assert lb <= e
            tight += lb == e
    assert tight > 0
