"""hp_phi_matrix (Eq. 2 numerators for every pair of phenotypes, compressed rows) against the oracle's
rows (or_neighbourhood, pinned entry by entry by direct counting), and the matrix's own invariants:
rows sum to N N_q, the diagonal is the robustness numerator, the -1 column is phi_del's, and flips
are symmetric (M[q][p] = M[p][q])."""
import numpy as np
import pytest

import oracle
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


def synthetic_map(N, S, seed):
    g = np.arange(1 << N, dtype=np.uint64)
    p = (inputs.splitmix64((g >> np.uint64(max(N - 7, 0))) ^ np.uint64(seed)) % np.uint64(S)).astype(np.int32)
    p[inputs.splitmix64(g ^ np.uint64(seed + 5)) % np.uint64(4) == 0] = -1
    return p


def dense_from_csr(row_ptr, col, count, S):
    M = np.zeros((S + 1, S + 1), dtype=np.uint64)
    for q in range(S + 1):
        a, b = int(row_ptr[q]), int(row_ptr[q + 1])
        c = col[a:b]
        assert (np.diff(c) > 0).all(), "columns ascending, no duplicates"
        M[q, c] = count[a:b]
    return M


def check_against_oracle(hp, phen_np, N, S, cap=None):
    phen = torch.from_numpy(phen_np).cuda()
    row_ptr, col, count = hp.phi_matrix(phen, N, S, cap=cap)
    row_ptr, col, count = row_ptr.cpu().numpy(), col.cpu().numpy(), count.cpu().numpy()
    assert row_ptr[0] == 0 and row_ptr[S + 1] == len(col)
    assert (count > 0).all()
    M = dense_from_csr(row_ptr, col, count, S)
    for q in range(-1, S):
        np.testing.assert_array_equal(M[q if q >= 0 else S], oracle.neighbourhood(phen_np, N, S, q))
    return M


@pytest.mark.parametrize("N,S,seed", [(12, 7, 1), (16, 40, 2), (18, 300, 3)])
def test_phi_matrix_synthetic_maps_equal_oracle_rows(hp, N, S, seed):
    M = check_against_oracle(hp, synthetic_map(N, S, seed), N, S)
    np.testing.assert_array_equal(M, M.T)


def test_phi_matrix_grows_its_capacity(hp):
    """A capacity far below the entry count: the call reports the count needed and the binding retries."""
    check_against_oracle(hp, synthetic_map(16, 120, 4), 16, 120, cap=8)


@pytest.mark.parametrize("dims", [(4, 4), (4, 5)])
def test_phi_matrix_real_maps_equal_oracle_rows(hp, obox, dims):
    b = obox(dims)
    M = check_against_oracle(hp, b.full_map(), b.N, b.S)
    np.testing.assert_array_equal(M, M.T)


def test_phi_matrix_3x3x3(hp):
    """Full 3x3x3 map: rows sum to N N_q, the diagonal and -1 column equal hp_robustness, rows equal
    hp_neighbourhood for the top fold and seeded phenotypes; the top fold touches 0.86% of the
    phenotypes (Section 3.2)."""
    s = hp.Structs((3, 3, 3))
    N, S = s.N, s.S
    phen = hp.phenotype_map(s)
    hist = hp.designability(phen, S).cpu().numpy()
    neutral, to_del = (t.cpu().numpy() for t in hp.robustness(phen, N, S))
    row_ptr, col, count = (t.cpu().numpy() for t in hp.phi_matrix(phen, N, S))
    rows = np.repeat(np.arange(S + 1), np.diff(row_ptr))
    sums = np.bincount(rows, weights=count.astype(np.float64), minlength=S + 1)
    np.testing.assert_array_equal(sums.astype(np.int64), N * hist.astype(np.int64))
    diag = rows == col
    np.testing.assert_array_equal(np.bincount(rows[diag], weights=count[diag], minlength=S + 1).astype(np.uint64),
                                  neutral.astype(np.uint64))
    mcol = (col == S) & (rows < S)
    np.testing.assert_array_equal(np.bincount(rows[mcol], weights=count[mcol], minlength=S + 1)[:S].astype(np.uint64),
                                  to_del[:S].astype(np.uint64))
    top = int(np.argmax(hist[:S]))
    picks = [top] + [int(x) % S for x in inputs.sample_ids(30, 12, seed=55)]
    for q in picks:
        a, b = int(row_ptr[q]), int(row_ptr[q + 1])
        want = hp.neighbourhood(phen, N, S, q).cpu().numpy()
        got = np.zeros(S + 1, dtype=np.int64)
        got[col[a:b]] = count[a:b]
        np.testing.assert_array_equal(got, want)
    a, b = int(row_ptr[top]), int(row_ptr[top + 1])
    neighbours = int(((col[a:b] != top) & (col[a:b] != S)).sum())
    designable = int((hist[:S] > 0).sum())
    print("top fold neighbours:", neighbours, "of", designable, "designable =", neighbours / designable)
    assert round(100 * neighbours / designable, 2) == 0.86  # Section 3.2, read as in test_gpu_parity
