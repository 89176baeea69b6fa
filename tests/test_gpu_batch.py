"""Batched persistent launch, kernel shapes, autotuner and CUDA-graph plans (GPU).

Every path must give exactly the maps of the single-box entry point, and those
are checked against the oracle elsewhere; here the small boxes are also checked
against the oracle directly."""
import numpy as np
import pytest

from paper_2008_05612_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED = [(4, 4), (4, 5), (5, 5), (2, 3, 4), (3, 3, 3)]


@pytest.fixture(scope="module")
def hp():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2008_05612_gb300 as m

    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available for a gpu-marked test")
    return m


@pytest.fixture(scope="module")
def singles(hp):
    out = {}
    for dims in MIXED:
        s = hp.Structs(dims)
        out[dims] = (s, hp.phenotype_map(s))
    torch.cuda.synchronize()
    return out


def test_mixed_batch_equals_single_maps(hp, singles, obox):
    structs = [singles[d][0] for d in MIXED]
    ranges = [(0, 1 << s.N) for s in structs]
    outs = [torch.full((1 << s.N,), -7, dtype=torch.int32, device="cuda") for s in structs]
    hp.phenotype_map_batch(structs, ranges, outs)
    for d, o in zip(MIXED, outs):
        assert torch.equal(o, singles[d][1]), d
    np.testing.assert_array_equal(outs[0].cpu().numpy(), obox((4, 4)).full_map())
    np.testing.assert_array_equal(outs[1].cpu().numpy(), obox((4, 5)).full_map())


def test_batch_with_ragged_ranges(hp, singles):
    structs = [singles[(4, 5)][0], singles[(3, 3, 3)][0], singles[(4, 4)][0]]
    ranges = [(12345, 300001), (1 << 26, 3 << 22), (7, 1)]
    outs = [torch.empty(r[1], dtype=torch.int32, device="cuda") for r in ranges]
    hp.phenotype_map_batch(structs, ranges, outs)
    full = [singles[(4, 5)][1], singles[(3, 3, 3)][1], singles[(4, 4)][1]]
    for o, r, f in zip(outs, ranges, full):
        assert torch.equal(o, f[r[0] : r[0] + r[1]])


@pytest.mark.parametrize("dims", [(4, 5), (3, 3, 3)])
def test_every_compiled_shape_gives_the_same_map(hp, singles, obox, dims):
    s, ref = singles[dims]
    shapes = hp.tile_cfg_list()
    assert len(shapes) >= 6 and (5, 256) in shapes
    n = 1 << s.N  # the full space: every role real for 3x3x3, virtual roles for 4x5
    want = ref[:n]
    for sh in shapes:
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        hp.phenotype_map_batch([s], [(0, n)], [out], cfg=sh)
        assert torch.equal(out, want), sh


def test_unsupported_shape_rejected(hp, singles):
    s = singles[(4, 4)][0]
    with pytest.raises(hp.HPError):
        s.set_tile_cfg(7, 32)
    with pytest.raises(hp.HPError):
        hp.phenotype_map_batch([s], [(0, 16)], [torch.empty(16, dtype=torch.int32, device="cuda")], cfg=(5, 96))


def test_autotune_keeps_a_compiled_shape(hp, singles):
    s, ref = singles[(3, 3, 3)]
    best, ms = s.autotune()
    assert best in hp.tile_cfg_list()
    assert s.tile_cfg() == best
    assert ms[best] > 0 and all(v == -1 or v > 0 for v in ms.values())
    assert ms[best] == min(v for v in ms.values() if v > 0)
    # the tuned shape is used by the plain entry point and changes nothing in the result
    out = hp.phenotype_map(s, 1 << 25, 1 << 24)
    assert torch.equal(out, ref[1 << 25 : (1 << 25) + (1 << 24)])
    s.set_tile_cfg()
    assert s.tile_cfg() == (5, 256)


def test_graph_plan_replays(hp, singles):
    structs = [singles[(4, 4)][0], singles[(2, 3, 4)][0], singles[(3, 3, 3)][0]]
    ranges = [(0, 1 << 16), (0, 1 << 24), (3 << 24, 1 << 24)]
    outs = [torch.empty(r[1], dtype=torch.int32, device="cuda") for r in ranges]
    plan = hp.BatchPlan(structs, ranges, outs)
    full = [singles[(4, 4)][1], singles[(2, 3, 4)][1], singles[(3, 3, 3)][1]]
    for _ in range(2):
        for o in outs:
            o.fill_(-7)
        plan.launch()
        plan.status()
        for o, r, f in zip(outs, ranges, full):
            assert torch.equal(o, f[r[0] : r[0] + r[1]])
    # replay inside a user stream
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        for o in outs:
            o.fill_(-7)
        plan.launch(st)
        plan.status(st)
    for o, r, f in zip(outs, ranges, full):
        assert torch.equal(o, f[r[0] : r[0] + r[1]])
    del plan


@pytest.mark.parametrize("dims", [(3, 3), (5, 5), (3, 3, 3)])
def test_half_enumeration_equals_two_half_ranges(hp, obox, dims):
    """Odd chains use the reversal symmetry for a full-space map; two half ranges (which do not)
    must give the same map and labels."""
    s = hp.Structs(dims)
    n = 1 << s.N
    full = torch.empty(n, dtype=torch.int32, device="cuda")
    fa = torch.empty(n, dtype=torch.int32, device="cuda")
    hp.phenotype_map(s, 0, n, out=full, aux=fa)
    halves = torch.empty(n, dtype=torch.int32, device="cuda")
    ha = torch.empty(n, dtype=torch.int32, device="cuda")
    hp.phenotype_map(s, 0, n // 2, out=halves[: n // 2], aux=ha[: n // 2])
    hp.phenotype_map(s, n // 2, n // 2, out=halves[n // 2 :], aux=ha[n // 2 :])
    assert torch.equal(full, halves)
    assert torch.equal(fa, ha)
    if s.N <= 16:
        want, want_aux = obox(dims).full_map(aux=True)
        np.testing.assert_array_equal(full.cpu().numpy(), want)
        np.testing.assert_array_equal(fa.cpu().numpy(), want_aux)


@pytest.mark.parametrize("T", [2, 7])
def test_batch_at_a_gap_threshold_equals_single_maps(hp, obox, T):
    """hp_phenotype_map_batch_gap: several boxes at an energy-gap threshold T in one launch, equal to
    the single maps at T (those are checked against the oracle's thresholds elsewhere), and to the
    oracle on the small boxes."""
    dims_list = [(4, 4), (4, 5), (2, 3, 4)]
    structs = [hp.Structs(d) for d in dims_list]
    ranges = [(0, 1 << s.N) for s in structs]
    outs = [torch.full((1 << s.N,), -7, dtype=torch.int32, device="cuda") for s in structs]
    hp.phenotype_map_batch(structs, ranges, outs, gap_threshold=T)
    for d, s, o in zip(dims_list, structs, outs):
        assert torch.equal(o, hp.phenotype_map(s, gap_threshold=T)), d
        if s.N <= 20:
            np.testing.assert_array_equal(o.cpu().numpy(), obox(d).full_map(gap=T))
    with pytest.raises(hp.HPError):
        hp.phenotype_map_batch(structs, ranges, outs, gap_threshold=(1 << 20) + 1)
