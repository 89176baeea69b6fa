"""Shard streamer (GPU): exact totals equal to the full-map reductions, and resume from records."""
import os
import shutil
import tempfile

import numpy as np
import pytest

import oracle

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


@pytest.mark.parametrize("dims,bits", [((4, 5), 4), ((5, 5), 3), ((4, 4), 0)])
def test_streamed_totals_equal_full_map_reductions(hp, obox, dims, bits):
    s = hp.Structs(dims)
    hist, neutral, to_del, computed = hp.stream_shards(s, bits)
    assert computed == 1 << bits
    phen = hp.phenotype_map(s)
    np.testing.assert_array_equal(hist, hp.designability(phen, s.S).cpu().numpy().astype(np.uint64))
    gn, gd = hp.robustness(phen, s.N, s.S)
    np.testing.assert_array_equal(neutral, gn.cpu().numpy().astype(np.uint64))
    np.testing.assert_array_equal(to_del, gd.cpu().numpy().astype(np.uint64))
    if s.N <= 20:
        want = obox(dims).full_map()
        on, od = oracle.robustness(want, s.N, s.S)
        np.testing.assert_array_equal(neutral, on)
        np.testing.assert_array_equal(to_del, od)


def test_resume_reuses_records(hp):
    s = hp.Structs((5, 5))
    d = tempfile.mkdtemp(prefix="hp_shards_")
    try:
        full = hp.stream_shards(s, 3, out_dir=d)
        assert full[3] == 8 and os.path.exists(os.path.join(d, "manifest.txt"))
        again = hp.stream_shards(s, 3, out_dir=d)
        assert again[3] == 0
        for a, b in zip(full[:3], again[:3]):
            np.testing.assert_array_equal(a, b)
        # an interrupted run: the records of shard 5 and one of its pairs are lost
        os.remove(os.path.join(d, "in_5.bin"))
        os.remove(os.path.join(d, "cross_1_5.bin"))
        part = hp.stream_shards(s, 3, out_dir=d)
        assert 0 < part[3] < 8
        for a, b in zip(full[:3], part[:3]):
            np.testing.assert_array_equal(a, b)
        # a record of another library is not reused
        other = hp.Structs((2, 3, 4))
        with pytest.raises(hp.HPError):
            hp.stream_shards(other, 30, out_dir=d)
    finally:
        shutil.rmtree(d, ignore_errors=True)


def test_corrupted_record_is_recomputed(hp):
    """A record whose payload was damaged (one flipped byte) fails its checksum and is not reused:
    the shard it belongs to is mapped again and the totals stay exact."""
    s = hp.Structs((4, 5))
    d = tempfile.mkdtemp(prefix="hp_shards_")
    try:
        full = hp.stream_shards(s, 3, out_dir=d)
        path = os.path.join(d, "in_6.bin")
        raw = bytearray(open(path, "rb").read())
        raw[40] ^= 0x10  # inside the payload, after the 24-byte header
        open(path, "wb").write(bytes(raw))
        again = hp.stream_shards(s, 3, out_dir=d)
        assert again[3] == 1
        for a, b in zip(full[:3], again[:3]):
            np.testing.assert_array_equal(a, b)
        # a truncated record is not reused either
        path = os.path.join(d, "cross_2_6.bin")
        raw = open(path, "rb").read()
        open(path, "wb").write(raw[:-8])
        again = hp.stream_shards(s, 3, out_dir=d)
        assert again[3] == 2
        for a, b in zip(full[:3], again[:3]):
            np.testing.assert_array_equal(a, b)
    finally:
        shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("dims,bits", [((4, 4), 2), ((4, 5), 0), ((4, 5), 3), ((4, 5), 5), ((5, 5), 4)])
def test_streamed_components_equal_full_map_components(hp, obox, dims, bits):
    """Neutral-network counts over the whole space from shards (local union-find + joins across
    the shard bits) equal the full map's hp_neutral_components, and the oracle's on small boxes."""
    s = hp.Structs(dims)
    ncomp, computed = hp.stream_components(s, bits)
    assert computed == 1 << bits
    phen = hp.phenotype_map(s)
    _, want = hp.neutral_components(phen, s.N, s.S)
    np.testing.assert_array_equal(ncomp, want.cpu().numpy().astype(np.uint64))
    if s.N <= 20:
        _, on = oracle.components(obox(dims).full_map(), s.N, s.S)
        np.testing.assert_array_equal(ncomp, on)


def test_stream_components_refuses_a_small_window(hp):
    s = hp.Structs((4, 4))
    with pytest.raises(hp.HPError) as e:
        hp.stream_components(s, 3, window=4)
    assert e.value.code == hp.HP_EINVAL and "window" in str(e.value)
