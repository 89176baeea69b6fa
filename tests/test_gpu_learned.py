"""The learned proposal + exact bound pruning at full scale: over EVERY 3x3x3 sequence against the
exhaustive map, and on seeded 6x6 shards (the paper's Table 3 sampling workload) against the plain
per-sequence scan and the oracle.  Pruning is exact, so the phenotypes must agree everywhere however
well the network is trained; training only changes how much is pruned."""
import numpy as np
import pytest

from paper_2008_05612_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROWS = 16384  # proposal chunk (max_batch) of the networks below


@pytest.fixture(scope="module")
def hp():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2008_05612_gb300 as m

    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available for a gpu-marked test")
    return m


def params(N, S, seed):
    return [inputs.init_weights((512, N), N, seed), inputs.init_weights((512,), N, seed + 1),
            inputs.init_weights((512, 512), 512, seed + 2), inputs.init_weights((512,), 512, seed + 3),
            inputs.init_weights((S, 512), 512, seed + 4), inputs.init_weights((S,), 512, seed + 5)]


def train(net, ids, labels, steps, batch=4096, lr=1e-3):
    perm = torch.randperm(ids.numel(), device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    losses = []
    for st in range(steps):
        j = perm[(st * batch) % (ids.numel() - batch):][:batch]
        l = net.train_step(ids[j].contiguous(), labels[j].contiguous(), lr, want_loss=(st == 0 or st == steps - 1))
        if l is not None:
            losses.append(l)
    net.status()
    return losses


def test_learned_pruned_over_the_whole_3x3x3_space(hp):
    """All 2^27 ids: network top-4 -> candidate conformations -> pruned scan, equal to the exhaustive
    map id by id; the network is trained on the exhaustive kernel's labels of the seeded 1-in-10 sample
    of a 2^22-id stretch of the space."""
    s = hp.Structs((3, 3, 3))
    n = 1 << s.N
    phen = torch.empty(n, dtype=torch.int32, device="cuda")
    aux = torch.empty(n, dtype=torch.int32, device="cuda")
    hp.phenotype_map(s, 0, n, out=phen, aux=aux)
    ids_np = (np.arange(1 << 22, dtype=np.uint64) * np.uint64(32) + np.uint64(5))
    ids_np = ids_np[inputs.training_mask(ids_np)]
    tids = torch.from_numpy(ids_np.view(np.int64)).cuda()
    net = hp.MLP(s.N, 512, 512, s.S, ROWS, params(s.N, s.S, 71))
    losses = train(net, tids, aux[tids], 400)
    assert losses[-1] < losses[0] - 2.0
    del aux
    mism = torch.zeros((), dtype=torch.int64, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    chunk = 1 << 21
    for off in range(0, n, chunk):
        ids = torch.arange(off, off + chunk, dtype=torch.int64, device="cuda")
        cand = hp.proposal_conformations(s, net.topk(ids, 4))
        got = hp.sequence_scan(s, ids, cand=cand, counters=cnt)
        mism += (got != phen[off:off + chunk]).sum()
    net.status()
    frac = int(cnt[0]) / (n * s.S_dir)
    print(f"exact evaluations: {frac:.4f} of all (sequence, conformation) pairs")
    assert int(mism) == 0
    assert frac < 0.5


def test_learned_pruned_on_seeded_6x6_shards(hp, obox):
    """6x6 (N = 36): labels from the plain per-sequence scan on seeded uniform ids; evaluation on
    seeded ids of two seeded 2^32-id shards (shard = the top 4 bits): learned + pruned equals the plain
    scan on every id and the oracle on a sample of them, with fewer exact evaluations when trained."""
    s = hp.Structs((6, 6))
    N, S = s.N, s.S
    tids = torch.from_numpy(inputs.sample_ids(N, 1 << 19, seed=612).view(np.int64)).cuda()
    _, tlab = hp.sequence_scan(s, tids, aux=True)
    p0 = params(N, S, 81)
    net = hp.MLP(N, 512, 512, S, ROWS, p0)
    untrained = hp.MLP(N, 512, 512, S, ROWS, p0)
    losses = train(net, tids, tlab, 300)
    assert losses[-1] < losses[0] - 1.0
    parts = []
    for j in range(2):
        k = inputs.shard_index(j)
        parts.append(inputs.sample_ids(32, 2048, seed=720 + j) | (np.uint64(k) << np.uint64(32)))
    ids_np = np.concatenate(parts)
    ids = torch.from_numpy(ids_np.view(np.int64)).cuda()
    plain = hp.sequence_scan(s, ids)
    evals = {}
    for name, model in (("trained", net), ("untrained", untrained)):
        cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
        got = hp.sequence_scan(s, ids, cand=hp.proposal_conformations(s, model.topk(ids, 4)), counters=cnt)
        model.status()
        assert torch.equal(got, plain), name
        evals[name] = int(cnt[0])
    print("exact evaluations:", evals, "plain:", ids.numel() * s.S_dir)
    assert evals["trained"] < evals["untrained"] <= ids.numel() * s.S_dir
    # the oracle on 128 ids of each shard
    pick = np.r_[0:128, 2048:2048 + 128]
    want = obox((6, 6)).phenotypes(ids_np[pick])
    np.testing.assert_array_equal(plain.cpu().numpy()[pick], want)
