"""The learned proposal on the GPU: GEMM / forward against an fp64 reference on bf16-rounded
operands, gradients against the oracle's fp64 network, training on labels from the exhaustive
kernel, top-k, and what the trained network gains for the bound-pruned scan."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2008_05612_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# bf16 keeps 8 significant bits (unit roundoff u = 2^-8); operands of every product are rounded once,
# sums are fp32, and an error passes through at most three layers: a normalised error of ~6u = 0.023
# bounds the forward pass and the gradients; the tests allow 0.05.
TOL = 0.05


@pytest.fixture(scope="module")
def hp():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2008_05612_gb300 as m

    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available for a gpu-marked test")
    return m


def init(N, H1, H2, S, seed):
    return [inputs.init_weights((H1, N), N, seed), inputs.init_weights((H1,), N, seed + 1),
            inputs.init_weights((H2, H1), H1, seed + 2), inputs.init_weights((H2,), H1, seed + 3),
            inputs.init_weights((S, H2), H2, seed + 4), inputs.init_weights((S,), H2, seed + 5)]


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def ids_tensor(ids):
    return torch.from_numpy(np.asarray(ids, dtype=np.uint64).view(np.int64)).cuda()


@pytest.mark.parametrize("N,H1,H2,S,n", [(27, 64, 96, 300, 100), (36, 512, 512, 1000, 257), (27, 512, 512, 9000, 512)])
def test_logits_match_fp64_reference(hp, N, H1, H2, S, n):
    p = init(N, H1, H2, S, 11)
    net = hp.MLP(N, H1, H2, S, 512, p)
    ids = inputs.sample_ids(N, n, seed=3)
    got = net.logits(ids_tensor(ids)).cpu().numpy().astype(np.float64)
    net.status()  # no tcgen05 wait gave up
    x = omlp.bits(ids, N)
    # reference with the bf16 roundings the GPU applies to operands and hidden activations
    W1, b1, W2, b2, W3, b3 = p
    a1 = bf16_round(np.maximum(x @ bf16_round(W1).T + b1, 0))
    a2 = bf16_round(np.maximum(a1 @ bf16_round(W2).T + b2, 0))
    want = a2 @ bf16_round(W3).T + b3
    assert rel(got, want) < 1e-3
    # and against the exact fp64 network, within the bf16 bound
    assert rel(got, omlp.forward(p, x)[4]) < TOL


@pytest.mark.parametrize("N,H1,H2,S,n", [(27, 64, 64, 200, 96), (36, 128, 192, 1000, 250), (27, 512, 512, 8200, 512)])
def test_gradients_match_oracle(hp, N, H1, H2, S, n):
    """Forward and backward GEMMs with K % 64 == 0 run on the tcgen05 kernel (ragged M and N tiles in the
    second shape, eight K chunks in the third); the rest on mma.sync."""
    p = init(N, H1, H2, S, 21)
    net = hp.MLP(N, H1, H2, S, max(128, n), p)
    ids = inputs.sample_ids(N, n, seed=8)
    labels = (inputs.splitmix64(ids) % np.uint64(S)).astype(np.int32)
    loss, grads = net.gradients(ids_tensor(ids), torch.from_numpy(labels).cuda())
    # reference: the oracle's fp64 network on the bf16-rounded weights the GPU multiplies with, so that
    # parameter quantisation (which flips a few near-zero ReLU masks in wide layers) is not counted
    # as arithmetic error
    pr = [bf16_round(a) if a.ndim == 2 else a.astype(np.float64) for a in p]
    ref_loss, ref_grads = omlp.loss_and_grads(pr, omlp.bits(ids, N), labels.astype(np.int64))
    assert abs(loss - ref_loss) < TOL * abs(ref_loss)
    errs = [rel(g.astype(np.float64), r) for g, r in zip(grads, ref_grads)]
    print("gradient errors (W1 b1 W2 b2 W3 b3):", ["%.4f" % e for e in errs])
    assert max(errs) < TOL


def test_ignored_rows_do_not_contribute(hp):
    N, H1, H2, S = 20, 32, 32, 50
    p = init(N, H1, H2, S, 31)
    net = hp.MLP(N, H1, H2, S, 64, p)
    ids = inputs.sample_ids(N, 40, seed=9)
    labels = (inputs.splitmix64(ids) % np.uint64(S)).astype(np.int32)
    l1, g1 = net.gradients(ids_tensor(ids[:30]), torch.from_numpy(labels[:30]).cuda())
    lab = labels.copy()
    lab[30:] = -1
    l2, g2 = net.gradients(ids_tensor(ids), torch.from_numpy(lab).cuda())
    # the loss is the sum over labelled rows divided by the number of rows passed (40)
    f = 30.0 / 40.0
    assert abs(l2 - f * l1) < 1e-4 * abs(l1)
    for a, b in zip(g1, g2):
        # both are bf16-rounded products (the 1/n scale enters before the rounding): within ~2u
        assert rel(b, f * a) < 1e-2 or np.abs(a).max() == 0


def test_topk_matches_sorted_logits(hp):
    N, H1, H2, S = 27, 64, 64, 700
    net = hp.MLP(N, H1, H2, S, 512, init(N, H1, H2, S, 41))
    ids = ids_tensor(inputs.sample_ids(N, 300, seed=4))
    z = net.logits(ids).cpu().numpy()
    top = net.topk(ids, 5).cpu().numpy()
    want = np.argsort(-z, axis=1, kind="stable")[:, :5]
    np.testing.assert_array_equal(top, want)


@pytest.mark.parametrize("k", [1, 4, 7, 16])
def test_topk_ties_tiles_and_chunks(hp, k):
    """Fused top-k (per 256-class tile, then merged) against a stable sort of the logits: classes
    repeat every 97 rows of W3 (many exact ties, resolved toward the lower class), S = 1291 leaves an
    11-class last tile (fewer than k = 16 candidates), and 700 ids run in chunks of 256."""
    N, H1, H2, S = 27, 64, 128, 1291
    W1, b1, W2, b2, W3, b3 = init(N, H1, H2, S, 43)
    W3 = W3[np.arange(S) % 97].copy()
    b3 = b3[np.arange(S) % 97].copy()
    net = hp.MLP(N, H1, H2, S, 256, [W1, b1, W2, b2, W3, b3])
    ids = ids_tensor(inputs.sample_ids(N, 700, seed=6))
    z = np.concatenate([net.logits(ids[i:i + 256]).cpu().numpy() for i in range(0, 700, 256)])
    top = net.topk(ids, k).cpu().numpy()
    net.status()
    want = np.argsort(-z, axis=1, kind="stable")[:, :k]
    np.testing.assert_array_equal(top, want)


@pytest.fixture(scope="module")
def trained_3x3x3(hp):
    """Network trained on the GPU with labels (lowest-index minimiser) from the exhaustive kernel,
    on the seeded 1-in-10 sample of 3x3x3 ids restricted to a 2^20 block for test time."""
    s = hp.Structs((3, 3, 3))
    block = np.arange(1 << 20, dtype=np.uint64) * np.uint64(128) + np.uint64(37)  # spread over the space
    train = block[inputs.training_mask(block)]
    ids = ids_tensor(train)
    # labels from the exhaustive kernel: map aligned 2^7-blocks would be wasteful; the per-sequence scan
    # computes the same aux labels exactly for arbitrary ids
    _, aux = hp.sequence_scan(s, ids, aux=True)
    N, H1, H2, S = 27, 512, 512, s.S
    p0 = init(N, H1, H2, S, 51)
    net = hp.MLP(N, H1, H2, S, 1024, p0)
    losses = []
    perm = torch.randperm(ids.numel(), device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    for step in range(300):
        j = perm[(step * 1024) % ids.numel():][:1024]
        if j.numel() < 1024:
            j = perm[:1024]
        l = net.train_step(ids[j].contiguous(), aux[j].contiguous(), 1e-3, want_loss=(step % 50 == 0 or step == 299))
        if l is not None:
            losses.append(l)
    return s, net, p0, losses


def test_training_reduces_loss(trained_3x3x3):
    _, _, _, losses = trained_3x3x3
    assert losses[0] > 9.0  # about ln(51704) = 10.85 at initialisation
    assert losses[-1] < losses[0] - 2.0


def test_trained_proposal_prunes_more_than_untrained(hp, trained_3x3x3):
    """What the network gains: the same exact phenotypes with fewer exact evaluations."""
    s, net, p0, _ = trained_3x3x3
    untrained = hp.MLP(27, 512, 512, s.S, 1024, p0)
    ids = ids_tensor(inputs.sample_ids(27, 2048, seed=99))
    plain = hp.sequence_scan(s, ids)
    evals = {}
    for name, model in (("trained", net), ("untrained", untrained)):
        cand = hp.proposal_conformations(s, model.topk(ids, 4))
        cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
        phen = hp.sequence_scan(s, ids, cand=cand, counters=cnt)
        assert torch.equal(phen, plain)
        evals[name] = int(cnt[0])
    print("exact evaluations:", evals, "plain:", 2048 * s.S_dir)
    assert evals["trained"] < evals["untrained"] < 2048 * s.S_dir


def test_host_or_strided_ids_are_refused(hp):
    """ids must be contiguous int64 device tensors: the binding checks them before any launch."""
    net = hp.MLP(27, 64, 96, 300, 512, init(27, 64, 96, 300, 11))
    with pytest.raises(TypeError):
        net.topk(torch.zeros(4, dtype=torch.int64), 1)
    with pytest.raises(TypeError):
        net.logits(torch.zeros(8, dtype=torch.int64, device="cuda")[::2])
    with pytest.raises(TypeError):
        net.train_step(torch.zeros(4, dtype=torch.int64), torch.zeros(4, dtype=torch.int32, device="cuda"), 1e-3)


@pytest.mark.parametrize("N,H1,H2,S,n", [(27, 64, 96, 1000, 250), (27, 512, 512, 8200, 512)])
def test_train_step_is_one_adam_step_on_the_gradients(hp, N, H1, H2, S, n):
    """The training step (its output layer's update fused into the GEMM that forms the layer's weight
    gradient, which also writes the weights' bf16 copy and its transpose) equals one plain Adam step
    (Kingma & Ba, first step from zero moments) on the gradients of the same batch: a second network
    built from the updated parameters gives the same logits and the same next gradients."""
    p = init(N, H1, H2, S, 51)
    A = hp.MLP(N, H1, H2, S, 512, p)
    ids = inputs.sample_ids(N, n, seed=12)
    labels = (inputs.splitmix64(ids) % np.uint64(S)).astype(np.int32)
    ids_t, lab_t = ids_tensor(ids), torch.from_numpy(labels).cuda()
    probe = ids_tensor(inputs.sample_ids(N, 300, seed=13))
    z0 = A.logits(probe).cpu().numpy().astype(np.float64)
    _, g = A.gradients(ids_t, lab_t)
    lr, b1, b2, eps = np.float32(1e-3), np.float32(0.9), np.float32(0.999), np.float32(1e-8)
    c1, c2 = np.float32(1) / (np.float32(1) - b1), np.float32(1) / (np.float32(1) - b2)
    p1 = []
    for w, gi in zip(p, g):
        w, gi = np.asarray(w, np.float32), np.asarray(gi, np.float32)
        m = (np.float32(1) - b1) * gi
        v = (np.float32(1) - b2) * gi * gi
        p1.append((w - lr * (m * c1) / (np.sqrt(v * c2) + eps)).astype(np.float32))
    A.train_step(ids_t, lab_t, float(lr))
    A.status()
    B = hp.MLP(N, H1, H2, S, 512, p1)
    zA = A.logits(probe).cpu().numpy().astype(np.float64)
    zB = B.logits(probe).cpu().numpy().astype(np.float64)
    moved = rel(zA, z0)
    print("logit change of the step %.4f, fused vs plain %.2e" % (moved, rel(zA, zB)))
    assert moved > 1e-3
    assert rel(zA, zB) < min(5e-3, 0.1 * moved)
    ids2 = inputs.sample_ids(N, n, seed=14)
    lab2 = torch.from_numpy((inputs.splitmix64(ids2) % np.uint64(S)).astype(np.int32)).cuda()
    lA, gA = A.gradients(ids_tensor(ids2), lab2)
    lB, gB = B.gradients(ids_tensor(ids2), lab2)
    assert abs(lA - lB) < 1e-3 * abs(lB)
    for a, b in zip(gA, gB):
        assert rel(a.astype(np.float64), b.astype(np.float64)) < 1e-2
