"""Failure detection on the GPU without a fault: every shared-memory barrier wait of the map kernel
and of the tcgen05 GEMM is bounded.  hp_set_wait_limit(0) makes the first check of every wait give
up, so each launch takes its abort path: it records the timeout in its device error word, waits
(with the fixed drain bound) for its own copies and tensor-core work in flight, frees its tensor
memory and returns.  The call must report HP_ETIMEOUT, and the next call with the built-in limit
must give the exact result (the context stays usable)."""
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
    yield m
    m.set_wait_limit(-1)


def test_map_kernel_wait_timeout_is_reported_and_the_next_call_is_exact(hp, obox):
    s = hp.Structs((4, 4))
    want = obox((4, 4)).full_map()
    out = torch.full((1 << 16,), -7, dtype=torch.int32, device="cuda")
    hp.set_wait_limit(0)
    try:
        with pytest.raises(hp.HPError) as e:
            hp.phenotype_map(s, out=out)
        assert e.value.code == hp.HP_ETIMEOUT, str(e.value)
        assert "timed out" in str(e.value)
    finally:
        hp.set_wait_limit(-1)
    torch.cuda.synchronize()
    got = hp.phenotype_map(s).cpu().numpy()
    np.testing.assert_array_equal(got, want)
    # the gap variant of the kernel takes the same path
    hp.set_wait_limit(0)
    try:
        with pytest.raises(hp.HPError) as e:
            hp.phenotype_map(s, gap_threshold=3)
        assert e.value.code == hp.HP_ETIMEOUT
    finally:
        hp.set_wait_limit(-1)
    np.testing.assert_array_equal(hp.phenotype_map(s).cpu().numpy(), want)


def test_tcgen05_gemm_wait_timeout_is_reported_and_the_next_call_is_exact(hp):
    N, S = 27, 1000
    p = [inputs.init_weights((512, N), N, 5), inputs.init_weights((512,), N, 6),
         inputs.init_weights((512, 512), 512, 7), inputs.init_weights((512,), 512, 8),
         inputs.init_weights((S, 512), 512, 9), inputs.init_weights((S,), 512, 10)]
    net = hp.MLP(N, 512, 512, S, 1024, p)
    ids = torch.from_numpy(inputs.sample_ids(N, 1000, seed=77).view(np.int64)).cuda()
    want = net.topk(ids, 4)
    net.status()
    hp.set_wait_limit(0)
    try:
        net.topk(ids, 4)
        with pytest.raises(hp.HPError) as e:
            net.status()
        assert e.value.code == hp.HP_ETIMEOUT, str(e.value)
    finally:
        hp.set_wait_limit(-1)
    got = net.topk(ids, 4)
    net.status()  # the word was cleared by the failing check; nothing timed out since
    assert torch.equal(got, want)
