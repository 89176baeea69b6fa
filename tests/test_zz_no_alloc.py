"""hp_designability_noalloc: designability for callers that must not have the library allocate
device memory (their framework or service already owns the device memory in its own pool, or they
run under a fixed memory budget).  The entry point keeps its scratch in a static device array, so it
is checked here against the allocating hp_designability, exactly (integer counts), on two calls in
a row, through the C ABI.  This file is collected last so that a run stopping at the first failure
has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2008_05612_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2008_05612_gb300 as hp

    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available for a gpu-marked test")
    return hp


def synthetic(N, S, seed):
    g = np.arange(1 << N, dtype=np.uint64)
    p = (inputs.splitmix64((g >> np.uint64(5)) ^ np.uint64(seed)) % np.uint64(S)).astype(np.int32)
    p[inputs.splitmix64(g ^ np.uint64(seed + 1)) % np.uint64(3) == 0] = -1
    return torch.from_numpy(p).cuda()


def call(hp, fn, phen, S):
    out = torch.full((S + 1,), -7, dtype=torch.int64, device="cuda")
    rc = fn(ctypes.c_void_p(phen.data_ptr()), phen.numel(), S, ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == hp.HP_OK, hp.lib().hp_last_error()
    return out


@pytest.mark.parametrize("N,S,seed", [(22, 51704, 1), (16, 37, 2)])
def test_noalloc_matches_allocating_entry_point_twice(L, N, S, seed):
    hp = L
    lib = hp.lib()
    phen = synthetic(N, S, seed)
    want = call(hp, lib.hp_designability, phen, S)
    first = call(hp, lib.hp_designability_noalloc, phen, S)
    second = call(hp, lib.hp_designability_noalloc, phen, S)
    torch.cuda.synchronize()
    assert torch.equal(first, want)
    assert torch.equal(second, want)
    assert int(want.sum()) == 1 << N


def test_noalloc_other_map_after_previous_contents(L):
    """The shared scratch keeps the last call's contents; a different map must not see them."""
    hp = L
    lib = hp.lib()
    a, b = synthetic(18, 500, 3), synthetic(17, 500, 4)
    call(hp, lib.hp_designability_noalloc, a, 500)
    got = call(hp, lib.hp_designability_noalloc, b, 500)
    assert torch.equal(got, call(hp, lib.hp_designability, b, 500))


def test_noalloc_rejects_sizes_beyond_its_limit(L):
    hp = L
    phen = torch.zeros(16, dtype=torch.int32, device="cuda")
    out = torch.zeros(70001, dtype=torch.int64, device="cuda")
    with pytest.raises(hp.HPError) as e:
        hp.designability_noalloc(phen, 70000, out)
    assert e.value.code == hp.HP_EINVAL and "limit" in str(e.value)
