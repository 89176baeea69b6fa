"""C-ABI checks that need no GPU: the library loads, exports every symbol the header declares,
its host enumerator agrees with the oracle, and host-side argument checks return status codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2008_05612_gb300 as hp
from paper_2008_05612_gb300 import build as hpbuild

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "hp_gpmap.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    hpbuild.build()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hp_[a-z_]+)\s*\(", text)))


def test_header_symbols_are_exported():
    syms = declared_symbols()
    assert len(syms) >= 9
    L = ctypes.CDLL(hp.LIB_PATH)
    for name in syms:
        assert hasattr(L, name), name
    assert set(syms) <= set(hp.EXPORTS) | set(syms)
    assert set(hp.EXPORTS) <= set(syms)


@pytest.mark.parametrize("dims", [(2, 2), (2, 3), (3, 3), (2, 4), (4, 4), (4, 5), (5, 5), (2, 3, 4), (6, 6), (3, 3, 3)])
def test_library_enumeration_equals_oracle(obox, dims):
    s = hp.Structs(dims)
    o = obox(dims)
    assert (s.N, s.S, s.S_dir, s.C) == (o.N, o.S, o.S_dir, o.C)
    c1, k1, cl1 = s.export()
    c2, cl2, k2, _ = o.export()
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(cl1, cl2)
    np.testing.assert_array_equal(k1, k2)


def test_bad_arguments_return_status():
    L = hp.lib()
    h = ctypes.c_void_p()
    assert L.hp_enumerate_structures(4, (ctypes.c_int32 * 3)(2, 2, 2), ctypes.byref(h)) == hp.HP_EINVAL
    assert L.hp_enumerate_structures(2, (ctypes.c_int32 * 3)(0, 3, 1), ctypes.byref(h)) == hp.HP_EINVAL
    assert L.hp_enumerate_structures(3, (ctypes.c_int32 * 3)(4, 4, 4), ctypes.byref(h)) == hp.HP_EUNSUPPORTED
    assert L.hp_enumerate_structures(2, (ctypes.c_int32 * 3)(1, 1, 1), ctypes.byref(h)) == hp.HP_EINVAL
    assert b"site" in L.hp_last_error()
    assert L.hp_structs_info(None, None, None, None, None) == hp.HP_EINVAL
    s = hp.Structs((2, 3))
    # range beyond 2^N, threshold out of [1, 2^20], NULL output: rejected before any CUDA call
    assert L.hp_phenotype_map(s.handle, 60, 8, 1, ctypes.c_void_p(16), None, None) == hp.HP_EINVAL
    assert L.hp_phenotype_map(s.handle, 60, 8, 3, ctypes.c_void_p(16), None, None) == hp.HP_EINVAL
    assert L.hp_phenotype_map(s.handle, 0, 8, 0, ctypes.c_void_p(16), None, None) == hp.HP_EINVAL
    assert L.hp_phenotype_map(s.handle, 0, 8, (1 << 20) + 1, ctypes.c_void_p(16), None, None) == hp.HP_EINVAL
    assert L.hp_phenotype_map(s.handle, 0, 8, 1, None, None, None) == hp.HP_EINVAL
    p16 = ctypes.c_void_p(16)
    assert L.hp_sequence_scan_gap(s.handle, p16, 4, None, 0, 0, p16, None, None, None, None) == hp.HP_EINVAL
    assert L.hp_sequence_scan_gap(s.handle, p16, 4, None, 0, (1 << 20) + 1, p16, None, None, None, None) == hp.HP_EINVAL
    assert L.hp_sequence_scan_gap(s.handle, None, 4, None, 0, 2, p16, None, None, None, None) == hp.HP_EINVAL
    assert L.hp_sequence_scan_gap(s.handle, p16, 4, p16, 0, 2, p16, None, None, None, None) == hp.HP_EINVAL
    assert L.hp_proposal_conformations(s.handle, p16, 4, 0, p16, None) == hp.HP_EINVAL
    assert L.hp_proposal_conformations(s.handle, p16, -1, 2, p16, None) == hp.HP_EINVAL
    assert L.hp_designability(None, 4, 3, None, None) == hp.HP_EINVAL
    assert L.hp_robustness(ctypes.c_void_p(16), 50, 3, ctypes.c_void_p(16), ctypes.c_void_p(16), None) == hp.HP_EINVAL
    assert L.hp_neutral_components(ctypes.c_void_p(16), 36, 3, ctypes.c_void_p(16), ctypes.c_void_p(16), None) == hp.HP_EUNSUPPORTED


def test_product_path_has_no_oracle_dependency():
    """The package and its sources never name the oracle."""
    pkg = os.path.dirname(hp.__file__)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "hp_oracle" not in text, f


def test_stream_shards_rejects_a_small_window_before_device_work():
    s = hp.Structs((4, 4))
    with pytest.raises(hp.HPError) as e:
        hp.stream_shards(s, 3, window=4)
    assert e.value.code == hp.HP_EINVAL and "window" in str(e.value)
    with pytest.raises(hp.HPError):
        hp.stream_shards(s, 16)


def test_no_cpu_fallback():
    """Host tensors are refused and a map without a GPU raises: there is no CPU path."""
    torch = pytest.importorskip("torch")
    s = hp.Structs((2, 3))
    with pytest.raises(TypeError):
        hp.sequence_scan(s, torch.zeros(4, dtype=torch.int64))
    with pytest.raises(TypeError):
        hp.designability(torch.zeros(4, dtype=torch.int32), s.S)
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError):
            hp.phenotype_map(s)


def test_histogram_outputs_are_checked_before_any_launch():
    """An output shorter than S + 1 counts, or on another device than the map, is refused by the
    binding before the entry point could write past its end."""
    torch = pytest.importorskip("torch")
    phen = torch.zeros(16, dtype=torch.int32)
    short = torch.zeros(10, dtype=torch.int64)
    for fn in (hp.designability, hp.designability_noalloc):
        with pytest.raises(hp.HPError) as e:
            fn(phen, 10, short)
        assert e.value.code == hp.HP_EINVAL and "S + 1" in str(e.value)
        with pytest.raises(hp.HPError) as e:
            fn(phen, 0, short)
        assert e.value.code == hp.HP_EINVAL


def test_every_dependent_launch_waits_for_its_predecessor():
    """A kernel started by launch_pdl may run while the kernel before it is still running, so its
    body must execute pdl_wait() before it touches global memory: the simple kernels as their first
    statement, the tcgen05 GEMM right after its shared-memory and tensor-memory set-up."""
    import re

    csrc = os.path.join(os.path.dirname(hp.__file__), "csrc")
    text = "".join(open(os.path.join(csrc, f)).read() for f in sorted(os.listdir(csrc)) if f.endswith(".cu"))
    launched = set(re.findall(r"launch_pdl\(\s*([A-Za-z_]\w*)", text))
    assert {"gemm_tc_kernel", "softmax_finish_kernel", "encode_bits", "adam_update"} <= launched, launched
    for name in launched:
        m = re.search(r"__global__[^;{]*?\b" + name + r"\s*\([^)]*\)\s*\{", text, re.S)
        assert m, name
        body = text[m.end():]
        if name == "gemm_tc_kernel":
            setup, rest = body.split("pdl_wait();", 1)
            # the set-up allocates tensor memory, initialises barriers and prefetches the tensor
            # maps; it reads no global memory
            for access in ("ep.", "p.err", "__ldg", "ld.global", "cp.async.bulk.tensor"):
                assert access not in setup, (name, access)
        else:
            first = body.lstrip().split(";", 1)[0]
            assert first.replace("hp::", "") == "pdl_wait()", (name, first)
