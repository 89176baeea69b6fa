"""Plain CPU oracle for the HP genotype-phenotype map (arXiv 2008.05612).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
leg of the benchmark are the only callers.  Nothing in the CUDA library imports
or links this package, and this package imports nothing from the library.

`hp_oracle.c` holds the arithmetic (enumeration, Eq. 1 energies, ground state,
designability, Eq. 2 numerators, neutral components); this module only loads
it with ctypes and marshals numpy arrays.  `mlp.py` holds the fp64 reference of
the proposal network used by the learned variant.

Parity status: every function here is pinned by tests against values the paper
prints (S = 51,704 for 3x3x3, N_FOLD = 57,337 for 6x6, the 3x3x3 folding
fraction), hand-worked cases, brute force and closed-form invariants; see
tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhp_oracle.so")
_lib = None
_lock = threading.Lock()

READING_A, READING_B, READING_C = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile hp_oracle.c with the host C compiler (plain gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.or_enumerate.restype = vp
        lib.or_enumerate.argtypes = [ctypes.c_int, vp]
        lib.or_free.argtypes = [vp]
        lib.or_info.argtypes = [vp, vp]
        lib.or_export.argtypes = [vp, vp, vp, vp, vp]
        lib.or_class_reps.argtypes = [vp, vp]
        lib.or_energy.restype = ctypes.c_int
        lib.or_energy.argtypes = [vp, ctypes.c_uint64, i32]
        lib.or_energy_coords.restype = ctypes.c_int
        lib.or_energy_coords.argtypes = [vp, ctypes.c_uint64, i32]
        lib.or_lower_bound.restype = ctypes.c_int
        lib.or_lower_bound.argtypes = [vp, ctypes.c_uint64, i32]
        lib.or_phenotypes.restype = ctypes.c_int
        lib.or_phenotypes.argtypes = [vp, vp, i64, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int]
        lib.or_phenotypes_gaps.restype = ctypes.c_int
        lib.or_phenotypes_gaps.argtypes = [vp, vp, i64, ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.c_int]
        lib.or_designability.argtypes = [vp, ctypes.c_uint64, i32, vp]
        lib.or_robustness.argtypes = [vp, ctypes.c_int, i32, vp, vp]
        lib.or_neighbourhood.argtypes = [vp, ctypes.c_int, i32, i32, vp]
        lib.or_components.restype = ctypes.c_int
        lib.or_components.argtypes = [vp, ctypes.c_int, i32, vp, vp]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Box:
    """Fold library of one lattice box: conformations, classes and contacts."""

    def __init__(self, dims):
        dims = tuple(int(d) for d in dims)
        if len(dims) not in (2, 3):
            raise ValueError("dims must have 2 or 3 entries")
        self.dims = dims
        self.ndim = len(dims)
        lib = _load()
        d = np.array(list(dims) + [1] * (3 - len(dims)), dtype=np.int32)
        h = lib.or_enumerate(self.ndim, _ptr(d))
        if not h:
            raise ValueError(f"oracle cannot enumerate box {dims}")
        self._h = ctypes.c_void_p(h)
        info = np.zeros(8, dtype=np.int64)
        lib.or_info(self._h, _ptr(info))
        self.N, self.S, self.S_dir, self.C, self.nsym = (int(v) for v in info[:5])
        self.n_paths = int(info[5])
        self.fix_rev = int(info[6])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.or_free(h)
            self._h = None

    def export(self):
        """(coords S_dir x N, conf_class S_dir, contacts S_dir x C x 2, contact_count S_dir)"""
        coords = np.zeros((self.S_dir, self.N), dtype=np.uint8)
        cls = np.zeros(self.S_dir, dtype=np.int32)
        con = np.zeros((self.S_dir, max(self.C, 1), 2), dtype=np.uint8)
        cnt = np.zeros(self.S_dir, dtype=np.int32)
        _load().or_export(self._h, _ptr(coords), _ptr(cls), _ptr(con), _ptr(cnt))
        return coords, cls, con[:, : self.C, :], cnt

    def class_reps(self):
        reps = np.zeros((self.S, self.N), dtype=np.uint8)
        _load().or_class_reps(self._h, _ptr(reps))
        return reps

    def energy(self, g: int, s: int) -> int:
        return int(_load().or_energy(self._h, int(g), int(s)))

    def energy_coords(self, g: int, s: int) -> int:
        return int(_load().or_energy_coords(self._h, int(g), int(s)))

    def lower_bound(self, g: int, s: int) -> int:
        return int(_load().or_lower_bound(self._h, int(g), int(s)))

    def phenotypes(self, seqs, reading: int = READING_B, gap: int = 1, nthreads: int | None = None, aux: bool = False,
                   gaps: bool = False):
        """Phenotypes of the ids (Section 2.1 with energy-gap threshold `gap`); with aux, also the class of
        the lowest-index minimiser; with gaps, also E2 - E1 (second-lowest energy counted with
        multiplicity minus the lowest; INT32_MAX for a single competitor).  Returns phen, then aux and
        gaps in that order when requested."""
        seqs = np.ascontiguousarray(np.asarray(seqs, dtype=np.uint64))
        n = seqs.shape[0]
        phen = np.zeros(n, dtype=np.int32)
        auxa = np.zeros(n, dtype=np.int32) if aux else None
        gapa = np.zeros(n, dtype=np.int32) if gaps else None
        nt = nthreads or min(os.cpu_count() or 1, 64)
        rc = _load().or_phenotypes_gaps(self._h, _ptr(seqs), n, int(reading), int(gap), _ptr(phen),
                                        _ptr(auxa) if aux else None, _ptr(gapa) if gaps else None, int(nt))
        if rc != 0:
            raise ValueError("oracle rejected the phenotype request")
        out = (phen,) + ((auxa,) if aux else ()) + ((gapa,) if gaps else ())
        return out if len(out) > 1 else phen

    def full_map(self, reading: int = READING_B, gap: int = 1, nthreads: int | None = None, aux: bool = False,
                 gaps: bool = False):
        return self.phenotypes(np.arange(1 << self.N, dtype=np.uint64), reading, gap, nthreads, aux, gaps)


def designability(phen: np.ndarray, S: int) -> np.ndarray:
    phen = np.ascontiguousarray(phen, dtype=np.int32)
    hist = np.zeros(S + 1, dtype=np.uint64)
    _load().or_designability(_ptr(phen), phen.shape[0], int(S), _ptr(hist))
    return hist


def robustness(phen: np.ndarray, N: int, S: int):
    phen = np.ascontiguousarray(phen, dtype=np.int32)
    if phen.shape[0] != (1 << N):
        raise ValueError("robustness needs the full map of 2^N genotypes")
    neutral = np.zeros(S + 1, dtype=np.uint64)
    to_del = np.zeros(S + 1, dtype=np.uint64)
    _load().or_robustness(_ptr(phen), int(N), int(S), _ptr(neutral), _ptr(to_del))
    return neutral, to_del


def neighbourhood(phen: np.ndarray, N: int, S: int, q: int) -> np.ndarray:
    phen = np.ascontiguousarray(phen, dtype=np.int32)
    out = np.zeros(S + 1, dtype=np.uint64)
    _load().or_neighbourhood(_ptr(phen), int(N), int(S), int(q), _ptr(out))
    return out


def components(phen: np.ndarray, N: int, S: int):
    phen = np.ascontiguousarray(phen, dtype=np.int32)
    if phen.shape[0] != (1 << N):
        raise ValueError("components need the full map of 2^N genotypes")
    label = np.zeros(1 << N, dtype=np.int32)
    ncomp = np.zeros(max(S, 1), dtype=np.uint64)
    rc = _load().or_components(_ptr(phen), int(N), int(S), _ptr(label), _ptr(ncomp))
    if rc != 0:
        raise ValueError("oracle components failed")
    return label, ncomp[:S]
