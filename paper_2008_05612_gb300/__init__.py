"""GB300 HP-model genotype-phenotype map (arXiv 2008.05612), Python binding.

Every function here only marshals arguments for the C ABI declared in
include/hp_gpmap.h; all computation runs in libhp_gpmap.so (host enumeration
in C++, everything per sequence in CUDA kernels for sm_103a).  PyTorch only
provides device memory and streams.  There is no CPU fallback: if the library
is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libhp_gpmap.so")

HP_OK, HP_EINVAL, HP_ENOMEM, HP_ECUDA, HP_ETIMEOUT, HP_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
_STATUS = {0: "HP_OK", -1: "HP_EINVAL", -2: "HP_ENOMEM", -3: "HP_ECUDA", -4: "HP_ETIMEOUT", -5: "HP_EUNSUPPORTED"}

# every symbol the header declares (checked by the CPU test-suite)
EXPORTS = (
    "hp_enumerate_structures", "hp_structs_info", "hp_structs_export", "hp_structs_free",
    "hp_phenotype_map", "hp_set_tile_cfg", "hp_get_tile_cfg", "hp_tile_cfg_list", "hp_autotune",
    "hp_phenotype_map_batch", "hp_phenotype_map_batch_gap", "hp_batch_plan_create", "hp_batch_plan_launch", "hp_batch_plan_status",
    "hp_batch_plan_free", "hp_sequence_scan", "hp_sequence_scan_gap", "hp_mlp_create", "hp_mlp_free", "hp_mlp_gradients",
    "hp_mlp_train_step", "hp_mlp_logits", "hp_mlp_topk", "hp_mlp_status", "hp_proposal_conformations", "hp_designability", "hp_designability_noalloc", "hp_robustness", "hp_neighbourhood", "hp_phi_matrix", "hp_robustness_cross", "hp_stream_shards", "hp_stream_components",
    "hp_neutral_components",
    "hp_last_error", "hp_set_wait_limit",
)
_VOID = ("hp_structs_free", "hp_last_error", "hp_batch_plan_free", "hp_mlp_free")


class TileCfg(ctypes.Structure):
    _fields_ = [("reg_bits", ctypes.c_int32), ("tile", ctypes.c_int32)]

    def __repr__(self):
        return f"TileCfg(reg_bits={self.reg_bits}, tile={self.tile})"

_lib = None
_lock = threading.Lock()


class HPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Load libhp_gpmap.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhp_gpmap.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64
        L.hp_enumerate_structures.argtypes = [ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.hp_structs_info.argtypes = [vp, vp, vp, vp, vp]
        L.hp_structs_export.argtypes = [vp, vp, vp, vp]
        L.hp_structs_free.argtypes = [vp]
        L.hp_structs_free.restype = None
        L.hp_phenotype_map.argtypes = [vp, u64, u64, i32, vp, vp, vp]
        L.hp_set_tile_cfg.argtypes = [vp, vp]
        L.hp_get_tile_cfg.argtypes = [vp, vp]
        L.hp_tile_cfg_list.argtypes = [vp, vp]
        L.hp_autotune.argtypes = [vp, vp, vp, vp]
        L.hp_phenotype_map_batch.argtypes = [vp, vp, vp, i32, vp, vp, vp]
        L.hp_phenotype_map_batch_gap.argtypes = [vp, vp, vp, i32, i32, vp, vp]
        L.hp_batch_plan_create.argtypes = [vp, vp, vp, i32, vp, vp, vp, ctypes.POINTER(vp)]
        L.hp_batch_plan_launch.argtypes = [vp, vp]
        L.hp_batch_plan_status.argtypes = [vp, vp]
        L.hp_sequence_scan.argtypes = [vp, vp, ctypes.c_int64, vp, i32, vp, vp, vp, vp]
        L.hp_sequence_scan_gap.argtypes = [vp, vp, ctypes.c_int64, vp, i32, i32, vp, vp, vp, vp, vp]
        L.hp_mlp_create.argtypes = [i32, i32, i32, i32, i32, vp, ctypes.POINTER(vp)]
        L.hp_mlp_free.argtypes = [vp]
        L.hp_mlp_free.restype = None
        L.hp_mlp_gradients.argtypes = [vp, vp, vp, i32, vp, vp, vp]
        L.hp_mlp_train_step.argtypes = [vp, vp, vp, i32, ctypes.c_float, vp, vp]
        L.hp_mlp_logits.argtypes = [vp, vp, i32, vp, vp]
        L.hp_mlp_topk.argtypes = [vp, vp, ctypes.c_int64, i32, vp, vp]
        L.hp_mlp_status.argtypes = [vp, vp]
        L.hp_proposal_conformations.argtypes = [vp, vp, ctypes.c_int64, i32, vp, vp]
        L.hp_batch_plan_free.argtypes = [vp]
        L.hp_batch_plan_free.restype = None
        L.hp_designability.argtypes = [vp, u64, i32, vp, vp]
        L.hp_designability_noalloc.argtypes = [vp, u64, i32, vp, vp]
        L.hp_robustness.argtypes = [vp, i32, i32, vp, vp, vp]
        L.hp_neutral_components.argtypes = [vp, i32, i32, vp, vp, vp]
        L.hp_neighbourhood.argtypes = [vp, i32, i32, i32, vp, vp]
        L.hp_phi_matrix.argtypes = [vp, i32, i32, u64, vp, vp, vp, vp, vp]
        L.hp_robustness_cross.argtypes = [vp, vp, u64, i32, vp, vp, vp]
        L.hp_stream_shards.argtypes = [vp, i32, i32, ctypes.c_char_p, vp, vp, vp, vp, vp]
        L.hp_stream_components.argtypes = [vp, i32, i32, vp, vp, vp]
        L.hp_last_error.restype = ctypes.c_char_p
        L.hp_set_wait_limit.argtypes = [ctypes.c_int64]
        for name in EXPORTS:
            if name not in _VOID:
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def set_wait_limit(polls: int):
    """hp_set_wait_limit: poll limit of the kernels' bounded waits for later launches (< 0: built-in)."""
    _check(lib().hp_set_wait_limit(int(polls)))


def _check(rc: int):
    if rc != HP_OK:
        raise HPError(rc, lib().hp_last_error().decode())


def _stream_ptr(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, dtype, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


class Structs:
    """Fold library of a box (hp_enumerate_structures)."""

    def __init__(self, dims):
        dims = tuple(int(d) for d in dims)
        if len(dims) not in (2, 3):
            raise ValueError("dims must have 2 or 3 entries")
        self.dims = dims
        d = (ctypes.c_int32 * 3)(*(list(dims) + [1] * (3 - len(dims))))
        h = ctypes.c_void_p()
        _check(lib().hp_enumerate_structures(len(dims), d, ctypes.byref(h)))
        self._h = h
        vals = [ctypes.c_int32() for _ in range(4)]
        _check(lib().hp_structs_info(h, *[ctypes.byref(v) for v in vals]))
        self.N, self.S, self.S_dir, self.C = (v.value for v in vals)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.hp_structs_free(h)
            self._h = None

    def set_tile_cfg(self, reg_bits=None, tile=None):
        """hp_set_tile_cfg; no arguments restores the default shape."""
        if reg_bits is None:
            _check(lib().hp_set_tile_cfg(self._h, None))
        else:
            c = TileCfg(reg_bits, tile)
            _check(lib().hp_set_tile_cfg(self._h, ctypes.byref(c)))

    def tile_cfg(self):
        c = TileCfg()
        _check(lib().hp_get_tile_cfg(self._h, ctypes.byref(c)))
        return (c.reg_bits, c.tile)

    def autotune(self, stream=None):
        """hp_autotune: returns (best (reg_bits, tile), {shape: ms})."""
        shapes = tile_cfg_list()
        ms = (ctypes.c_float * len(shapes))()
        best = TileCfg()
        _check(lib().hp_autotune(self._h, ctypes.byref(best), ms, _stream_ptr(stream)))
        return (best.reg_bits, best.tile), {sh: float(ms[i]) for i, sh in enumerate(shapes)}

    def export(self):
        """(coords S_dir x N uint8, contacts S_dir x C x 2 uint8, conf_class S_dir int32)"""
        coords = np.zeros((self.S_dir, self.N), dtype=np.uint8)
        contacts = np.zeros((self.S_dir, max(self.C, 1), 2), dtype=np.uint8)
        cls = np.zeros(self.S_dir, dtype=np.int32)
        _check(lib().hp_structs_export(self._h, coords.ctypes.data_as(ctypes.c_void_p),
                                       contacts.ctypes.data_as(ctypes.c_void_p), cls.ctypes.data_as(ctypes.c_void_p)))
        return coords, contacts[:, : self.C], cls


def phenotype_map(structs: Structs, begin: int = 0, count: int | None = None, out=None, aux=None,
                  gap_threshold: int = 1, stream=None):
    """Phenotype of every id in [begin, begin + count) into a device int32 tensor (hp_phenotype_map)."""
    import torch

    if count is None:
        count = (1 << structs.N) - begin
    if out is None:
        out = torch.empty(count, dtype=torch.int32, device="cuda")
    if out.numel() < count:
        raise ValueError("out is smaller than count")
    paux = _dptr(aux, torch.int32, "aux") if aux is not None else None
    if aux is not None and aux.numel() < count:
        raise ValueError("aux is smaller than count")
    _check(lib().hp_phenotype_map(structs.handle, begin, count, gap_threshold, _dptr(out, torch.int32, "out"), paux,
                                  _stream_ptr(stream)))
    return out


def tile_cfg_list():
    """Compiled kernel shapes (reg_bits, tile) (hp_tile_cfg_list)."""
    n = ctypes.c_int32(0)
    _check(lib().hp_tile_cfg_list(None, ctypes.byref(n)))
    arr = (TileCfg * n.value)()
    _check(lib().hp_tile_cfg_list(arr, ctypes.byref(n)))
    return [(c.reg_bits, c.tile) for c in arr]


def _batch_args(structs, ranges, outs, cfg):
    import torch

    n = len(structs)
    if not (len(ranges) == len(outs) == n):
        raise ValueError("structs, ranges and outs must have the same length")
    libs = (ctypes.c_void_p * n)(*[s.handle.value for s in structs])
    begins = (ctypes.c_uint64 * n)(*[int(r[0]) for r in ranges])
    counts = (ctypes.c_uint64 * n)(*[int(r[1]) for r in ranges])
    for o, r in zip(outs, ranges):
        if o.numel() < int(r[1]):
            raise ValueError("an output is smaller than its range")
    ptrs = (ctypes.c_void_p * n)(*[_dptr(o, torch.int32, "out").value for o in outs])
    c = ctypes.byref(TileCfg(*cfg)) if cfg is not None else None
    return libs, begins, counts, n, ptrs, c


def phenotype_map_batch(structs, ranges, outs, cfg=None, stream=None, gap_threshold: int = 1):
    """Batched persistent launches for several boxes (hp_phenotype_map_batch, or hp_phenotype_map_batch_gap
    for gap_threshold > 1); ranges = [(begin, count)]."""
    libs, begins, counts, n, ptrs, c = _batch_args(structs, ranges, outs, cfg)
    if gap_threshold == 1:
        _check(lib().hp_phenotype_map_batch(libs, begins, counts, n, ptrs, c, _stream_ptr(stream)))
    else:
        if cfg is not None:
            raise ValueError("a threshold above 1 runs the one compiled gap shape; cfg must be None")
        _check(lib().hp_phenotype_map_batch_gap(libs, begins, counts, n, int(gap_threshold), ptrs, _stream_ptr(stream)))
    return outs


class BatchPlan:
    """A batch captured into a CUDA graph (hp_batch_plan_*); keeps its inputs alive."""

    def __init__(self, structs, ranges, outs, cfg=None, stream=None):
        self._keep = (list(structs), list(outs))
        libs, begins, counts, n, ptrs, c = _batch_args(structs, ranges, outs, cfg)
        h = ctypes.c_void_p()
        _check(lib().hp_batch_plan_create(libs, begins, counts, n, ptrs, c, _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(lib().hp_batch_plan_launch(self._h, _stream_ptr(stream)))

    def status(self, stream=None):
        _check(lib().hp_batch_plan_status(self._h, _stream_ptr(stream)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.hp_batch_plan_free(h)
            self._h = None


def sequence_scan(structs: Structs, ids, cand=None, aux=False, counters=None, stream=None, gap_threshold=1,
                  gaps=False):
    """Phenotypes of arbitrary ids (hp_sequence_scan, or hp_sequence_scan_gap for gap_threshold > 1 or
    gaps); cand: int32 [n, k] candidate conformations or None.  Returns phen, then aux and the int32
    energy gaps E2 - E1 in that order when requested; counters (int64[2] CUDA tensor) accumulates
    (conformations evaluated exactly, contact-count group bounds evaluated)."""
    import torch

    n = ids.numel()
    if ids.dtype != torch.int64:
        raise TypeError("ids must be int64 (bit patterns of uint64 ids)")
    phen = torch.empty(n, dtype=torch.int32, device=ids.device)
    ax = torch.empty(n, dtype=torch.int32, device=ids.device) if aux else None
    gp = torch.empty(n, dtype=torch.int32, device=ids.device) if gaps else None
    k = 0
    pc = None
    if cand is not None:
        if cand.dim() != 2 or cand.shape[0] != n:
            raise ValueError("cand must be [n, k]")
        k = cand.shape[1]
        pc = _dptr(cand, torch.int32, "cand")
    pids = _dptr(ids, torch.int64, "ids")
    pphen = _dptr(phen, torch.int32, "phen")
    pax = _dptr(ax, torch.int32, "aux") if aux else None
    pcnt = _dptr(counters, torch.int64, "counters") if counters is not None else None
    if gap_threshold == 1 and not gaps:
        _check(lib().hp_sequence_scan(structs.handle, pids, n, pc, k, pphen, pax, pcnt, _stream_ptr(stream)))
    else:
        _check(lib().hp_sequence_scan_gap(structs.handle, pids, n, pc, k, int(gap_threshold), pphen, pax,
                                          _dptr(gp, torch.int32, "gaps") if gaps else None, pcnt,
                                          _stream_ptr(stream)))
    out = (phen,) + ((ax,) if aux else ()) + ((gp,) if gaps else ())
    return out if len(out) > 1 else phen


class MLP:
    """The learned proposal network (hp_mlp_*): N -> H1 -> H2 -> S, ReLU, softmax; bf16 GEMMs, fp32 Adam."""

    def __init__(self, N, H1, H2, S, max_batch, params):
        """params: six float32 numpy arrays W1 [H1,N], b1, W2 [H2,H1], b2, W3 [S,H2], b3."""
        self.N, self.H1, self.H2, self.S, self.max_batch = N, H1, H2, S, max_batch
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in params]
        shapes = [(H1, N), (H1,), (H2, H1), (H2,), (S, H2), (S,)]
        for a, sh in zip(arrs, shapes):
            if a.shape != sh:
                raise ValueError(f"parameter shape {a.shape} != {sh}")
        ptrs = (ctypes.c_void_p * 6)(*[a.ctypes.data for a in arrs])
        h = ctypes.c_void_p()
        _check(lib().hp_mlp_create(N, H1, H2, S, max_batch, ptrs, ctypes.byref(h)))
        self._h = h
        self._shapes = shapes

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.hp_mlp_free(h)
            self._h = None

    def gradients(self, ids, labels, stream=None):
        """(mean loss, [six fp32 numpy gradients]) without updating."""
        import torch

        grads = [np.zeros(sh, dtype=np.float32) for sh in self._shapes]
        ptrs = (ctypes.c_void_p * 6)(*[g.ctypes.data for g in grads])
        loss = ctypes.c_float()
        _check(lib().hp_mlp_gradients(self._h, _dptr(ids, torch.int64, "ids"), _dptr(labels, torch.int32, "labels"),
                                      ids.numel(), ptrs, ctypes.byref(loss), _stream_ptr(stream)))
        return loss.value, grads

    def train_step(self, ids, labels, lr, want_loss=False, stream=None):
        import torch

        loss = ctypes.c_float()
        _check(lib().hp_mlp_train_step(self._h, _dptr(ids, torch.int64, "ids"), _dptr(labels, torch.int32, "labels"),
                                       ids.numel(), ctypes.c_float(lr), ctypes.byref(loss) if want_loss else None,
                                       _stream_ptr(stream)))
        return loss.value if want_loss else None

    def logits(self, ids, stream=None):
        import torch

        out = torch.empty((ids.numel(), self.S), dtype=torch.float32, device=ids.device)
        _check(lib().hp_mlp_logits(self._h, _dptr(ids, torch.int64, "ids"), ids.numel(), _dptr(out, torch.float32, "out"),
                                   _stream_ptr(stream)))
        return out

    def topk(self, ids, k, stream=None):
        import torch

        out = torch.empty((ids.numel(), k), dtype=torch.int32, device=ids.device)
        _check(lib().hp_mlp_topk(self._h, _dptr(ids, torch.int64, "ids"), ids.numel(), k, _dptr(out, torch.int32, "out"),
                                 _stream_ptr(stream)))
        return out

    def status(self, stream=None):
        """Drain the stream; raise HPError if a GEMM's bounded wait gave up since the last check."""
        _check(lib().hp_mlp_status(self._h, _stream_ptr(stream)))


def proposal_conformations(structs: Structs, top, stream=None):
    """[n, k] classes -> [n, 2k] conformations (hp_proposal_conformations)."""
    import torch

    n, k = top.shape
    cand = torch.empty((n, 2 * k), dtype=torch.int32, device=top.device)
    _check(lib().hp_proposal_conformations(structs.handle, _dptr(top.contiguous(), torch.int32, "top"), n, k,
                                           _dptr(cand, torch.int32, "cand"), _stream_ptr(stream)))
    return cand


def _hist_out_checks(phen, S: int, out, name: str):
    """Refuse, before any launch, an output too short for S + 1 counts or tensors on different devices:
    the entry point writes S + 1 uint64 counts and launches on the current device."""
    if S < 1:
        raise HPError(HP_EINVAL, f"{name}: S must be >= 1")
    if out.numel() < S + 1:
        raise HPError(HP_EINVAL, f"{name}: out holds {out.numel()} counts, S + 1 = {S + 1} are written")
    if out.device != phen.device:
        raise HPError(HP_EINVAL, f"{name}: phen ({phen.device}) and out ({out.device}) are on different devices")


def designability(phen, S: int, out=None, stream=None):
    """Designability N_p (hp_designability): int64[S + 1], index S counts -1."""
    import torch

    if out is None:
        out = torch.empty(S + 1, dtype=torch.int64, device=phen.device)
    _hist_out_checks(phen, S, out, "designability")
    pp, po = _dptr(phen, torch.int32, "phen"), _dptr(out, torch.int64, "out")
    with torch.cuda.device(phen.device):
        _check(lib().hp_designability(pp, phen.numel(), S, po, _stream_ptr(stream)))
    return out


def designability_noalloc(phen, S: int, out, stream=None):
    """hp_designability_noalloc: designability into a caller-provided int64[S+1] tensor, with no device
    allocation by the library (scratch is a static device array shared by all calls)."""
    import torch

    _hist_out_checks(phen, S, out, "designability_noalloc")
    pp, po = _dptr(phen, torch.int32, "phen"), _dptr(out, torch.int64, "out")
    with torch.cuda.device(phen.device):
        _check(lib().hp_designability_noalloc(pp, phen.numel(), S, po, _stream_ptr(stream)))
    return out


def robustness(phen, N: int, S: int, stream=None):
    """(neutral[S+1], to_del[S+1]) numerators of Eq. 2 over a full 2^N map (hp_robustness)."""
    import torch

    if phen.numel() != (1 << N):
        raise ValueError("robustness needs the full map of 2^N sequences")
    neutral = torch.empty(S + 1, dtype=torch.int64, device=phen.device)
    to_del = torch.empty(S + 1, dtype=torch.int64, device=phen.device)
    _check(lib().hp_robustness(_dptr(phen, torch.int32, "phen"), N, S, _dptr(neutral, torch.int64, "neutral"),
                               _dptr(to_del, torch.int64, "to_del"), _stream_ptr(stream)))
    return neutral, to_del


def neighbourhood(phen, N: int, S: int, q: int, stream=None):
    """Row q of the Eq. 2 numerators (hp_neighbourhood): int64[S+1], index S for -1."""
    import torch

    if phen.numel() != (1 << N):
        raise ValueError("the neighbourhood needs the full map of 2^N sequences")
    row = torch.empty(S + 1, dtype=torch.int64, device=phen.device)
    _check(lib().hp_neighbourhood(_dptr(phen, torch.int32, "phen"), N, S, q, _dptr(row, torch.int64, "row"),
                                  _stream_ptr(stream)))
    return row


def phi_matrix(phen, N: int, S: int, cap: int | None = None, stream=None):
    """The Eq. 2 numerator matrix in compressed rows (hp_phi_matrix): (row_ptr int64[S+2], col int32[nnz],
    count int64[nnz]); row and column S stand for -1.  cap: output capacity, grown and retried when
    the call reports that the matrix is larger."""
    import torch

    if phen.numel() != (1 << N):
        raise ValueError("the phi matrix needs the full map of 2^N sequences")
    cap = int(cap or max(1 << 16, 8 * (S + 1)))
    pp = _dptr(phen, torch.int32, "phen")
    row_ptr = torch.empty(S + 2, dtype=torch.int64, device=phen.device)
    while True:
        col = torch.empty(cap, dtype=torch.int32, device=phen.device)
        count = torch.empty(cap, dtype=torch.int64, device=phen.device)
        nnz = ctypes.c_uint64(0)
        with torch.cuda.device(phen.device):
            rc = lib().hp_phi_matrix(pp, N, S, cap, _dptr(row_ptr, torch.int64, "row_ptr"), _dptr(col, torch.int32, "col"),
                                     _dptr(count, torch.int64, "count"), ctypes.byref(nnz), _stream_ptr(stream))
        if rc == HP_ENOMEM and cap < (1 << 30) and "cap" in lib().hp_last_error().decode():
            cap = min(1 << 30, max(2 * cap, int(nnz.value)))
            continue
        _check(rc)
        return row_ptr, col[: nnz.value], count[: nnz.value]


def stream_shards(structs: Structs, shard_bits: int, window: int | None = None, out_dir: str | None = None,
                  stream=None):
    """hp_stream_shards: (hist, neutral, to_del) numpy uint64 [S+1] over the whole space, and the number of
    shard maps computed (fewer on a resumed run)."""
    S = structs.S
    hist = np.zeros(S + 1, dtype=np.uint64)
    neutral = np.zeros(S + 1, dtype=np.uint64)
    to_del = np.zeros(S + 1, dtype=np.uint64)
    computed = ctypes.c_int32(0)
    if window is None:
        window = (1 << (shard_bits - 1)) + 1 if shard_bits > 0 else 1
    _check(lib().hp_stream_shards(structs.handle, shard_bits, window, out_dir.encode() if out_dir else None,
                                  hist.ctypes.data_as(ctypes.c_void_p), neutral.ctypes.data_as(ctypes.c_void_p),
                                  to_del.ctypes.data_as(ctypes.c_void_p), ctypes.byref(computed),
                                  _stream_ptr(stream) if _cuda_ready() else None))
    return hist, neutral, to_del, computed.value


def stream_components(structs: Structs, shard_bits: int, window: int | None = None, stream=None):
    """hp_stream_components: (ncomp numpy uint64[S], shard maps computed) over the whole space."""
    ncomp = np.zeros(structs.S, dtype=np.uint64)
    computed = ctypes.c_int32(0)
    if window is None:
        window = (1 << (shard_bits - 1)) + 1 if shard_bits > 0 else 1
    _check(lib().hp_stream_components(structs.handle, shard_bits, window, ncomp.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.byref(computed), _stream_ptr(stream) if _cuda_ready() else None))
    return ncomp, computed.value


def _cuda_ready():
    try:
        import torch

        return torch.cuda.is_available()
    except ImportError:
        return False


def neutral_components(phen, N: int, S: int, stream=None, out_label=None):
    """(label[2^N], ncomp[S]) of the neutral networks (hp_neutral_components); the labels go to
    out_label (int32[2^N] on the map's device) when it is given."""
    import torch

    if phen.numel() != (1 << N):
        raise ValueError("components need the full map of 2^N sequences")
    if out_label is not None:
        if out_label.dtype != torch.int32 or out_label.numel() != (1 << N) or out_label.device != phen.device:
            raise HPError(HP_EINVAL, "neutral_components: out_label must be int32[2^N] on the map's device")
        label = out_label
    else:
        label = torch.empty(1 << N, dtype=torch.int32, device=phen.device)
    ncomp = torch.empty(S, dtype=torch.int64, device=phen.device)
    _check(lib().hp_neutral_components(_dptr(phen, torch.int32, "phen"), N, S, _dptr(label, torch.int32, "label"),
                                       _dptr(ncomp, torch.int64, "ncomp"), _stream_ptr(stream)))
    return label, ncomp
