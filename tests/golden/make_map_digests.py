"""Write tests/golden/map_digests.json: digests of oracle phenotype maps for whole-map parity.

Calls only the CPU oracle (oracle/) and the seeded input generators; nothing here touches the
CUDA library.  For each case the oracle computes the phenotypes (Section 2.1: ground state with
threshold 1, reading B) and the lowest-index minimising class (the aux output) of a range or a
seeded sample of sequence ids; the stored values are, per chunk of 2^chunk_bits consecutive
entries, the first 16 hex digits of the SHA-256 of the int32 little-endian bytes, plus the
designability histogram of the whole case (its -1 count, designable classes, maximum and digest).  A GPU
map is compared chunk by chunk, so a mismatch names the chunk that holds it.

    python tests/golden/make_map_digests.py [case ...] [--threads T]

Cases (all ids of a box or a seeded part of it):
  4x5        the whole 4x5 space (2^20 ids)
  5x5        the whole 5x5 space (2^25 ids)
  2x3x4      the whole 2x3x4 space (2^24 ids)
  3x3x3blk   a 2^20-id aligned block of 3x3x3 at a seeded offset
  3x3x3smp   2^16 seeded 3x3x3 ids
  6x6smp     2^16 seeded 6x6 ids spread over the seeded 2^32-id shards
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2008_05612_gb300 import inputs  # noqa: E402  (seeded generators only)

OUT = os.path.join(HERE, "map_digests.json")


def chunk_digests(a: np.ndarray, chunk_bits: int):
    a = np.ascontiguousarray(a, dtype="<i4")
    step = 1 << chunk_bits
    return [hashlib.sha256(a[i:i + step].tobytes()).hexdigest()[:16] for i in range(0, a.shape[0], step)]


def histogram(phen: np.ndarray, S: int):
    """Designability of the case (oracle.designability: uint64[S + 1], index S for -1), summarised."""
    h = oracle.designability(phen, S)
    return {"minus1": int(h[S]), "designable": int((h[:S] > 0).sum()), "max": int(h[:S].max()),
            "sha": hashlib.sha256(np.ascontiguousarray(h, dtype="<u8").tobytes()).hexdigest()[:16]}


def case_ids(name: str):
    """(dims, ids, description) of a case; ids are the seeded generators' output, never a map's."""
    if name == "4x5":
        return (4, 5), np.arange(1 << 20, dtype=np.uint64), "all 2^20 ids"
    if name == "5x5":
        return (5, 5), np.arange(1 << 25, dtype=np.uint64), "all 2^25 ids"
    if name == "2x3x4":
        return (2, 3, 4), np.arange(1 << 24, dtype=np.uint64), "all 2^24 ids"
    if name == "3x3x3blk":
        base = int(inputs.sample_ids(7, 1, seed=901)[0]) << 20  # one of the 128 aligned 2^20 blocks
        return (3, 3, 3), np.arange(base, base + (1 << 20), dtype=np.uint64), f"ids [{base}, {base} + 2^20)"
    if name == "3x3x3smp":
        return (3, 3, 3), inputs.sample_ids(27, 1 << 16, seed=902), "inputs.sample_ids(27, 2^16, seed=902)"
    if name == "6x6smp":
        # 2^14 ids in each of four seeded 2^32-id shards (shard k = the top 4 of the 36 bits)
        parts = []
        for j in range(4):
            k = inputs.shard_index(j)
            low = inputs.sample_ids(32, 1 << 14, seed=903 + j)
            parts.append(low | (np.uint64(k) << np.uint64(32)))
        return (6, 6), np.concatenate(parts), "2^14 ids of each shard inputs.shard_index(j), j < 4, low bits sample_ids(32, 2^14, seed=903 + j)"
    raise KeyError(name)


CASES = ("4x5", "5x5", "3x3x3smp", "6x6smp", "3x3x3blk", "2x3x4")


def main(argv):
    threads = None
    names = []
    it = iter(argv)
    for a in it:
        if a == "--threads":
            threads = int(next(it))
        else:
            names.append(a)
    names = names or list(CASES)
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        dims, ids, desc = case_ids(name)
        box = oracle.Box(dims)
        t = time.time()
        phen, aux = box.phenotypes(ids, aux=True, nthreads=threads)
        dt = time.time() - t
        chunk_bits = 16 if ids.shape[0] >= (1 << 20) else 12
        data[name] = {
            "dims": list(dims), "N": box.N, "S": box.S, "S_dir": box.S_dir, "ids": desc, "count": int(ids.shape[0]),
            "chunk_bits": chunk_bits, "phen": chunk_digests(phen, chunk_bits), "aux": chunk_digests(aux, chunk_bits),
            "designability": histogram(phen, box.S),
            "oracle_seconds": round(dt, 1), "threads": threads or min(os.cpu_count() or 1, 64),
        }
        print(f"{name}: {ids.shape[0]} ids x {box.S_dir} conformations in {dt:.1f} s", flush=True)
        data["_source"] = ("oracle/ (reading B, threshold 1) via tests/golden/make_map_digests.py; "
                           "digest = sha256(int32 LE bytes)[:16] per chunk")
        tmp = OUT + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, OUT)


if __name__ == "__main__":
    main(sys.argv[1:])
