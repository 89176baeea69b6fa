"""Benchmark of the HP genotype-phenotype map hot path on GB300.

One step = the whole map path over the full 3x3x3 sequence space (2^27 HP
sequences x 103,346 directed conformations): phenotype map, designability,
robustness / phi_del numerators and neutral components.  Metric: sequence x
conformation evaluations per second (and sequences per second).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the CPU oracle (the only reference this project has:
the paper ships no runnable code) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HP seq×struct evals/s & sequences/s (3x3x3, 6x6); learned-pruned vs plain"
DIMS = (3, 3, 3)
WORKLOAD = "3x3x3 full map: all 2^27 HP sequences x 103,346 directed conformations (51,704 classes)"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one full 3x3x3 phenotype-kernel launch, from
# an ncu capture of the current kernel; None whenever the kernel has changed since the last capture.
TRAFFIC_PER_LAUNCH = 1_757_442_304
# ALU lane-ops per sequence x conformation evaluation of the map kernel's pass 1 (default shape)
ALU_OPS_PER_EVAL = 24 / 64


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value: float) -> float:
    """Largest value over all ranks (the job's time is its slowest rank); identity without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank processes units_per_rank per step (weak scaling)."""
    return world * units_per_rank / (ms_per_step * 1e-3)


def performed_sequences(N: int) -> int:
    """Sequences the map kernel evaluates for the full space of an N-residue chain."""
    if N % 2 == 0:
        return 1 << N
    no, ne = N // 2, N // 2 + 1
    canonical = ((1 << no) + (1 << ((no + 1) // 2))) // 2  # odd patterns with o <= reverse(o)
    return canonical << ne


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_baseline(dims, budget_s: float = 12.0):
    """The oracle as it stands, on all host cores, on a bounded seeded sample of the workload."""
    import oracle
    from paper_2008_05612_gb300 import inputs

    b = oracle.Box(dims)
    cores = os.cpu_count() or 1
    n = 64
    ids = inputs.sample_ids(b.N, n, seed=41)
    t = time.perf_counter()
    b.phenotypes(ids, nthreads=cores)
    dt = time.perf_counter() - t
    n = int(max(64, min(200000, n * budget_s / max(dt, 1e-3))))
    ids = inputs.sample_ids(b.N, n, seed=43)
    t = time.perf_counter()
    b.phenotypes(ids, nthreads=cores)
    dt = time.perf_counter() - t
    evals = n * b.S_dir
    return {"value": evals / dt, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} seeded 3x3x3 sequences x {b.S_dir} conformations (direct contact sums), {dt:.1f} s",
            "sequences_per_s": n / dt}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2008_05612_gb300 import inputs

    b = oracle.Box(DIMS)
    cores = os.cpu_count() or 1
    n = 2048 * max(1, cores // 8)
    ids = inputs.sample_ids(b.N, n, seed=47)
    for _ in range(args.warmup):
        b.phenotypes(ids[:256], nthreads=cores)
    times = []
    for k in range(args.steps):
        t = time.perf_counter()
        b.phenotypes(inputs.sample_ids(b.N, n, seed=100 + k), nthreads=cores)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    evals = n * b.S_dir * args.steps
    v = evals / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic (exhaustive sequence space, seeded sample)",
            "config": {"workload": WORKLOAD + f"; oracle timed on a seeded sample of {n} sequences per step"},
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} seeded sequences per step"},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sequences_per_s": n * args.steps / tot}
    print(json.dumps(line))
    return 0


def map_statistics(hist, neutral, to_del, N, S):
    """Section 3.2 statistics of a whole-space map from exact counters (index S is -1)."""
    hist = hist.astype(np.int64)
    neutral = neutral.astype(np.int64)
    to_del = to_del.astype(np.int64)
    total = int(hist.sum())
    d = hist[:S] > 0
    Np = hist[:S][d].astype(np.float64)
    rho = neutral[:S][d] / (N * Np)
    phid = to_del[:S][d] / (N * Np)
    other = 1.0 - rho - phid
    flips_other = N * int(hist[:S].sum()) - int(neutral[:S].sum()) - int(to_del[:S].sum())
    return {
        "sequences": total,
        "fold_fraction": 1.0 - hist[S] / total,
        "designable": int(d.sum()),
        "classes": S,
        "top_designability": int(hist[:S].max()),
        "mean_robustness": float(rho.mean()),
        "mean_phi_del": float(phid.mean()),
        "mean_other_fraction": float(other.mean()),
        "isolated": int(((neutral[:S] + to_del[:S])[d] == N * hist[:S][d]).sum()),
        "checks": {
            "sum_designability_is_2^N": total == (1 << N),
            "neutral_counts_even": bool((neutral % 2 == 0).all()),
            "minus1_row_consistent": int(neutral[S]) == int(to_del[S]),
            "flips_other_nonnegative": flips_other >= 0,
        },
    }


def run_stream(args):
    """The whole space of a box through the shard streamer (hp_stream_shards)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2008_05612_gb300 as hp

    parts = args.stream.split(":")
    dims = tuple(int(x) for x in parts[0].split("x"))
    bits = int(parts[1])
    window = int(parts[2]) if len(parts) > 2 and parts[2] else None
    out_dir = parts[3] if len(parts) > 3 else None
    s = hp.Structs(dims)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist, neutral, to_del, computed = hp.stream_shards(s, bits, window=window, out_dir=out_dir)
    dt = time.perf_counter() - t0
    evals = (1 << s.N) * s.S_dir
    line = {"case": f"stream {args.stream}", "box": parts[0], "N": s.N, "S": s.S, "S_dir": s.S_dir,
            "shards": 1 << bits, "maps_computed": computed, "seconds": dt,
            "evals_per_s": evals / dt if computed == (1 << bits) else None,
            "statistics": map_statistics(hist, neutral, to_del, s.N, s.S)}
    print(json.dumps(line))
    return 0


def run_stream_components(args):
    """Neutral-network counts of the whole space of a box through shards (hp_stream_components)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2008_05612_gb300 as hp

    parts = args.stream_components.split(":")
    dims = tuple(int(x) for x in parts[0].split("x"))
    bits = int(parts[1])
    window = int(parts[2]) if len(parts) > 2 and parts[2] else None
    s = hp.Structs(dims)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ncomp, computed = hp.stream_components(s, bits, window=window)
    dt = time.perf_counter() - t0
    nz = ncomp[ncomp > 0]
    print(json.dumps({"case": f"stream components {args.stream_components}", "box": parts[0], "N": s.N, "S": s.S,
                      "shards": 1 << bits, "maps_computed": computed, "seconds": dt,
                      "components": int(ncomp.sum()), "phenotypes_with_components": int(nz.size),
                      "max_components_of_a_phenotype": int(ncomp.max()),
                      "phenotypes_with_one_component": int((ncomp == 1).sum())}))
    return 0


def run_map_only(args):
    """Phenotype map of one aligned id block, W + K launches, CUDA-event timed (a small case for ncu)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2008_05612_gb300 as hp

    box, bits = args.map_only.split(":")
    dims = tuple(int(x) for x in box.split("x"))
    bits = int(bits)
    s = hp.Structs(dims)
    n = 1 << bits
    phen = torch.empty(n, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        hp.phenotype_map(s, 0, n, out=phen)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        hp.phenotype_map(s, 0, n, out=phen)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"case": args.map_only, "ms_per_launch": ms, "evals_per_s": n * s.S_dir / (ms * 1e-3),
                      "sequences": n, "conformations": s.S_dir}))
    return 0


def map_block_6x6(hp, torch, peak_ops: float, bits: int = 27, reps: int = 3):
    """The metric's second box: the 6x6 phenotype map of the aligned id block [0, 2^bits) (every id of the
    block is evaluated: 6x6 is an even chain, so there is no reversal half enumeration), 1 warm-up + `reps`
    launches timed with CUDA events on the launching stream."""
    s = hp.Structs((6, 6))
    n = 1 << bits
    phen = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    hp.phenotype_map(s, 0, n, out=phen)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        hp.phenotype_map(s, 0, n, out=phen)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    evals = n * s.S_dir
    achieved = ALU_OPS_PER_EVAL * evals / (ms * 1e-3)
    folded = int((phen >= 0).sum().item())
    return {"workload": f"6x6 phenotype map of ids [0, 2^{bits}) x {s.S_dir} conformations ({s.S} classes)",
            "map_ms": ms, "evals_per_s": evals / (ms * 1e-3), "sequences_per_s": n / (ms * 1e-3),
            "fold_fraction": folded / n,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "ALU lane-ops/s",
                         "frac": achieved / peak_ops, "kernel": "phenotype_kernel<Cfg<5,256>, false>",
                         "note": "0.375 ALU lane-ops per performed evaluation (all 2^27 ids of the block are evaluated)"}}


BATCH_BOXES = ((4, 4), (4, 5), (5, 5), (2, 3, 4), (3, 3, 3))


def small_boxes_and_batch(hp, torch, reps: int = 3):
    """Whole maps of the other boxes of the batched workload, one launch each (CUDA events, 1 warm-up +
    `reps` launches), and the same five maps in ONE persistent batched launch."""
    stream = torch.cuda.current_stream()
    libs = [hp.Structs(d) for d in BATCH_BOXES]
    outs = [torch.empty(1 << s.N, dtype=torch.int32, device="cuda") for s in libs]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    singles = {}
    for d, s, o in zip(BATCH_BOXES, libs, outs):
        ms = timed(lambda: hp.phenotype_map(s, 0, 1 << s.N, out=o))
        n = 1 << s.N
        performed = performed_sequences(s.N) * s.S_dir
        singles["x".join(map(str, d))] = {"sequences": n, "conformations": s.S_dir, "map_ms": ms,
                                          "evals_per_s": n * s.S_dir / (ms * 1e-3),
                                          "performed_evals_per_s": performed / (ms * 1e-3)}
    ranges = [(0, 1 << s.N) for s in libs]
    ms_batch = timed(lambda: hp.phenotype_map_batch(libs, ranges, outs))
    total = sum((1 << s.N) * s.S_dir for s in libs)
    return {"singles": singles, "batch": {"boxes": ["x".join(map(str, d)) for d in BATCH_BOXES], "map_ms": ms_batch,
                                          "sum_of_singles_ms": sum(v["map_ms"] for v in singles.values()),
                                          "evals_per_s": total / (ms_batch * 1e-3)}}


PROPOSAL_ROWS = 16384  # ids per proposal chunk (the network's max_batch)


def proposal_params(N, S, H: int = 512):
    from paper_2008_05612_gb300 import inputs

    return [inputs.init_weights((H, N), N, 61), inputs.init_weights((H,), N, 62),
            inputs.init_weights((H, H), H, 63), inputs.init_weights((H,), H, 64),
            inputs.init_weights((S, H), H, 65), inputs.init_weights((S,), H, 66)]


def train_proposal(hp, s, torch, tids, tlab, epochs: float = 1.0, batch: int = 4096, lr: float = 1e-3, width: int = 512):
    """N -> width -> width -> S network trained on the GPU with the library's kernels (one Adam step per
    batch of `batch` (id, label) pairs, `epochs` passes over the training set); returns (trained, untrained,
    info)."""
    N, S = s.N, s.S
    params = proposal_params(N, S, width)
    net = hp.MLP(N, width, width, S, PROPOSAL_ROWS, params)
    untrained = hp.MLP(N, width, width, S, PROPOSAL_ROWS, params)
    steps = max(1, int(epochs * tids.numel() / batch))
    gen = torch.Generator(device="cuda").manual_seed(0)
    perm = torch.randperm(tids.numel(), device="cuda", generator=gen)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    first_loss = last_loss = None
    for st in range(steps):
        j = perm[st * batch % (tids.numel() - batch):][:batch]
        want = st == 0 or st == steps - 1
        loss = net.train_step(tids[j].contiguous(), tlab[j].contiguous(), lr, want_loss=want)
        if st == 0:
            first_loss = loss
        if st == steps - 1:
            last_loss = loss
    torch.cuda.synchronize()
    net.status()
    info = {"train_ids": int(tids.numel()), "train_steps": steps, "batch": batch, "lr": lr,
            "train_s": time.perf_counter() - t0, "loss_first": first_loss, "loss_last": last_loss}
    return net, untrained, info


def compare_on_ids(hp, s, torch, ev, models, k: int = 4, plain=None):
    """Plain per-sequence scan vs (network top-k + candidate expansion + pruned scan) on the same ids,
    CUDA-event timed (1 warm-up + 3 calls); phenotypes must agree exactly.  With `plain` (the plain
    scan's phenotypes of `ev`) given, the plain scan is not run again."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = ev.numel()

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / reps

    res = {}
    if plain is None:
        plain, ms_plain = timed(lambda: hp.sequence_scan(s, ev))
        res["plain_per_sequence"] = {"ms": ms_plain, "sequences_per_s": n / (ms_plain * 1e-3)}
    for name, model in models.items():
        cnt = torch.zeros(2, dtype=torch.int64, device="cuda")

        def learned():
            cand = hp.proposal_conformations(s, model.topk(ev, k))
            return hp.sequence_scan(s, ev, cand=cand, counters=cnt)

        out, ms = timed(learned)
        _, ms_prop = timed(lambda: hp.proposal_conformations(s, model.topk(ev, k)))
        model.status()
        exact = int(cnt[0]) / 4  # four calls accumulated (warm-up + 3 timed)
        bounds = int(cnt[1]) / 4
        res[name] = {"ms": ms, "ms_proposal": ms_prop, "sequences_per_s": n / (ms * 1e-3),
                     "exact_eval_fraction": exact / (n * s.S_dir), "group_bounds_per_sequence": bounds / n,
                     "mismatches_vs_plain": int((out != plain).sum().item())}
    return res


def learned_full_space(hp, s, torch, net, phen, k: int = 4, chunk: int = 1 << 20):
    """The learned + pruned form over EVERY id of the box, compared with the exhaustive map `phen`;
    CUDA events around each chunk's proposal + expansion + pruned scan (the id ranges are made and the
    comparison is done outside them)."""
    total = 1 << s.N
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    mism = torch.zeros((), dtype=torch.int64, device="cuda")
    evs = []
    for off in range(0, total, chunk):
        ids = torch.arange(off, min(off + chunk, total), dtype=torch.int64, device="cuda")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        cand = hp.proposal_conformations(s, net.topk(ids, k))
        got = hp.sequence_scan(s, ids, cand=cand, counters=cnt)
        b.record()
        evs.append((a, b))
        mism += (got != phen[off:off + ids.numel()]).sum()
    torch.cuda.synchronize()
    net.status()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    return {"ids": total, "ms": ms, "sequences_per_s": total / (ms * 1e-3),
            "exact_eval_fraction": int(cnt[0]) / (total * s.S_dir), "mismatches_vs_exhaustive_map": int(mism.item())}


def labels_3x3x3(hp, s, torch):
    """The exhaustive map of the box, its CUDA-event time, and the training set: the seeded 1-in-10
    sample of the space labelled with the lowest-index minimiser (aux output) of the map kernel."""
    from paper_2008_05612_gb300 import inputs

    N = s.N
    phen = torch.empty(1 << N, dtype=torch.int32, device="cuda")
    aux = torch.empty(1 << N, dtype=torch.int32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    hp.phenotype_map(s, 0, 1 << N, out=phen, aux=aux)
    e1.record()
    torch.cuda.synchronize()
    ms_map = e0.elapsed_time(e1)
    ids_all = np.arange(1 << N, dtype=np.uint64)
    train_ids = ids_all[inputs.training_mask(ids_all)]
    del ids_all
    tids = torch.from_numpy(train_ids.view(np.int64)).to("cuda")
    tlab = aux[tids]
    return phen, ms_map, tids, tlab


def learned_leg(hp, s, torch, full_space: bool = True, eval_n: int = 1 << 16, k: int = 4):
    """3x3x3: labels = the lowest-index minimiser (aux output) of the exhaustive kernel's full map on the
    seeded 1-in-10 sample of the space; evaluation on `eval_n` seeded ids and on the whole space."""
    from paper_2008_05612_gb300 import inputs

    N = s.N
    phen, ms_map, tids, tlab = labels_3x3x3(hp, s, torch)
    net, untrained, info = train_proposal(hp, s, torch, tids, tlab)
    del tids, tlab
    ev = torch.from_numpy(inputs.sample_ids(N, eval_n, seed=123).view(np.int64)).to("cuda")
    res = compare_on_ids(hp, s, torch, ev, {"learned_pruned": net, "untrained_pruned": untrained}, k)
    out = {"box": "3x3x3", "labels": "aux output of the exhaustive map kernel, seeded 1-in-10 sample of the space", **info,
           "eval_ids": eval_n, "eval": "inputs.sample_ids(27, 65536, seed=123)", "topk": k, **res,
           "exhaustive_map": {"ms": ms_map, "sequences_per_s": (1 << N) / (ms_map * 1e-3)}}
    if full_space:
        out["full_space"] = learned_full_space(hp, s, torch, net, phen, k)
    return out


def proposal_sweep(hp, s, torch, settings=((128, 1.0), (256, 1.0), (512, 1.0), (512, 3.0)), ks=(1, 2, 4, 8, 16),
                   eval_n: int = 1 << 16):
    """3x3x3 learned proposal: hidden width and training epochs (`settings`) against top-k (`ks`); per
    setting the pruned scan's time, proposal time, exact-evaluation fraction and mismatches on `eval_n`
    seeded ids (one JSON line each, then the plain scan's line)."""
    from paper_2008_05612_gb300 import inputs

    _, _, tids, tlab = labels_3x3x3(hp, s, torch)
    ev = torch.from_numpy(inputs.sample_ids(s.N, eval_n, seed=123).view(np.int64)).to("cuda")
    base = compare_on_ids(hp, s, torch, ev, {}, 4)
    plain = hp.sequence_scan(s, ev)
    for width, epochs in settings:
        net, _, info = train_proposal(hp, s, torch, tids, tlab, epochs=epochs, width=width)
        for k in ks:
            res = compare_on_ids(hp, s, torch, ev, {"learned_pruned": net}, k, plain=plain)["learned_pruned"]
            print(json.dumps({"box": "3x3x3", "width": width, "epochs": epochs, "topk": k, "train_s": info["train_s"],
                              "loss_last": info["loss_last"], **res}), flush=True)
        del net
    print(json.dumps({"box": "3x3x3", "eval_ids": eval_n, **base}), flush=True)


def learned_leg_6x6(hp, torch, n_train: int = 13_421_773, eval_per_shard: int = 1 << 15, shards: int = 2, k: int = 4):
    """6x6 (N = 36, the paper's Table 3 sampling workload): labels = the lowest-index minimiser from the plain
    per-sequence scan on seeded uniform ids (the evaluation draws uniform ids, so the training ids do too);
    evaluation on `eval_per_shard` seeded ids of each of `shards` seeded 2^32-id shards (shard k = the top 4
    bits), plain scan vs learned + pruned."""
    from paper_2008_05612_gb300 import inputs

    s = hp.Structs((6, 6))
    N = s.N
    tids = torch.from_numpy(inputs.sample_ids(N, n_train, seed=611).view(np.int64)).to("cuda")
    tlab = torch.empty(n_train, dtype=torch.int32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for off in range(0, n_train, 1 << 20):
        _, a = hp.sequence_scan(s, tids[off:off + (1 << 20)], aux=True)
        tlab[off:off + a.numel()] = a
    e1.record()
    torch.cuda.synchronize()
    label_ms = e0.elapsed_time(e1)
    net, untrained, info = train_proposal(hp, s, torch, tids, tlab)
    del tids, tlab
    parts, kk = [], []
    for j in range(shards):
        kj = inputs.shard_index(j)
        kk.append(kj)
        low = inputs.sample_ids(32, eval_per_shard, seed=700 + j)
        parts.append(low | (np.uint64(kj) << np.uint64(32)))
    ev = torch.from_numpy(np.concatenate(parts).view(np.int64)).to("cuda")
    res = compare_on_ids(hp, s, torch, ev, {"learned_pruned": net, "untrained_pruned": untrained}, k)
    return {"box": "6x6", "labels": f"aux output of the plain per-sequence scan on {n_train} seeded uniform ids",
            "label_ms": label_ms, **info, "eval_ids": int(ev.numel()),
            "eval": f"{eval_per_shard} seeded ids in each of the shards {kk} (inputs.shard_index(j), j < {shards})",
            "topk": k, **res}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal leg")
    ap.add_argument("--learned-only", action="store_true", help="only the learned-proposal leg (one JSON line)")
    ap.add_argument("--proposal-sweep", action="store_true",
                    help="3x3x3 proposal network: hidden width, epochs and top-k against the pruned scan's cost")
    ap.add_argument("--stream", default=None, metavar="BOX:BITS[:WINDOW[:DIR]]",
                    help="whole-space map of BOX in 2^BITS shards with exact designability and Eq. 2 statistics")
    ap.add_argument("--stream-components", default=None, metavar="BOX:BITS[:WINDOW]",
                    help="neutral-network counts per phenotype over the whole space of BOX from 2^BITS shards")
    ap.add_argument("--train-case", action="store_true",
                    help="time the proposal network's training step alone (batch 4096, 3x3x3 classes)")
    ap.add_argument("--proposal-case", action="store_true",
                    help="profiling case: top-4 proposals of an untrained 3x3x3 network for 65,536 ids, W + K times")
    ap.add_argument("--small-boxes", action="store_true",
                    help="only the whole maps of 4x4, 4x5, 5x5, 2x3x4, 3x3x3 one by one and in one batched launch")
    ap.add_argument("--map-only", default=None, metavar="BOX:BITS",
                    help="profiling case: only the phenotype map of ids [0, 2^BITS) of BOX (e.g. 6x6:27)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.map_only:
        return run_map_only(args)
    if args.small_boxes:
        import torch

        import __graft_entry__

        __graft_entry__.build()
        import paper_2008_05612_gb300 as hp

        print(json.dumps(small_boxes_and_batch(hp, torch)))
        return 0
    if args.stream:
        return run_stream(args)
    if args.stream_components:
        return run_stream_components(args)

    import torch

    import __graft_entry__

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    __graft_entry__.build()
    import paper_2008_05612_gb300 as hp

    s = hp.Structs(DIMS)
    N, S, Sdir = s.N, s.S, s.S_dir
    if args.proposal_sweep:
        proposal_sweep(hp, s, torch)
        return 0
    if args.learned_only:
        print(json.dumps({"metric": METRIC, "learned": {"3x3x3": learned_leg(hp, s, torch),
                                                         "6x6": learned_leg_6x6(hp, torch)}}))
        return 0
    if args.train_case:
        from paper_2008_05612_gb300 import inputs

        batch = 4096
        net = hp.MLP(N, 512, 512, S, PROPOSAL_ROWS, proposal_params(N, S))
        ids_np = inputs.sample_ids(N, batch * 8, seed=321)
        ids = torch.from_numpy(ids_np.view(np.int64)).cuda()
        labels = torch.from_numpy((inputs.splitmix64(ids_np) % np.uint64(S)).astype(np.int32)).cuda()
        chunks = [(ids[i * batch:(i + 1) * batch].contiguous(), labels[i * batch:(i + 1) * batch].contiguous())
                  for i in range(8)]
        for i in range(args.warmup):
            net.train_step(*chunks[i % 8], 1e-3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(args.steps):
            net.train_step(*chunks[i % 8], 1e-3)
        e1.record()
        torch.cuda.synchronize()
        net.status()
        ms = e0.elapsed_time(e1) / args.steps
        # forward 2 B (N*512 + 512*512 + 512*S) + backward twice that, per id
        flops = 6.0 * batch * (N * 512 + 512 * 512 + 512 * S)
        print(json.dumps({"case": "training step, batch 4096, 3x3x3 classes", "ms_per_step": ms,
                          "gemm_tflops_equiv": flops / (ms * 1e-3) / 1e12}))
        return 0
    if args.proposal_case:
        from paper_2008_05612_gb300 import inputs

        net = hp.MLP(N, 512, 512, S, PROPOSAL_ROWS, proposal_params(N, S))
        ev = torch.from_numpy(inputs.sample_ids(N, 1 << 16, seed=123).view(np.int64)).cuda()
        for _ in range(args.warmup):
            net.topk(ev, 4)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            net.topk(ev, 4)
        e1.record()
        torch.cuda.synchronize()
        net.status()
        ms = e0.elapsed_time(e1) / args.steps
        flops = 2.0 * ev.numel() * (N * 512 + 512 * 512 + 512 * S)
        print(json.dumps({"case": "proposal top-4, 65536 ids", "ms": ms, "gemm_tflops_equiv": flops / (ms * 1e-3) / 1e12}))
        return 0
    nseq = 1 << N
    stream = torch.cuda.current_stream()
    phen = torch.empty(nseq, dtype=torch.int32, device="cuda")

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        hp.phenotype_map(s, 0, nseq, out=phen)
        if ev is not None:
            ev[1].record(stream)
        hist = hp.designability(phen, S)
        neutral, to_del = hp.robustness(phen, N, S)
        label, ncomp = hp.neutral_components(phen, N, S)
        return hist, neutral, to_del, label, ncomp

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # ---- device-resident timed region (inputs resident: the structure tables are on the device)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0.record(stream)
        for k in range(args.steps):
            out = step(evs[k])
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(t0.elapsed_time(t1))
    map_ms = [a.elapsed_time(b) for a, b in evs]
    ms_step = ms / args.steps
    evals_step = nseq * Sdir
    value = job_value(evals_step, world, ms_step)
    hist = out[0].cpu().numpy()

    # ---- end to end through the public API with host buffers (pinned), copies inside the timed region:
    # each step's map, labels and reductions go to pinned host memory on a copy stream while the next
    # step computes (two sets of buffers); the timed region ends when the last copy has landed
    copy_stream = torch.cuda.Stream()
    d_phen = [phen, torch.empty(nseq, dtype=torch.int32, device="cuda")]
    d_label = [torch.empty(nseq, dtype=torch.int32, device="cuda") for _ in range(2)]
    h_phen = [torch.empty(nseq, dtype=torch.int32, pin_memory=True) for _ in range(2)]
    h_label = [torch.empty(nseq, dtype=torch.int32, pin_memory=True) for _ in range(2)]
    h_small = [[torch.empty(S + 1, dtype=torch.int64, pin_memory=True) for _ in range(3)] +
               [torch.empty(S, dtype=torch.int64, pin_memory=True)] for _ in range(2)]
    copied = [None, None]  # copy-stream event of the buffer set's last copy
    for hb in h_phen + h_label:  # first touch of the pinned pages outside the timed region
        hb.copy_(phen, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(2, args.steps)
    e0.record(stream)
    d2h = 0
    for i in range(e2e_steps):
        b = i & 1
        if copied[b] is not None:
            stream.wait_event(copied[b])
        hp.phenotype_map(s, 0, nseq, out=d_phen[b])
        hist_d = hp.designability(d_phen[b], S)
        neutral, to_del = hp.robustness(d_phen[b], N, S)
        label, ncomp = hp.neutral_components(d_phen[b], N, S, out_label=d_label[b])
        ready = torch.cuda.Event()
        ready.record(stream)
        copy_stream.wait_event(ready)
        with torch.cuda.stream(copy_stream):
            outs = (d_phen[b], label, hist_d, neutral, to_del, ncomp)
            for t in outs:
                t.record_stream(copy_stream)
            h_phen[b].copy_(d_phen[b], non_blocking=True)
            h_label[b].copy_(label, non_blocking=True)
            for h, t in zip(h_small[b], (hist_d, neutral, to_del, ncomp)):
                h.copy_(t, non_blocking=True)
            copied[b] = torch.cuda.Event()
            copied[b].record(copy_stream)
        d2h = (nseq * 2) * 4 + sum(h.numel() for h in h_small[b]) * 8
    for ev in copied:
        if ev is not None:
            stream.wait_event(ev)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps

    peaks = measured_peaks()
    clocks = clk.summary()
    sm_max = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    # ALU-pipe roofline of the phenotype kernel.  Its ALU work per evaluation, counted from the
    # source: per thread, two conformations x 32 sequences (16 packed registers) take 8 three-input
    # packed maxes and 16 fused add + max, i.e. ALU_OPS_PER_EVAL lane-ops per evaluation (the
    # subset-sum additions are IMADs on the FMA pipe).  The ALU pipe retires 64 lane-ops per clock
    # per SM for these instructions (probed with operands that change every iteration) on 152 SMs.
    peak_ops = 64 * 152 * sm_max * 1e6
    map_avg_ms = float(np.mean(map_ms))
    map_evals = evals_step / (map_avg_ms * 1e-3)
    # evaluations the kernel actually performs: for an odd-length chain the full map is computed for one
    # id of each reversal pair (odd-residue patterns o <= reverse(o)) and mirrored
    performed = performed_sequences(N) * Sdir
    achieved = ALU_OPS_PER_EVAL * performed / (map_avg_ms * 1e-3)
    tile_cfg = s.tile_cfg()
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(3, args.warmup),
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic (exhaustive: every sequence of the box; fold library enumerated by the library)",
        "config": {"workload": WORKLOAD, "box": "3x3x3", "sequences": nseq, "conformations": Sdir, "classes": S,
                   "step": "phenotype map + designability + robustness + neutral components",
                   "l2": "map and labels (512 MB each) exceed L2 every step; the 7 MB conformation table stays resident by design",
                   "parallelism": "replicas" if world == 1 else f"replicas x{world}"},
        "sequences_per_s": world * nseq / (ms_step * 1e-3),
        "map_ms": map_avg_ms,
        "map_evals_per_s": map_evals,
        "map_performed_evals": performed,
        "tile_cfg": {"reg_bits": tile_cfg[0], "tile": tile_cfg[1]},
        "fold_fraction": float(1.0 - hist[S] / nseq),
        "gpu_launches": args.steps * (8 + 1 + max(0, -(-(N - 13) // 8))),
        "e2e": {"value": world * evals_step / (e2e_ms * 1e-3), "unit": "evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(d2h),
                "note": "public Python API; each step's map, labels and reductions copied to pinned host memory inside "
                        "the timed region, on a copy stream overlapping the next step's compute (two buffer sets); the "
                        "only input is the sequence range (no per-step input data)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "ALU lane-ops/s",
                     "frac": achieved / peak_ops, "traffic": TRAFFIC_PER_LAUNCH,
                     "kernel": f"phenotype_kernel<Cfg<{tile_cfg[0]},{tile_cfg[1]}>, false>",
                     "peak_source": "64 ALU lane-ops/clk/SM (max.u16x2, three-input max and fused add+max each measured "
                                    "at 63.5 lane-ops/clk/SM on GB300 by a throughput probe) x 152 SMs x max SM clock",
                     "note": "ALU work = 0.375 lane-ops per performed sequence x conformation evaluation (8 three-input "
                             "packed maxes + 16 fused add+max per 2 conformations x 32 sequences per thread), counted from "
                             "the kernel source; odd chains evaluate one id of each reversal pair (50.8% of 2^27 for "
                             "3x3x3); achieved uses the map kernel's CUDA-event time inside the step"},
        "clocks": clocks,
    }
    if rank == 0:
        line["box_6x6"] = map_block_6x6(hp, torch, peak_ops)
        line["other_boxes"] = small_boxes_and_batch(hp, torch)
    if rank == 0 and not args.no_learned:
        line["learned"] = {}
        for name, fn in (("3x3x3", lambda: learned_leg(hp, s, torch)), ("6x6", lambda: learned_leg_6x6(hp, torch))):
            try:
                line["learned"][name] = fn()
            except Exception as exc:  # reported in the line, never hides the main measurement
                line["learned"][name] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(DIMS)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
