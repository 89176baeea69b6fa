"""Independent brute force for tiny boxes (pins for the oracle).

Written separately from oracle/hp_oracle.c: paths come from a Python DFS over
coordinate tuples, the box group from signed permutation matrices, energies
from a coordinate pair scan with the Table 1 values x 10.  Only usable for a
handful of sites.
"""
from __future__ import annotations

import itertools

import numpy as np

E10 = {(0, 0): 0, (0, 1): -10, (1, 0): -10, (1, 1): -23}


def sites(dims):
    dims = tuple(dims) + (1,) * (3 - len(dims))
    return [(x, y, z) for z in range(dims[2]) for y in range(dims[1]) for x in range(dims[0])]


def site_id(c, dims):
    dims = tuple(dims) + (1,) * (3 - len(dims))
    return c[0] + dims[0] * (c[1] + dims[1] * c[2])


def hamiltonian_paths(dims):
    """All directed Hamiltonian paths as tuples of coordinates."""
    pts = sites(dims)
    pset = set(pts)
    out = []

    def nbrs(c):
        for k in range(3):
            for d in (-1, 1):
                n = list(c)
                n[k] += d
                n = tuple(n)
                if n in pset:
                    yield n

    def rec(path, seen):
        if len(path) == len(pts):
            out.append(tuple(path))
            return
        for n in nbrs(path[-1]):
            if n not in seen:
                seen.add(n)
                path.append(n)
                rec(path, seen)
                path.pop()
                seen.remove(n)

    for p in pts:
        rec([p], {p})
    return out


def group(dims):
    """Signed axis permutations mapping the box onto itself, as functions on coordinates."""
    full = tuple(dims) + (1,) * (3 - len(dims))
    nd = len(dims)
    ops = []
    for perm in itertools.permutations(range(nd)):
        if any(full[perm[k]] != full[k] for k in range(nd)):
            continue
        for signs in itertools.product((0, 1), repeat=nd):
            def f(c, perm=perm, signs=signs):
                out = list(c)
                for k in range(nd):
                    v = c[perm[k]]
                    out[k] = full[k] - 1 - v if signs[k] else v
                return tuple(out)
            ops.append(f)
    return ops


def library(dims):
    """(conformations as site-id tuples in canonical order, class of each, number of classes)."""
    paths = hamiltonian_paths(dims)
    G = group(dims)
    confs = set()
    for p in paths:
        imgs = [tuple(site_id(g(c), dims) for c in p) for g in G]
        confs.add(min(imgs))
    reps = {}
    for c in confs:
        coords = [sites(dims)[s] for s in c]
        rev = coords[::-1]
        imgs = [tuple(site_id(g(x), dims) for x in rev) for g in G]
        other = min(imgs)
        reps[c] = min(c, other)
    order = sorted(confs, key=lambda c: (reps[c], c))
    rep_list = sorted(set(reps.values()))
    cls = [rep_list.index(reps[c]) for c in order]
    return order, cls, len(rep_list)


def energy(conf, g, dims):
    pts = sites(dims)
    e = 0
    n = len(conf)
    for i in range(n):
        for j in range(i + 2, n):
            a, b = pts[conf[i]], pts[conf[j]]
            if sum(abs(a[k] - b[k]) for k in range(3)) == 1:
                e += E10[((g >> i) & 1, (g >> j) & 1)]
    return e


def phenotype_map(dims):
    """Reading B by brute force: every conformation competes; strict unique minimum."""
    order, cls, S = library(dims)
    N = len(order[0])
    out = np.empty(1 << N, dtype=np.int32)
    for g in range(1 << N):
        es = [energy(c, g, dims) for c in order]
        m = min(es)
        idx = [k for k, e in enumerate(es) if e == m]
        out[g] = cls[idx[0]] if len(idx) == 1 else -1
    return out, S


def gap_map(dims):
    """Per genotype: class of the lowest-index minimiser and E2 - E1 (second-lowest energy counted
    with multiplicity minus the lowest; None for a single conformation)."""
    order, cls, S = library(dims)
    N = len(order[0])
    first, gaps = [], []
    for g in range(1 << N):
        es = [energy(c, g, dims) for c in order]
        m = min(es)
        first.append(cls[es.index(m)])
        srt = sorted(es)
        gaps.append(srt[1] - srt[0] if len(srt) > 1 else None)
    return first, gaps, S
