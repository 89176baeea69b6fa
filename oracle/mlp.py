"""fp64 reference of the proposal network (TEST INFRASTRUCTURE ONLY).

The paper has no learned component; this is the plain definition of the
network the library trains on its own phenotype maps:
    x = bits of the sequence id (1 = H), length N, as 0/1 floats
    z1 = x W1^T + b1,  a1 = relu(z1)          (N -> H1)
    z2 = a1 W2^T + b2, a2 = relu(z2)          (H1 -> H2)
    z3 = a2 W3^T + b3                         (H2 -> S logits)
    loss = mean over the batch of  logsumexp(z3) - z3[label]
Gradients are the textbook chain rule.  Pinned by central finite differences
in tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np


def bits(ids: np.ndarray, N: int) -> np.ndarray:
    ids = np.asarray(ids, dtype=np.uint64)
    return ((ids[:, None] >> np.arange(N, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.float64)


def forward(params, x):
    W1, b1, W2, b2, W3, b3 = params
    z1 = x @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    z3 = a2 @ W3.T + b3
    return z1, a1, z2, a2, z3


def loss_and_grads(params, x, labels):
    W1, b1, W2, b2, W3, b3 = params
    z1, a1, z2, a2, z3 = forward(params, x)
    B = x.shape[0]
    m = z3.max(axis=1, keepdims=True)
    e = np.exp(z3 - m)
    lse = np.log(e.sum(axis=1, keepdims=True)) + m
    loss = float(np.mean(lse[:, 0] - z3[np.arange(B), labels]))
    d3 = e / e.sum(axis=1, keepdims=True)
    d3[np.arange(B), labels] -= 1.0
    d3 /= B
    gW3 = d3.T @ a2
    gb3 = d3.sum(0)
    d2 = (d3 @ W3) * (z2 > 0)
    gW2 = d2.T @ a1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (z1 > 0)
    gW1 = d1.T @ x
    gb1 = d1.sum(0)
    return loss, (gW1, gb1, gW2, gb2, gW3, gb3)


def topk(params, x, k):
    """Indices of the k largest logits per row (ties broken toward the lower index)."""
    z3 = forward(params, x)[4]
    order = np.argsort(-z3, axis=1, kind="stable")
    return order[:, :k]
