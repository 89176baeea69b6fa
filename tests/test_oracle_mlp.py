"""Pin for the fp64 proposal-network reference: analytic gradients vs central differences."""
import numpy as np

from oracle import mlp
from paper_2008_05612_gb300 import inputs


def test_gradients_match_finite_differences():
    N, H1, H2, S, B = 9, 7, 6, 5, 11
    params = [
        inputs.init_weights((H1, N), N, 1), inputs.init_weights((H1,), N, 2),
        inputs.init_weights((H2, H1), H1, 3), inputs.init_weights((H2,), H1, 4),
        inputs.init_weights((S, H2), H2, 5), inputs.init_weights((S,), H2, 6),
    ]
    ids = inputs.sample_ids(N, B, seed=9)
    x = mlp.bits(ids, N)
    labels = (ids % np.uint64(S)).astype(np.int64)
    _, grads = mlp.loss_and_grads(params, x, labels)
    eps = 1e-6
    for p, g in zip(params, grads):
        flat = p.reshape(-1)
        gf = g.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 12)):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = mlp.loss_and_grads(params, x, labels)
            flat[idx] = old - eps
            lm, _ = mlp.loss_and_grads(params, x, labels)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - gf[idx]) < 1e-7 + 1e-5 * abs(fd)


def test_loss_of_uniform_logits_is_log_S():
    N, S = 4, 7
    params = [np.zeros((3, N)), np.zeros(3), np.zeros((3, 3)), np.zeros(3), np.zeros((S, 3)), np.zeros(S)]
    x = mlp.bits(np.arange(5, dtype=np.uint64), N)
    loss, _ = mlp.loss_and_grads(params, x, np.arange(5) % S)
    assert abs(loss - np.log(S)) < 1e-12
