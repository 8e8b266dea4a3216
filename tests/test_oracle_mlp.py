"""Pin of the FP64 reference network against central finite differences."""
import numpy as np

from oracle import mlp as M


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(3)
    n_out, nA, nB = 32, 20, 8
    n = sum(o * i + o for o, i in M.shapes(n_out))
    flat = rng.normal(0, 0.3, n)
    X = rng.normal(0, 1, (6, M.N_IN))
    tA = np.array([3, 0, 19, -1, 7, 11])
    tB = np.array([1, 7, 0, 2, 5, 3])
    loss, g = M.loss_and_grad(flat, n_out, nA, nB, X, tA, tB)
    idx = rng.choice(n, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(n)
        e[i] = h
        lp, _ = M.loss_and_grad(flat + e, n_out, nA, nB, X, tA, tB)
        lm, _ = M.loss_and_grad(flat - e, n_out, nA, nB, X, tA, tB)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    # the ignored row contributes no gradient and no loss
    l2, g2 = M.loss_and_grad(flat, n_out, nA, nB, X[[0, 1, 2, 4, 5]], tA[[0, 1, 2, 4, 5]], tB[[0, 1, 2, 4, 5]])
    assert np.isclose(l2 * 5, loss * 6) and np.allclose(g2 * 5, g * 6)
