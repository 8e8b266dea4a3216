"""Pin of the FP64 reference network against central finite differences."""
import numpy as np
import pytest

from oracle import mlp as M


@pytest.mark.parametrize("with_c", [False, True])
def test_backprop_matches_finite_differences(with_c):
    rng = np.random.default_rng(3)
    n_out, nA, nB = (48, 20, 8) if with_c else (32, 20, 8)
    nC, S = (18, 3) if with_c else (0, 0)
    tC = np.array([4, 17, 0, 2, -1, 9]) if with_c else None
    n = sum(o * i + o for o, i in M.shapes(n_out))
    flat = rng.normal(0, 0.3, n)
    X = rng.normal(0, 1, (6, M.N_IN))
    tA = np.array([3, 0, 19, -1, 7, 11])
    tB = np.array([1, 7, 0, 2, 5, 3])
    loss, g = M.loss_and_grad(flat, n_out, nA, nB, X, tA, tB, nC, S, tC)
    idx = rng.choice(n, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(n)
        e[i] = h
        lp, _ = M.loss_and_grad(flat + e, n_out, nA, nB, X, tA, tB, nC, S, tC)
        lm, _ = M.loss_and_grad(flat - e, n_out, nA, nB, X, tA, tB, nC, S, tC)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    # the ignored row contributes no gradient and no loss
    keep = [0, 1, 2, 4, 5]
    l2, g2 = M.loss_and_grad(flat, n_out, nA, nB, X[keep], tA[keep], tB[keep], nC, S,
                             None if tC is None else tC[keep])
    assert np.isclose(l2 * 5, loss * 6) and np.allclose(g2 * 5, g * 6)
    if with_c:
        # head C only sees the target's slice: logits of the other slices get no gradient
        W4g = g[-(n_out * M.N_HID + n_out):-n_out].reshape(n_out, M.N_HID)
        b4g = g[-n_out:]
        used = set()
        for r in range(6):
            if tA[r] >= 0 and tC[r] >= 0:
                used.update(range(nA + nB + (tC[r] // S) * S, nA + nB + (tC[r] // S + 1) * S))
        for k in range(nA + nB, n_out):
            if k not in used:
                assert b4g[k] == 0.0 and not W4g[k].any()

