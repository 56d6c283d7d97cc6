"""Pins of the MSE training oracle (Sec. 4.2.1, Algorithm 4): the blocks stay on their
label rows, exact block minimisation never increases the objective, the q = 0 BRP step
equals the truncated SVD on an exactly low-rank block, and on synthetic multi-label data
each learned subspace is the row space that generated its label's component."""
import numpy as np

import oracle.mse as MS


def _synthetic(seed, n=300, p=40, k=4, r=2, K=150, noise=1e-3):
    g = np.random.default_rng(seed)
    Y = (g.uniform(size=(n, k)) < 0.35).astype(int)
    Y[Y.sum(axis=1) == 0, 0] = 1                                   # every sample has a label
    bases = [np.linalg.qr(g.standard_normal((p, r)))[0].T for _ in range(k)]   # r x p row spaces
    X = np.zeros((n, p))
    for i in range(k):
        rows = np.flatnonzero(Y[:, i])
        X[rows] += g.standard_normal((rows.size, r)) @ bases[i] * 3.0
    S = np.zeros(n * p)
    S[g.choice(n * p, K, replace=False)] = g.uniform(5, 10, K) * g.choice([-1, 1], K)
    X += S.reshape(n, p) + noise * g.standard_normal((n, p))
    return X, Y, bases


def test_blocks_live_on_their_label_rows():
    X, Y, _ = _synthetic(1)
    res = MS.mse_train(X, Y, [2] * 4, 150, 3)
    for i, L in enumerate(res["L"]):
        assert not L[Y[:, i] == 0].any()


def test_exact_blocks_never_increase_the_objective():
    X, Y, _ = _synthetic(2)
    h = np.array(MS.mse_train(X, Y, [2] * 4, 150, 12)["history"])
    assert np.all(np.diff(h) <= 1e-10 * h[:-1])


def test_brp_step_is_the_truncated_svd_on_an_exact_low_rank_block():
    g = np.random.default_rng(3)
    N = g.standard_normal((50, 3)) @ g.standard_normal((3, 30))
    L = MS.brp_q0(N, g.standard_normal((30, 3)))
    assert np.linalg.norm(L - MS.truncated(N, 3)) <= 1e-10 * np.linalg.norm(N)


def test_learned_subspaces_match_the_generating_row_spaces():
    X, Y, bases = _synthetic(4)
    for rng in (None, np.random.default_rng(5)):                 # exact SVD and Algorithm 4's BRP
        res = MS.mse_train(X, Y, [2] * 4, 150, 30, brp_rng=rng)
        for C, B in zip(res["C"], bases):
            # sines of the principal angles between the learned and the true row spaces
            s = np.linalg.svd(C @ B.T, compute_uv=False)
            assert np.sqrt(max(0.0, 1.0 - s.min() ** 2)) <= 1e-2
