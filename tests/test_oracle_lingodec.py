"""Pins of the LinGoDec oracle (Sec. 4.3, eqs. LinGoDec, NLinGoDec): the rank-constrained
least squares is ordinary least squares at full rank and beats every rank-r competitor,
the objective never increases, and the paper's synthetic recipe (W a product of two
Gaussians, Gaussian features and noise, Bernoulli +-1 sparse part) is recovered."""
import numpy as np

import oracle.lingodec as LG


def test_full_rank_is_ordinary_least_squares():
    g = np.random.default_rng(1)
    Y, Z = g.standard_normal((40, 30)), g.standard_normal((30, 6))
    W = LG.reduced_rank_ls(Y, Z, 6)
    W_ols = np.linalg.lstsq(Z, Y.T, rcond=None)[0].T
    assert np.linalg.norm(W - W_ols) <= 1e-10 * np.linalg.norm(W_ols)


def test_rank_constrained_solution_beats_competitors():
    """The closed form against the brute-force alternative over rank-r W: random rank-r
    candidates, rank-r truncations of the ordinary least-squares W, and local rank-r
    perturbations of the solution itself never do better."""
    g = np.random.default_rng(2)
    Y, Z, r = g.standard_normal((30, 25)), g.standard_normal((25, 8)), 3
    W = LG.reduced_rank_ls(Y, Z, r)
    assert np.linalg.matrix_rank(W) == r
    f = lambda W_: np.linalg.norm(Y - W_ @ Z.T) ** 2
    best = f(W)
    W_ols = np.linalg.lstsq(Z, Y.T, rcond=None)[0].T
    U, s, Vt = np.linalg.svd(W_ols, full_matrices=False)
    assert best <= f((U[:, :r] * s[:r]) @ Vt[:r]) + 1e-9       # naive truncation is worse (Z not orthonormal)
    Uw, sw, Vtw = np.linalg.svd(W, full_matrices=False)
    for _ in range(200):
        A = Uw[:, :r] + 1e-3 * g.standard_normal((30, r))
        B = (sw[:r, None] * Vtw[:r]) + 1e-3 * g.standard_normal((r, 8))
        assert f(A @ B) >= best - 1e-9
        assert f(g.standard_normal((30, r)) @ g.standard_normal((r, 8))) >= best


def test_objective_never_increases():
    g = np.random.default_rng(3)
    m, n, d, r = 60, 80, 10, 3
    W = g.standard_normal((m, r)) @ g.standard_normal((r, d))
    Z = g.standard_normal((n, d))
    S = np.where(g.uniform(size=(m, n)) < 0.05, g.choice([-1.0, 1.0], size=(m, n)), 0.0)
    X = W @ Z.T + S + 0.05 * g.standard_normal((m, n))
    h = np.array(LG.lingodec(X, Z, r, lam=0.2, iters=15)["history"])
    assert np.all(np.diff(h) <= 1e-12 * h[:-1])


def test_paper_synthetic_recipe_is_recovered():
    g = np.random.default_rng(4)
    m, n, d, r = 120, 150, 12, 3
    W = g.standard_normal((m, r)) @ g.standard_normal((r, d))
    Z = g.standard_normal((n, d))
    S = np.where(g.uniform(size=(m, n)) < 0.05, g.choice([-1.0, 1.0], size=(m, n)), 0.0)
    X = W @ Z.T + S + 1e-3 * g.standard_normal((m, n))
    res = LG.lingodec(X, Z, r, lam=0.1, iters=40)
    eW = np.linalg.norm(res["W"] - W) / np.linalg.norm(W)
    supp = (np.abs(res["S"]) > 0) == (S != 0)
    assert eW <= 1e-2
    assert supp.mean() >= 0.99
