"""Pins of the GreBsmo oracle (Sec. 3.2.1, Algorithm 2, eqs. GreBsmoA, GreBsmoD, softt):
the soft threshold is the proximal map of lambda |.|, GreBsmo without a sparse part is
the truncated SVD, its objective never increases, and it finds the rank by itself."""
import numpy as np
import pytest

import oracle.grebsmo as GB


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_soft_threshold_is_the_prox_of_l1():
    g = np.random.default_rng(1)
    y = g.standard_normal(200) * 3.0
    lam = 0.7
    grid = np.linspace(-12.0, 12.0, 240001)                          # step 1e-4
    brute = np.array([grid[np.argmin(0.5 * (grid - v) ** 2 + lam * np.abs(grid))] for v in y])
    assert np.max(np.abs(GB.soft_threshold(y, lam) - brute)) <= 1e-4
    assert np.array_equal(GB.soft_threshold(np.array([0.5, -0.7, 0.71]), 0.7) != 0, [False, False, True])


def test_no_sparse_part_gives_the_truncated_svd():
    """With lambda above every |entry| S stays 0, the inner steps are a subspace iteration
    and each greedy increment adds the next singular directions: U V must equal the rank-r
    truncated SVD of X."""
    g = np.random.default_rng(2)
    Uf, _ = np.linalg.qr(g.standard_normal((60, 20)))
    Vf, _ = np.linalg.qr(g.standard_normal((45, 20)))
    lam_s = 10.0 * 0.6 ** np.arange(20)
    X = (Uf * lam_s) @ Vf.T
    res = GB.grebsmo(X, lam=1e12, dr=2, K=60, tau=0.0, r_max=6)
    assert res["r"] == 6 and not res["S"].any()
    best = (Uf[:, :6] * lam_s[:6]) @ Vf[:, :6].T
    assert _rel(res["U"] @ res["V"], best) <= 1e-10


def test_objective_never_increases():
    g = np.random.default_rng(3)
    m, n, r = 80, 60, 4
    L = g.standard_normal((m, r)) @ g.standard_normal((r, n))
    S = np.zeros(m * n)
    S[g.choice(m * n, 200, replace=False)] = g.uniform(-10, 10, 200)
    X = L + S.reshape(m, n) + 1e-2 * g.standard_normal((m, n))
    res = GB.grebsmo(X, lam=0.3, dr=1, K=6, tau=0.0, r_max=6, keep_history=True)
    h = np.array(res["history"])
    assert len(h) == 6 * 6
    assert np.all(np.diff(h) <= 1e-12 * h[:-1])


def test_rank_is_found_by_the_greedy_increments():
    """Low rank 3 plus large sparse entries (|S| in [20, 30]) plus small noise, lambda = 3
    (above the low-rank entries, below the sparse ones).  The residual of each rank stage
    falls until the third direction is in and then flattens at the shrinkage floor
    k lambda^2 / ||X||^2 (every entry S takes keeps lambda of its size); with tau at 1.5
    times that floor the loop stops at rank 3: the rank is estimated, not given.  L is
    recovered up to the l1 model's shrinkage bias."""
    g = np.random.default_rng(4)
    m, n, r, k, lam = 90, 70, 3, 150, 3.0
    L = g.standard_normal((m, r)) @ g.standard_normal((r, n))
    S = np.zeros(m * n)
    S[g.choice(m * n, k, replace=False)] = g.uniform(20, 30, k) * g.choice([-1, 1], k)
    X = L + S.reshape(m, n) + 1e-3 * g.standard_normal((m, n))
    floor = k * lam ** 2 / np.sum(X ** 2)
    res = GB.grebsmo(X, lam=lam, dr=1, K=30, tau=1.5 * floor, r_max=10)
    assert res["r"] == r
    assert all(e > 1.5 * floor for e in res["errors"][:-1]) and res["errors"][-1] <= 1.5 * floor
    assert _rel(res["U"] @ res["V"], L) <= 0.15


def _span_dist(A, B):
    """Sine of the largest principal angle between the row spaces of A and B."""
    Qa, _ = np.linalg.qr(A.T)
    Qb, _ = np.linalg.qr(B.T)
    return float(np.linalg.norm(Qa - Qb @ (Qb.T @ Qa), 2))


def test_random_projection_increment_converges_to_the_svd():
    """Reading R22 against the exact increment: on a matrix with a clear gap after the
    third singular value the randomized subspace iteration finds the same top right
    singular vectors (the subspace to 1e-10 after 6 power steps, each vector up to sign),
    and on a rank-3 matrix one power step is already exact (D^T D B spans its row space)."""
    g = np.random.default_rng(5)
    Uf, _ = np.linalg.qr(g.standard_normal((70, 40)))
    Vf, _ = np.linalg.qr(g.standard_normal((50, 40)))
    sv = np.concatenate([[30.0, 20.0, 10.0], 0.5 * 0.9 ** np.arange(37)])
    D = (Uf * sv) @ Vf.T
    omega = g.standard_normal((50, 8))
    exact = GB.top_right_singular_vectors(D, 3)
    rp = GB.rp_right_singular_vectors(D, 3, omega, 6)
    assert _span_dist(rp, exact) <= 1e-10
    assert np.allclose(np.abs(np.sum(rp * exact, axis=1)), 1.0, atol=1e-10)
    D3 = (Uf[:, :3] * sv[:3]) @ Vf[:, :3].T
    assert _span_dist(GB.rp_right_singular_vectors(D3, 3, omega, 1), Vf[:, :3].T) <= 1e-12


def test_grebsmo_with_random_projection_increments_matches_exact_increments():
    """The whole GreBsmo run with random-projection increments (R22, 4 power steps) equals
    the run with exact increments on the rank-finding case of the test above."""
    g = np.random.default_rng(4)
    m, n, r, k, lam = 90, 70, 3, 150, 3.0
    L = g.standard_normal((m, r)) @ g.standard_normal((r, n))
    S = np.zeros(m * n)
    S[g.choice(m * n, k, replace=False)] = g.uniform(20, 30, k) * g.choice([-1, 1], k)
    X = L + S.reshape(m, n) + 1e-3 * g.standard_normal((m, n))
    floor = k * lam ** 2 / np.sum(X ** 2)
    exact = GB.grebsmo(X, lam=lam, dr=1, K=30, tau=1.5 * floor, r_max=10)
    omegas = [g.standard_normal((n, 6)) for _ in range(10)]
    rp = GB.grebsmo(X, lam=lam, dr=1, K=30, tau=1.5 * floor, r_max=10, omegas=omegas, q_inc=4)
    assert rp["r"] == exact["r"] == r
    assert _rel(rp["U"] @ rp["V"], exact["U"] @ exact["V"]) <= 1e-8
    assert np.allclose(rp["S"], exact["S"], atol=1e-7)
