"""MSE training oracle in plain numpy float64 (test infrastructure only).

Multi-label subspace ensemble, training stage (Sec. 4.2.1, eqs. ms, mssub, mssolution,
msinitial, Algorithm 4): X (samples x features) = sum_i L^i + S, where L^i is nonzero
only on the rows Omega_i of the samples carrying label i, rank(L^i_{Omega_i}) <= r^i,
and card(S) <= K.  Block coordinate descent over L^1 .. L^k and S, each block solved
globally: L^i_{Omega_i} is the rank-r^i truncation of the residual on Omega_i (exact SVD,
eq. mssolution, or the q = 0 bilateral random projection of Algorithm 4), S the K
largest entries of the residual (the hard threshold of Algorithm 1's S-step).  The
output subspaces are C^i = (Q^i)^T from the QR of (L^i_{Omega_i})^T.
"""
from __future__ import annotations

import numpy as np

from .godec import hard_threshold


def truncated(N: np.ndarray, r: int) -> np.ndarray:
    """Rank-r truncated SVD of N (eq. mssolution)."""
    U, s, Vt = np.linalg.svd(N, full_matrices=False)
    return (U[:, :r] * s[:r]) @ Vt[:r]


def brp_q0(N: np.ndarray, A1: np.ndarray) -> np.ndarray:
    """The q = 0 bilateral random projection of Algorithm 4: Y1 = N A1, A2 = Y1,
    Y2 = N^T Y1, Y1 = N Y2, L = Y1 (A2^T Y1)^{-1} Y2^T."""
    Y1 = N @ A1
    A2 = Y1
    Y2 = N.T @ Y1
    Y1 = N @ Y2
    return Y1 @ np.linalg.solve(A2.T @ Y1, Y2.T)


def objective(X, Ls, S) -> float:
    R = X - sum(Ls) - S
    return float(np.sum(R * R))


def mse_train(X, labels, ranks, K: int, iters: int, brp_rng=None):
    """Algorithm 4 with a fixed number of outer iterations.

    labels: n x k 0/1 matrix Y; ranks: r^i per label; brp_rng: a numpy Generator to
    draw the Gaussian A1 of each BRP step (None: exact truncated SVD instead).
    Returns the L^i, S, the subspaces C^i and the objective after every outer iteration.
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(labels)
    n, k = Y.shape
    Omega = [np.flatnonzero(Y[:, i]) for i in range(k)]
    D = Y.sum(axis=1).astype(np.float64)
    Z = X / np.where(D > 0, D, 1.0)[:, None]                 # eq. msinitial: Z = D^{-1} X
    Ls = []
    for i in range(k):
        L = np.zeros_like(X)
        L[Omega[i]] = Z[Omega[i]]
        Ls.append(L)
    S = np.zeros_like(X)
    hist = []
    for _ in range(iters):
        for i in range(k):
            N = (X - sum(Ls[j] for j in range(k) if j != i) - S)[Omega[i]]
            if brp_rng is None:
                Li = truncated(N, ranks[i])
            else:
                Li = brp_q0(N, brp_rng.standard_normal((X.shape[1], ranks[i])))
            Ls[i] = np.zeros_like(X)
            Ls[i][Omega[i]] = Li
        idx, val = hard_threshold(X - sum(Ls), K)
        S = np.zeros(X.size)
        S[idx] = val
        S = S.reshape(X.shape)
        hist.append(objective(X, Ls, S))
    Cs = []
    for i in range(k):
        Q, _ = np.linalg.qr(Ls[i][Omega[i]].T)
        Cs.append(Q[:, :ranks[i]].T)
    return {"L": Ls, "S": S, "C": Cs, "history": hist}
