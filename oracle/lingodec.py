"""LinGoDec oracle in plain numpy float64 (test infrastructure only).

Linear functional GoDec (Sec. 4.3, eqs. LinGoDec and NLinGoDec): X (users x items) =
W Z^T + S + G with item features Z (items x d) given, W (users x d) of rank <= r and S
sparse, by alternating exact minimisation of
    1/2 ||X - W Z^T - S||_F^2 + lambda ||vec(S)||_1,   rank(W) <= r.

Readings (listed with the other readings of the paper):
R20 the W update of eq. NLinGoDec fits X - S_{k-1} (the printed update omits S, which
    the alternating minimisation it derives from needs).
R21 the rank-constrained least squares min ||Y - W Z^T|| over rank(W) <= r (the closed
    form the paper cites) is taken through the thin QR Z = Q R (Z of full column rank):
    ||Y - W Z^T||^2 = ||Y Q - W R^T||^2 + ||Y (I - Q Q^T)||^2, so W R^T is the rank-r
    truncated SVD of Y Q and W = P_r(Y Q) R^{-T}.
The S update is the soft threshold S_lambda of eq. softt, the exact minimiser over S.
"""
from __future__ import annotations

import numpy as np

from .grebsmo import soft_threshold


def reduced_rank_ls(Y: np.ndarray, Z: np.ndarray, r: int) -> np.ndarray:
    """argmin over rank(W) <= r of ||Y - W Z^T||_F (Reading R21)."""
    Q, R = np.linalg.qr(Z)
    Uy, s, Vty = np.linalg.svd(Y @ Q, full_matrices=False)
    M = (Uy[:, :r] * s[:r]) @ Vty[:r]                 # rank-r truncation of Y Q
    return np.linalg.solve(R, M.T).T                    # M R^{-T}


def objective(X, W, Z, S, lam: float) -> float:
    R = X - W @ Z.T - S
    return 0.5 * float(np.sum(R * R)) + lam * float(np.sum(np.abs(S)))


def lingodec(X, Z, r: int, lam: float, iters: int):
    """Alternating minimisation of eq. LinGoDec (eq. NLinGoDec with Reading R20).
    Returns W, S and the objective after every iteration."""
    X = np.asarray(X, dtype=np.float64)
    S = np.zeros_like(X)
    hist = []
    W = None
    for _ in range(iters):
        W = reduced_rank_ls(X - S, Z, r)                # Reading R20
        S = soft_threshold(X - W @ Z.T, lam)
        hist.append(objective(X, W, Z, S, lam))
    return {"W": W, "S": S, "history": hist}
