"""GreBsmo oracle in plain numpy float64 (test infrastructure only).

Greedy bilateral smoothing (Sec. 3.2.1, Algorithm 2 with the updates of eq. GreBsmoA):
L = U V with U orthonormal (m x r_i) and V (r_i x n), S from element-wise soft
thresholding (eq. softt).  Per inner step, with Z = X - S_{k-1}:
    U_k = Q from QR(Z V_{k-1}^T),   V_k = Q^T Z,   S_k = S_lambda(X - U_k V_k).
After K inner steps the rank grows by dr: the dr top right singular vectors of
the derivative X - U V - S (eq. GreBsmoD) are appended as rows of V.

Readings (marked "Reading Rn", listed with the other readings of the paper):
R17 the loop of Algorithm 2 runs while the residual error is ABOVE tau (the printed
    condition is reversed), and stops at r_max; the residual error is the squared
    relative error ||X - U V - S||_F^2 / ||X||_F^2 (the paper's error metric, Sec. 5).
R18 the initial V holds the dr top right singular vectors of X (the greedy direction
    from U = 0, S = 0: the derivative of eq. GreBsmoD is then X itself).
R19 the objective that S_lambda minimises exactly over S is
    1/2 ||X - U V - S||_F^2 + lambda ||vec(S)||_1 (eq. GreBsmo with its constant read so
    that the update of eq. GreBsmoA is its exact minimiser).
"""
from __future__ import annotations

import numpy as np


def soft_threshold(R: np.ndarray, lam: float) -> np.ndarray:
    """S_lambda (eq. softt): sgn(R_ij) max(|R_ij| - lambda, 0), element-wise."""
    return np.sign(R) * np.maximum(np.abs(R) - lam, 0.0)


def objective(X, U, V, S, lam: float) -> float:
    """Reading R19: 1/2 ||X - U V - S||_F^2 + lambda ||vec(S)||_1."""
    R = X - U @ V - S
    return 0.5 * float(np.sum(R * R)) + lam * float(np.sum(np.abs(S)))


def top_right_singular_vectors(D: np.ndarray, k: int) -> np.ndarray:
    """The k top right singular vectors of D as rows (k x n)."""
    _, _, Vt = np.linalg.svd(D, full_matrices=False)
    return Vt[:k]


def bilateral_step(X, V, S, lam: float):
    """One inner step of eq. GreBsmoA: (U_k, V_k, S_k) from (V_{k-1}, S_{k-1})."""
    Z = X - S
    Q, _ = np.linalg.qr(Z @ V.T)
    Vn = Q.T @ Z
    return Q, Vn, soft_threshold(X - Q @ Vn, lam)


def grebsmo(X, lam: float, dr: int, K: int, tau: float, r_max: int, keep_history: bool = False):
    """GreBsmo (Algorithm 2 with eq. GreBsmoA and eq. GreBsmoD).

    Returns a dict with U (m x r), V (r x n), S, the rank r, the residual error after each
    rank stage and, with keep_history, the objective (R19) after every inner step.
    """
    X = np.asarray(X, dtype=np.float64)
    normX2 = float(np.sum(X * X))
    S = np.zeros_like(X)
    V = top_right_singular_vectors(X, dr)                  # Reading R18
    U = np.zeros((X.shape[0], V.shape[0]))
    history, errors = [], []
    while True:
        for _ in range(K):
            U, V, S = bilateral_step(X, V, S, lam)
            if keep_history:
                history.append(objective(X, U, V, S, lam))
        D = X - U @ V - S
        err = float(np.sum(D * D)) / normX2
        errors.append(err)
        if err <= tau or V.shape[0] >= r_max:               # Reading R17
            break
        add = min(dr, r_max - V.shape[0])
        V = np.vstack([V, top_right_singular_vectors(D, add)])
    return {"U": U, "V": V, "S": S, "r": V.shape[0], "errors": errors, "history": history}
