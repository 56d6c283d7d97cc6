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
R22 the random-projection variant of the increment (the paper allows the row space of
    the top singular vectors of eq. GreBsmoD to be approximated by random projections)
    is read as a randomized subspace iteration: B = orth(Omega) for a given n x p test
    matrix Omega (p >= dr), q times B = orth(D^T orth(D B)), then the dr top right
    singular vectors of D B, mapped back by B (a Rayleigh-Ritz step).  With enough power
    steps it converges to the exact increment.
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


def rp_right_singular_vectors(D: np.ndarray, k: int, omega: np.ndarray, q: int) -> np.ndarray:
    """Reading R22: the k top right singular vectors of D (as rows, k x n) from the
    randomized subspace iteration started at omega (n x p, p >= k) with q power steps."""
    B, _ = np.linalg.qr(omega)
    for _ in range(q):
        Y, _ = np.linalg.qr(D @ B)
        B, _ = np.linalg.qr(D.T @ Y)
    _, _, Vyt = np.linalg.svd(D @ B, full_matrices=False)
    return (B @ Vyt[:k].T).T


def bilateral_step(X, V, S, lam: float):
    """One inner step of eq. GreBsmoA: (U_k, V_k, S_k) from (V_{k-1}, S_{k-1})."""
    Z = X - S
    Q, _ = np.linalg.qr(Z @ V.T)
    Vn = Q.T @ Z
    return Q, Vn, soft_threshold(X - Q @ Vn, lam)


def grebsmo(X, lam: float, dr: int, K: int, tau: float, r_max: int, keep_history: bool = False,
            omegas=None, q_inc: int = 0):
    """GreBsmo (Algorithm 2 with eq. GreBsmoA and eq. GreBsmoD).

    Returns a dict with U (m x r), V (r x n), S, the rank r, the residual error after each
    rank stage and, with keep_history, the objective (R19) after every inner step.
    With omegas (a list of n x p test matrices, one per increment, the first for the
    initial V), the increments use the random-projection variant (R22) with q_inc power
    steps instead of an exact SVD.
    """
    X = np.asarray(X, dtype=np.float64)
    normX2 = float(np.sum(X * X))
    S = np.zeros_like(X)

    def increment(D, k, stage):
        if omegas is None:
            return top_right_singular_vectors(D, k)
        return rp_right_singular_vectors(D, k, np.asarray(omegas[stage], dtype=np.float64), q_inc)

    stage = 0
    V = increment(X, dr, stage)                            # Reading R18
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
        stage += 1
        V = np.vstack([V, increment(D, add, stage)])
    return {"U": U, "V": V, "S": S, "r": V.shape[0], "errors": errors, "history": history}
