"""GoDec-BRP oracle in plain numpy float64 (test infrastructure only).

Readings of places where the paper is silent or ambiguous are marked
``Reading Rn`` and listed in the design notes of the repository.

Notation (Sec. 3.1, Algorithm 1): Z = X - S_{t-1};  L~ = (Z Z^T)^q Z;
Y1 = L~ A1, A2 = Y1;  Y2 = L~^T Y1 = Q2 R2;  Y1 = L~ Y2 = Q1 R1;
L_t = Q1 [R1 (A2^T Y1)^{-1} R2^T]^{1/(2q+1)} Q2^T;  S_t = P_Omega(X - L_t).
"""
from __future__ import annotations

import numpy as np

# Reading R6: relative tolerance of the numerical rank test of Algorithm 1.
RANK_TOL = 1e-4


# ----------------------------------------------------------------------------
# L-step (Sec. 3.1.1-3.1.3, eqs. lr_app / mlr_app, Algorithm 1)
# ----------------------------------------------------------------------------
def ltilde_times(Z: np.ndarray, B: np.ndarray, q: int) -> np.ndarray:
    """L~ B = (Z Z^T)^q Z B, evaluated right to left (Algorithm 1, the product L~ A1)."""
    Y = Z @ B
    for _ in range(q):
        Y = Z @ (Z.T @ Y)
    return Y


def ltilde_t_times(Z: np.ndarray, B: np.ndarray, q: int) -> np.ndarray:
    """L~^T B = Z^T (Z Z^T)^q B (Algorithm 1, the product L~^T Y1)."""
    Y = B
    for _ in range(q):
        Y = Z @ (Z.T @ Y)
    return Z.T @ Y


def numerical_rank(Z: np.ndarray, Q2: np.ndarray, tol: float = RANK_TOL) -> int:
    """Numerical rank used by the test 'rank(A2^T Y1) < r' (Algorithm 1's rank test).

    Reading R6: A2^T Y1 = Y2^T Y2 (since Y1 = L~ Y2 and A2 = Y1^0 = L~ A1), so
    its rank is rank(Y2) = rank(Z Q2) with Q2 an orthonormal basis of
    range(Y2).  The rank is the number of singular values of Z Q2 above
    ``tol`` times the largest one; Z Q2 carries Z's singular values on the
    sampled subspace, unlike A2^T Y1 whose spread is their (8q+4)-th power.
    """
    s = np.linalg.svd(Z @ Q2, compute_uv=False)
    if s.size == 0 or not s[0] > 0.0:
        return 0
    return int(np.sum(s > tol * s[0]))


def _root_factors(Q1, M, Q2, q):
    """L = Q1 M^{1/(2q+1)} Q2^T as factors U diag(sigma) V^T (eq. mlr_app).

    Reading R4: the fractional power of the non-symmetric r x r matrix M is
    taken on its singular values, M = Um Sm Vm^T -> Um Sm^{1/(2q+1)} Vm^T
    (the paper states that the step needs 'an SVD of an r x r matrix').
    """
    Um, s, Vmt = np.linalg.svd(M)
    sigma = s ** (1.0 / (2 * q + 1))
    return Q1 @ Um, sigma, Q2 @ Vmt.T


def _empty_factors(m, n):
    return np.zeros((m, 0)), np.zeros(0), np.zeros((n, 0))


def brp_literal(Z: np.ndarray, A1: np.ndarray, q: int, rank_tol: float = RANK_TOL):
    """One L-step exactly as Algorithm 1 prints it (no rescaling).

    Valid only while the unnormalised products stay well inside float64
    range and resolution (small, well-conditioned inputs); ``brp_stable``
    is the same map with orthonormalisation between products.
    Returns (U_L, sigma_L, V_L, r_eff).
    """
    m, n = Z.shape
    r = A1.shape[1]
    while True:
        if r == 0:
            return (*_empty_factors(m, n), 0)
        A = A1[:, :r]
        Y1 = ltilde_times(Z, A, q)          # Y1 = L~ A1
        A2 = Y1                             # A2 = Y1
        Y2 = ltilde_t_times(Z, Y1, q)       # Y2 = L~^T Y1 = Q2 R2
        Q2, R2 = np.linalg.qr(Y2)
        Y1 = ltilde_times(Z, Y2, q)         # Y1 = L~ Y2 = Q1 R1
        Q1, R1 = np.linalg.qr(Y1)
        r_new = numerical_rank(Z, Q2, rank_tol)
        if r_new < r:                       # r := rank(A2^T Y1); go to the first step
            r = r_new
            continue
        C = A2.T @ Y1
        # q = 0: L = Y1 C^{-1} Y2^T = Q1 [R1 C^{-1} R2^T] Q2^T (eq. lr_app), root 1.
        M = R1 @ np.linalg.solve(C, R2.T)
        U, s, V = _root_factors(Q1, M, Q2, q)
        return U, s, V, r


def brp_stable(Z: np.ndarray, A1: np.ndarray, q: int, rank_tol: float = RANK_TOL):
    """The same L-step with a Householder QR after every product.

    Algorithm 1 applies 6q+3 alternating factors Z, Z^T, Z, ... to A1:
    2q+1 for Y1 = L~ A1, 2q+1 for Y2 = L~^T Y1, 2q+1 for Y1 = L~ Y2.  Only
    range(Y2) enters L, and right-multiplying by an invertible r x r matrix
    keeps every range, so each product may be re-orthonormalised.  With
    Q2 = orth(Y2) the last chain gives L~ Q2 = Q1 (R_{2q} ... R_0), and since
    A2^T Y1 = R2^T R2 the core R1 (A2^T Y1)^{-1} R2^T equals that product M.
    Returns (U_L, sigma_L, V_L, r_eff).
    """
    m, n = Z.shape
    r = A1.shape[1]
    while True:
        if r == 0:
            return (*_empty_factors(m, n), 0)
        B = A1[:, :r]
        for i in range(4 * q + 2):          # L~ A1 then L~^T Y1: Z, Z^T, Z, ...
            B, _ = np.linalg.qr(Z @ B if i % 2 == 0 else Z.T @ B)
        Q2 = B
        P = Z @ Q2                          # first factor of L~ Q2
        r_new = numerical_rank(Z, Q2, rank_tol)
        if r_new < r:
            r = r_new
            continue
        Q, M = np.linalg.qr(P)
        for i in range(1, 2 * q + 1):
            Q, R = np.linalg.qr(Z.T @ Q if i % 2 == 1 else Z @ Q)
            M = R @ M
        U, s, V = _root_factors(Q, M, Q2, q)
        return U, s, V, r


def dense_L(U, sigma, V):
    return (U * sigma) @ V.T


# ----------------------------------------------------------------------------
# S-step (eq. raw_lss, Algorithm 1)
# ----------------------------------------------------------------------------
def hard_threshold(R: np.ndarray, k: int):
    """Omega = the nonzero subset of the k largest entries of |R|.

    Reading R7: equal magnitudes are ordered by ascending linear index
    i*n + j (row-major), and exact zeros are never selected, so
    |Omega| = min(k, number of nonzeros).  Returns (idx ascending, R[idx]).
    """
    a = np.abs(R).ravel()
    N = a.size
    k = min(int(k), N)
    if k <= 0:
        return np.zeros(0, dtype=np.int64), np.zeros(0)
    tau = np.partition(a, N - k)[N - k]              # k-th largest magnitude
    gt = np.flatnonzero(a > tau)
    eq = np.flatnonzero(a == tau)                    # ascending linear index
    idx = np.concatenate([gt, eq[: k - gt.size]])
    idx = idx[a[idx] != 0.0]
    idx.sort()
    return idx.astype(np.int64), R.ravel()[idx]


# ----------------------------------------------------------------------------
# GoDec loop (Algorithm 1) and naive GoDec (eq. raw_lss)
# ----------------------------------------------------------------------------
def _brp(variant):
    return {"stable": brp_stable, "literal": brp_literal}[variant]


def godec_step(X, A1, S_idx, S_val, k, q, variant="stable", rank_tol=RANK_TOL):
    """One iteration t of Algorithm 1 from S_{t-1} = (S_idx, S_val).

    Returns a dict with the L_t factors, S_t, r_eff and the two objective
    values of Appendix I: E1 = ||X - L_t - S_{t-1}||^2, E2 = ||X - L_t - S_t||^2.
    """
    X = np.asarray(X, dtype=np.float64)
    Z = X.copy()
    Z.ravel()[S_idx] -= S_val                        # Z = X - S_{t-1}
    U, s, V, r = _brp(variant)(Z, np.asarray(A1, dtype=np.float64), q, rank_tol)
    R = X - dense_L(U, s, V)                         # X - L_t
    D = R.copy()
    D.ravel()[S_idx] -= S_val
    E1 = float(np.sum(D * D))
    idx, val = hard_threshold(R, k)
    keep = np.ones(R.size, dtype=bool)
    keep[idx] = False
    E2 = float(np.sum(R.ravel()[keep] ** 2))         # sum over the complement of Omega
    return {"U": U, "sigma": s, "V": V, "r": r, "S_idx": idx, "S_val": val, "E1": E1, "E2": E2}


def godec(X, A1, k, q, tol=1e-7, max_iter=50, variant="stable", rank_tol=RANK_TOL,
          keep_history=False):
    """GoDec by BRP (Algorithm 1).

    Reading R1: L_0 := X, S_0 := 0 makes the loop test false only by
    accident, so the loop is a do-while: run at least one iteration and
    test ||X - L_t - S_t||_F^2 / ||X||_F^2 <= tol after each one.
    Reading R2: A1 (n x r) is drawn once by the caller and kept fixed.
    Reading R6: a rank drop keeps the first r_eff columns of A1 for the
    rest of the run.
    """
    X = np.asarray(X, dtype=np.float64)
    A = np.asarray(A1, dtype=np.float64)
    normX2 = float(np.sum(X * X))
    S_idx, S_val = np.zeros(0, dtype=np.int64), np.zeros(0)
    rel, E1s, E2s, hist = [], [], [], []
    t = 0
    while True:
        t += 1
        st = godec_step(X, A, S_idx, S_val, k, q, variant, rank_tol)
        A = A[:, :st["r"]]
        S_idx, S_val = st["S_idx"], st["S_val"]
        E1s.append(st["E1"])
        E2s.append(st["E2"])
        rel.append(st["E2"] / normX2 if normX2 > 0 else 0.0)
        if keep_history:
            hist.append(st)
        if rel[-1] <= tol or t >= max_iter:
            break
    st.update(iters=t, rel_err=rel, E1_hist=E1s, E2_hist=E2s, normX2=normX2, history=hist)
    return st


def naive_godec(X, r, k, tol=1e-7, max_iter=50):
    """Naive GoDec (eq. raw_lss): the L-step is the rank-r truncated SVD of X - S."""
    X = np.asarray(X, dtype=np.float64)
    normX2 = float(np.sum(X * X))
    S_idx, S_val = np.zeros(0, dtype=np.int64), np.zeros(0)
    E1s, E2s = [], []
    for _ in range(max_iter):
        Z = X.copy()
        Z.ravel()[S_idx] -= S_val
        Uf, s, Vt = np.linalg.svd(Z, full_matrices=False)
        L = (Uf[:, :r] * s[:r]) @ Vt[:r]
        R = X - L
        D = R.copy()
        D.ravel()[S_idx] -= S_val
        E1s.append(float(np.sum(D * D)))
        S_idx, S_val = hard_threshold(R, k)
        keep = np.ones(R.size, dtype=bool)
        keep[S_idx] = False
        E2s.append(float(np.sum(R.ravel()[keep] ** 2)))
        if E2s[-1] / normX2 <= tol:
            break
    return {"L": L, "S_idx": S_idx, "S_val": S_val, "E1_hist": E1s, "E2_hist": E2s}


# ----------------------------------------------------------------------------
# Precision form: one full-precision tangent-space correction (reading R11)
# ----------------------------------------------------------------------------
def tangent_refine(Z, U, V, r=None):
    """Re-truncate P_U Z + Z P_V - P_U Z P_V to rank r (U, V orthonormal).

    A = Z V and B = Z^T U come from one full-precision visit of Z.  With
    C = U^T A the correction is [U, A] K [V, B]^T, K = [[-C, I], [I, 0]];
    QR of both bases and an SVD of the 2r x 2r core give the rank-r part.
    Returns (U', sigma', V').
    """
    r = U.shape[1] if r is None else r
    A = Z @ V
    B = Z.T @ U
    C = U.T @ A
    Qa, Ra = np.linalg.qr(np.hstack([U, A]))
    Qb, Rb = np.linalg.qr(np.hstack([V, B]))
    I = np.eye(U.shape[1])
    K = np.block([[-C, I], [I, np.zeros_like(I)]])
    Uc, s, Vct = np.linalg.svd(Ra @ K @ Rb.T)
    return Qa @ Uc[:, :r], s[:r], Qb @ Vct[:r].T


# ----------------------------------------------------------------------------
# Differentiated form: T unrolled iterations at q = 0 with frozen masks (R14)
# ----------------------------------------------------------------------------
def _lstep_q0(Z, A1):
    """q = 0 L-step: L = Y1 (A2^T Y1)^{-1} Y2^T = Z P with P the projector on range(Y2)."""
    Y2 = Z.T @ (Z @ A1)                              # Y2 = Z^T A2, A2 = Z A1
    G = Y2.T @ Y2                                    # = A2^T Y1
    Y2p_T = np.linalg.solve(G, Y2.T).T               # (Y2^+)^T = Y2 (Y2^T Y2)^{-1}
    P = Y2p_T @ Y2.T
    return Z @ P, P, Y2, Y2p_T


def unrolled_forward(X, A1, k, T, masks=None):
    """T iterations of GoDec-BRP at q = 0.  Reading R14: the masks M_t (the
    supports Omega_t) are frozen, so S_t = M_t * (X - L_t) and
    Z_{t+1} = (1 - M_t) * X + M_t * L_t.  Returns (L_T, masks, tape)."""
    X = np.asarray(X, dtype=np.float64)
    A1 = np.asarray(A1, dtype=np.float64)
    Z = X.copy()
    tape, out_masks = [], []
    for t in range(T):
        L, P, Y2, Y2p_T = _lstep_q0(Z, A1)
        R = X - L
        if masks is None:
            idx, _ = hard_threshold(R, k)
        else:
            idx = masks[t]
        out_masks.append(idx)
        tape.append((Z, P, Y2p_T))
        Z = X.copy()
        Z.ravel()[idx] = L.ravel()[idx]               # X - S_t with S_t = R on Omega_t
    return L, out_masks, tape


def unrolled_loss(X, A1, k, T, Lstar, masks):
    L, _, _ = unrolled_forward(X, A1, k, T, masks)
    D = L - Lstar
    return float(np.sum(D * D))


def unrolled_vjp(X, A1, k, T, Lstar, masks):
    """Gradient of ||L_T - L*||_F^2 with respect to X (reverse mode, frozen masks).

    For L = Z P with Y2 = Z^T Z A1 and P = Y2 (Y2^T Y2)^{-1} Y2^T:
      dL = dZ P + Z dP,  dP = (I-P) dY2 Y2^+ + (Y2^+)^T dY2^T (I-P),
      dY2 = dZ^T Z A1 + Z^T dZ A1,
    so with H = Z^T gL:  gY2 = (I-P)(H + H^T)(Y2^+)^T and
      gZ = gL P + (Z A1) gY2^T + (Z gY2) A1^T.
    Z_1 = X and Z_{t+1} = (1-M_t) X + M_t L_t route gZ back to X and L_t.
    """
    X = np.asarray(X, dtype=np.float64)
    A1 = np.asarray(A1, dtype=np.float64)
    L, _, tape = unrolled_forward(X, A1, k, T, masks)
    gL = 2.0 * (L - Lstar)
    gX = np.zeros_like(X)
    n = X.shape[1]
    for t in range(T - 1, -1, -1):
        Z, P, Y2p_T = tape[t]
        IP = np.eye(n) - P
        W = Z.T @ (gL @ Y2p_T) + gL.T @ (Z @ Y2p_T)   # (H + H^T)(Y2^+)^T
        gY2 = IP @ W
        gZ = gL @ P + (Z @ A1) @ gY2.T + (Z @ gY2) @ A1.T
        if t == 0:
            gX += gZ
        else:
            m_idx = masks[t - 1]
            g_on = gZ.ravel()[m_idx].copy()
            gZ.ravel()[m_idx] = 0.0
            gX += gZ                                  # (1 - M_{t-1}) * gZ
            gL = np.zeros_like(X)
            gL.ravel()[m_idx] = g_on                  # M_{t-1} * gZ flows into L_{t-1}
    return gX


def unrolled_jvp(X, A1, k, T, Lstar, masks, Vdir):
    """Directional derivative of the loss along Vdir (forward mode, frozen masks)."""
    X = np.asarray(X, dtype=np.float64)
    A1 = np.asarray(A1, dtype=np.float64)
    Z = X.copy()
    dZ = np.asarray(Vdir, dtype=np.float64).copy()
    n = X.shape[1]
    for t in range(T):
        L, P, Y2, Y2p_T = _lstep_q0(Z, A1)
        dY2 = dZ.T @ (Z @ A1) + Z.T @ (dZ @ A1)
        IP = np.eye(n) - P
        dP = IP @ dY2 @ Y2p_T.T
        dP = dP + dP.T
        dL = dZ @ P + Z @ dP
        idx = masks[t]
        Z = X.copy()
        Z.ravel()[idx] = L.ravel()[idx]
        dZn = np.asarray(Vdir, dtype=np.float64).copy()
        dZn.ravel()[idx] = dL.ravel()[idx]
        dZ = dZn
    return float(2.0 * np.sum((L - Lstar) * dL))
