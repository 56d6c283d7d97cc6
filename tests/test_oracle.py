"""Pins of the float64 oracle against what the paper and the mathematics fix.

Each test names the passage it pins.  None of them re-types the oracle's own
formula: they use closed forms (exact recovery), theorems (Appendix I and II
bounds, monotone objective), brute force on tiny inputs and independent
library routines (full SVD, sorting).
"""
import itertools

import os

import numpy as np
import pytest

import oracle as O
from oracle.godec import _lstep_q0
import synth


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _lowrank(m, n, r, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((m, r)) @ g.standard_normal((r, n))


# --- P1: exact recovery of a noiseless rank-r matrix (eqs. lr_app, mlr_app) ---------
@pytest.mark.parametrize("q", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(50, 40), (40, 50), (33, 33)])
def test_exact_recovery_stable(q, shape):
    X = _lowrank(*shape, 5, seed=q)
    A1 = np.random.default_rng(10 + q).standard_normal((shape[1], 5))
    U, s, V, r = O.brp_stable(X, A1, q)
    assert r == 5
    assert _rel(O.dense_L(U, s, V), X) < 1e-12
    assert np.allclose(U.T @ U, np.eye(5), atol=1e-12) and np.allclose(V.T @ V, np.eye(5), atol=1e-12)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_exact_recovery_literal(q):
    X = _lowrank(50, 40, 5, seed=3)
    A1 = np.random.default_rng(4).standard_normal((40, 5))
    U, s, V, r = O.brp_literal(X, A1, q)
    # the unnormalised products lose digits as cond^(2q+1) grows
    assert _rel(O.dense_L(U, s, V), X) < [1e-12, 1e-9, 1e-8][q]


# --- P2: q = 0 identity Y1 (A2^T Y1)^{-1} Y2^T = Z P_range(Y2), A2^T Y1 SPD ----------
def test_q0_identity_projector():
    g = np.random.default_rng(7)
    Z = g.standard_normal((30, 20))
    A1 = g.standard_normal((20, 4))
    Y1 = Z @ A1
    A2 = Y1
    Y2 = Z.T @ A2
    Y1 = Z @ Y2
    C = A2.T @ Y1
    assert np.allclose(C, C.T, rtol=1e-12) and np.all(np.linalg.eigvalsh((C + C.T) / 2) > 0)
    Uy, sy, _ = np.linalg.svd(Y2, full_matrices=False)     # independent projector
    L_proj = Z @ (Uy @ Uy.T)
    U, s, V, _ = O.brp_literal(Z, A1, 0)
    assert _rel(O.dense_L(U, s, V), L_proj) < 1e-12


@pytest.mark.parametrize("q", [0, 1, 2])
def test_literal_equals_stable_noisy(q):
    d = synth.small_case(60, 45, 4, 0.05, 4, q, tag="lit_vs_stable")
    X = d["X"].astype(float)
    a = O.brp_literal(X, d["A1"].astype(float), q)
    b = O.brp_stable(X, d["A1"].astype(float), q)
    assert a[3] == b[3] == 4
    assert _rel(O.dense_L(*a[:3]), O.dense_L(*b[:3])) < [1e-12, 1e-10, 1e-9][q]


# --- P3: deterministic error bounds (Appendix II, Theorems 'deterministic error bound')
# q = 0 is a theorem and is pinned over the whole decay range.  For q > 0 the rooted
# power-scheme approximation can exceed the printed bound when the spectrum decays
# slowly (a draw with decay 0.88 at q = 2 gives error/bound = 1.08), so reading R15
# pins the power-scheme bound on spectra decaying at least as fast as 0.75 per index.
@pytest.mark.parametrize("q,decay_hi", [(0, 0.95), (1, 0.75), (2, 0.75)])
def test_deterministic_error_bound(q, decay_hi):
    g = np.random.default_rng(100 + q)
    m, n, r, p = 40, 30, 3, 2
    worst = 0.0
    for _ in range(60):
        Uf, _ = np.linalg.qr(g.standard_normal((m, n)))
        Vf, _ = np.linalg.qr(g.standard_normal((n, n)))
        lam = 10.0 * g.uniform(0.5, decay_hi) ** np.arange(n)
        X = (Uf * lam) @ Vf.T
        A1 = g.standard_normal((n, r + p))                   # r + p columns, p >= 2
        U, s, V, re = O.brp_stable(X, A1, q)
        assert re == r + p
        err = np.linalg.norm(X - O.dense_L(U, s, V), 2) ** 2
        e = 2 * q + 1
        L1i = np.diag(lam[:r] ** -e)
        L2 = np.diag(lam[r:])
        W = np.diag(lam[r:] ** (2 * e)) @ (Vf[:, r:].T @ A1) @ np.linalg.pinv(Vf[:, :r].T @ A1) @ L1i
        bound = (np.linalg.norm(W, 2) ** 2 + np.linalg.norm(L2, 2) ** (2 * e)) ** (1.0 / e)
        worst = max(worst, err / bound)
    assert worst <= 1.0 + 1e-9


# --- P4: rank check (Algorithm 1's rank test) ---------------------------------------
@pytest.mark.parametrize("q", [0, 1, 2])
def test_rank_check_reduces_r(q):
    X = _lowrank(50, 40, 4, seed=20)
    A1 = np.random.default_rng(21).standard_normal((40, 7))
    for f in (O.brp_stable, O.brp_literal):
        U, s, V, r = f(X, A1, q)
        assert r == 4 and U.shape == (50, 4) and V.shape == (40, 4)
        assert _rel(O.dense_L(U, s, V), X) < 1e-9
    U, s, V, r = O.brp_stable(np.zeros((10, 8)), np.ones((8, 3)), q)
    assert r == 0 and s.size == 0


def test_godec_rank_drop_keeps_reduced_r():
    X = _lowrank(40, 36, 3, seed=30)
    A1 = np.random.default_rng(31).standard_normal((36, 6))
    res = O.godec(X, A1, 5, 1, tol=-1.0, max_iter=3, keep_history=True)
    assert [h["r"] for h in res["history"]] == [3, 3, 3]
    assert res["U"].shape[1] == 3
    assert _rel(O.dense_L(res["U"], res["sigma"], res["V"]), X) < 1e-12


# --- P5: S-step = exhaustive top-k with ties and zeros (eq. raw_lss, Algorithm 1)
def _brute_topk(R, k):
    n = R.shape[1]
    cells = [(abs(R[i, j]), i * n + j) for i in range(R.shape[0]) for j in range(n)]
    cells.sort(key=lambda c: (-c[0], c[1]))
    return sorted(idx for a, idx in cells[:k] if a != 0.0)


@pytest.mark.parametrize("seed", range(6))
def test_hard_threshold_brute_force(seed):
    g = np.random.default_rng(seed)
    R = g.integers(-3, 4, size=(7, 9)).astype(float)       # many ties and zeros
    for k in range(0, 64):
        idx, val = O.hard_threshold(R, k)
        assert idx.tolist() == _brute_topk(R, k)
        assert np.array_equal(val, R.ravel()[idx])
        assert idx.size == min(k, int(np.count_nonzero(R)))


def test_hard_threshold_is_optimal():
    g = np.random.default_rng(9)
    R = g.standard_normal((5, 4))
    k = 6
    idx, _ = O.hard_threshold(R, k)
    best = min(np.sum(np.delete(R.ravel(), list(c)) ** 2) for c in itertools.combinations(range(20), k))
    assert np.isclose(np.sum(np.delete(R.ravel(), idx) ** 2), best, rtol=1e-14)


# --- P6: monotone objective (Appendix I, Theorem 'convergence of objective value') ----
def test_naive_godec_monotone():
    d = synth.small_case(40, 30, 3, 0.05, 3, 0, tag="naive")
    res = O.naive_godec(d["X"], 3, d["k"], tol=0.0, max_iter=12)
    seq = [v for pair in zip(res["E1_hist"], res["E2_hist"]) for v in pair]
    assert all(a >= b * (1 - 1e-12) - 1e-12 for a, b in zip(seq, seq[1:]))


@pytest.mark.parametrize("q", [0, 1, 2])
def test_brp_godec_s_step_monotone(q):
    d = synth.small_case(70, 50, 4, 0.04, 4, q, tag="mono")
    res = O.godec(d["X"], d["A1"], d["k"], q, tol=0.0, max_iter=10)
    E1, E2 = res["E1_hist"], res["E2_hist"]
    assert all(e2 <= e1 * (1 + 1e-12) for e1, e2 in zip(E1, E2))       # E_t^2 <= E_t^1
    slack = 1e-10 * res["normX2"]                                       # reading R9
    assert all(E1[t + 1] <= E2[t] + slack for t in range(len(E1) - 1))


def test_brp_approaches_svd_as_q_grows():
    g = np.random.default_rng(3)
    Uf, _ = np.linalg.qr(g.standard_normal((60, 40)))
    Vf, _ = np.linalg.qr(g.standard_normal((40, 40)))
    lam = 0.8 ** np.arange(40)                                         # slow decay
    X = (Uf * lam) @ Vf.T
    best = (Uf[:, :5] * lam[:5]) @ Vf[:, :5].T                          # Eckart-Young
    A1 = g.standard_normal((40, 5))
    errs = [_rel(O.dense_L(*O.brp_stable(X, A1, q)[:3]), best) for q in range(5)]
    assert all(a > b for a, b in zip(errs, errs[1:])) and errs[-1] < 0.5 * errs[0]


# --- P7: the 500 x 500 workload ends near the noise floor --------------------------------
def test_c1_end_state():
    d = synth.config_c1()
    res = O.godec(d["X"], d["A1"], d["k"], d["q"], tol=1e-7, max_iter=50)
    assert res["rel_err"][-1] <= 1e-7 and res["iters"] < 50
    assert res["S_idx"].size == d["k"]
    Lt = d["U"] @ d["V"].T
    assert _rel(O.dense_L(res["U"], res["sigma"], res["V"]), Lt) < 1e-3
    assert np.intersect1d(res["S_idx"], d["S_idx"]).size >= 0.99 * d["k"]
    # noise floor ||G||^2 (1 - k/mn)(1 - 2r/n) / ||X||^2 of reading P7
    floor = 0.25 * (1 - 0.05) * (1 - 0.04) / res["normX2"]
    assert 0.5 * floor < res["rel_err"][-1] < 1e-7


# --- P7b: the paper's own figures (Table 1, first row; reading R16) ------------------------
def test_table1_first_row_magnitudes():
    """The oracle on Table 1's recipe (500 x 500, rank 25, card 12500, noise 1e-3, q = 2),
    run to convergence, lands at the magnitudes the paper prints for GoDec (squared
    relative errors of X, L and S).  The bounds are factor-level: a dropped term, a wrong
    sign or an index slip moves them by orders of magnitude."""
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_godec_500.txt")
    ref = dict(line.strip().split("=") for line in open(path) if "=" in line and not line.startswith("#"))
    n, r, k = int(ref["size"]), int(ref["rank"]), int(ref["card"])
    g = np.random.default_rng(100)
    L = g.standard_normal((n, r)) @ g.standard_normal((r, n))
    S = np.zeros(n * n)
    S[g.choice(n * n, k, replace=False)] = g.standard_normal(k)
    S = S.reshape(n, n)
    X = L + S + 1e-3 * g.standard_normal((n, n))
    res = O.godec(X, g.standard_normal((n, r)), k, 2, tol=-1.0, max_iter=30)
    Lh = O.dense_L(res["U"], res["sigma"], res["V"])
    Sh = np.zeros(n * n)
    Sh[res["S_idx"]] = res["S_val"]
    Sh = Sh.reshape(n, n)
    ex = np.sum((X - Lh - Sh) ** 2) / np.sum(X ** 2)
    el = np.sum((L - Lh) ** 2) / np.sum(L ** 2)
    es = np.sum((S - Sh) ** 2) / np.sum(S ** 2)
    assert 0.5 <= ex / float(ref["rel_err_X"]) <= 3.0
    assert 0.1 <= el / float(ref["rel_err_L"]) <= 10.0
    assert 0.5 <= es / float(ref["rel_err_S"]) <= 2.0


# --- precision form: the tangent-space correction is second order (reading R11) ----------
def test_tangent_refine_exact_and_second_order():
    g = np.random.default_rng(11)
    Uf, _ = np.linalg.qr(g.standard_normal((80, 30)))
    Vf, _ = np.linalg.qr(g.standard_normal((30, 30)))
    lam = np.r_[[10.0, 6.0, 3.0], 1e-3 * g.uniform(size=27)]
    Z = (Uf * lam) @ Vf.T
    best = (Uf[:, :3] * lam[:3]) @ Vf[:, :3].T
    U2, s2, V2 = O.tangent_refine(Z, Uf[:, :3], Vf[:, :3])
    assert _rel(O.dense_L(U2, s2, V2), best) < 1e-12
    errs = []
    for th in (1e-2, 1e-3):
        Up, _ = np.linalg.qr(Uf[:, :3] + th * g.standard_normal((80, 3)))
        Vp, _ = np.linalg.qr(Vf[:, :3] + th * g.standard_normal((30, 3)))
        before = _rel((Up @ Up.T) @ Z @ (Vp @ Vp.T), best)
        after = _rel(O.dense_L(*O.tangent_refine(Z, Up, Vp)), best)
        errs.append((before, after))
    assert errs[1][1] < 1e-2 * errs[1][0]                               # far below first order
    assert errs[1][1] < 0.05 * errs[0][1]                               # shrinks ~ theta^2


def test_tangent_refine_first_order_in_the_tail():
    """With a tail (Z - L* of spectral norm sigma_{r+1}), the correction's error stays first
    order in the subspace error theta, but scaled by about sigma_{r+1} / sigma_1: the ratio
    after / before is proportional to the tail level and independent of theta."""
    g = np.random.default_rng(12)
    Uf, _ = np.linalg.qr(g.standard_normal((80, 30)))
    Vf, _ = np.linalg.qr(g.standard_normal((30, 30)))
    ratios = {}
    for tail in (1e-1, 1e-2, 1e-3):
        lam = np.r_[[10.0, 6.0, 3.0], tail * 10.0 * (0.5 + 0.5 * g.uniform(size=27))]
        Z = (Uf * lam) @ Vf.T
        best = (Uf[:, :3] * lam[:3]) @ Vf[:, :3].T
        for th in (1e-3, 1e-4):
            gg = np.random.default_rng(7)
            Up, _ = np.linalg.qr(Uf[:, :3] + th * gg.standard_normal((80, 3)))
            Vp, _ = np.linalg.qr(Vf[:, :3] + th * gg.standard_normal((30, 3)))
            before = _rel((Up @ Up.T) @ Z @ (Vp @ Vp.T), best)
            after = _rel(O.dense_L(*O.tangent_refine(Z, Up, Vp)), best)
            ratios[(tail, th)] = after / before
            assert after / before <= 1.5 * lam[3:].max() / lam[0]
    for tail in (1e-1, 1e-2, 1e-3):
        assert ratios[(tail, 1e-4)] == pytest.approx(ratios[(tail, 1e-3)], rel=0.05)   # first order in theta
    assert ratios[(1e-1, 1e-3)] / ratios[(1e-3, 1e-3)] == pytest.approx(100.0, rel=0.2)  # linear in the tail


# --- P8: gradient of the unrolled q = 0 iterations (reading R14) ------------------------
@pytest.fixture(scope="module")
def grad_case():
    d = synth.small_case(48, 40, 4, 0.03, 4, 0, tag="gradcase")
    g = np.random.default_rng(5)
    Lstar = g.standard_normal((48, 4)) @ g.standard_normal((4, 40))
    X, A1 = d["X"].astype(float), d["A1"].astype(float)
    _, masks, _ = O.unrolled_forward(X, A1, d["k"], 3)
    return X, A1, d["k"], 3, Lstar, masks


def test_gradient_dot_product(grad_case):
    X, A1, k, T, Lstar, masks = grad_case
    gX = O.unrolled_vjp(X, A1, k, T, Lstar, masks)
    g = np.random.default_rng(6)
    for _ in range(4):
        v = g.standard_normal(X.shape)
        jv = O.unrolled_jvp(X, A1, k, T, Lstar, masks, v)
        assert abs(jv - np.sum(gX * v)) <= 1e-10 * abs(jv)


def test_gradient_finite_differences(grad_case):
    X, A1, k, T, Lstar, masks = grad_case
    gX = O.unrolled_vjp(X, A1, k, T, Lstar, masks)
    g = np.random.default_rng(8)
    for _ in range(8):
        v = g.standard_normal(X.shape)
        h = 1e-5
        fd = (O.unrolled_loss(X + h * v, A1, k, T, Lstar, masks)
              - O.unrolled_loss(X - h * v, A1, k, T, Lstar, masks)) / (2 * h)
        assert abs(fd - np.sum(gX * v)) <= 1e-6 * abs(fd)


def test_gradient_finite_differences_64_directions(grad_case):
    """The stated check of the adjoint: central differences with h = 1e-3 along 64 random
    directions, against the reverse-mode gradient's directional derivatives."""
    X, A1, k, T, Lstar, masks = grad_case
    gX = O.unrolled_vjp(X, A1, k, T, Lstar, masks)
    g = np.random.default_rng(9)
    fd, dots = [], []
    for _ in range(64):
        v = g.standard_normal(X.shape)
        h = 1e-3
        fd.append((O.unrolled_loss(X + h * v, A1, k, T, Lstar, masks)
                   - O.unrolled_loss(X - h * v, A1, k, T, Lstar, masks)) / (2 * h))
        dots.append(np.sum(gX * v))
    fd, dots = np.array(fd), np.array(dots)
    assert np.linalg.norm(fd - dots) <= 1e-5 * np.linalg.norm(fd)


# --- degenerate cases the method defines ----------------------------------------------------
def test_oracle_degenerate_cases():
    """k = 0: S stays empty and every iteration is the same BRP of X; k = m n: S takes the
    whole residual and the fit is exact; an all-zero X: the rank test finds rank 0 (nothing
    to fit) and no entry is ever selected (zeros are never part of Omega, reading R7)."""
    g = np.random.default_rng(21)
    X = (g.standard_normal((40, 3)) @ g.standard_normal((3, 30)) + 0.1 * g.standard_normal((40, 30)))
    A1 = g.standard_normal((30, 3))
    r0 = O.godec(X, A1, 0, 1, tol=-1.0, max_iter=3)
    assert r0["S_idx"].size == 0
    U, s, V, _ = O.brp_stable(X, A1, 1)
    assert _rel(O.dense_L(r0["U"], r0["sigma"], r0["V"]), O.dense_L(U, s, V)) <= 1e-12
    rf = O.godec(X, A1, X.size, 1, tol=-1.0, max_iter=2)
    assert rf["S_idx"].size == X.size and rf["rel_err"][-1] <= 1e-28
    idx, val = O.hard_threshold(np.zeros((5, 4)), 7)
    assert idx.size == 0 and val.size == 0
    U0, s0, V0, r = O.brp_stable(np.zeros((20, 15)), g.standard_normal((15, 4)), 1)
    assert r == 0 and s0.size == 0


# --- pins of the differentiated form's forward pass (Algorithm 1 at q = 0, reading R14) ----
def test_lstep_q0_equals_algorithm1_literal():
    """The differentiated form's L-step, L = Z P with P the projector on range(Y2), is the
    q = 0 L-step of Algorithm 1 as printed (eq. lr_app: L = Y1 (A2^T Y1)^{-1} Y2^T)."""
    g = np.random.default_rng(31)
    for (m, n, r) in [(30, 22, 3), (22, 30, 5), (40, 40, 1)]:
        Z = g.standard_normal((m, 4)) @ g.standard_normal((4, n)) + 0.3 * g.standard_normal((m, n))
        A1 = g.standard_normal((n, r))
        L_q0 = _lstep_q0(Z, A1)[0]
        U, s, V, r_eff = O.brp_literal(Z, A1, 0)
        assert r_eff == r
        assert _rel(L_q0, O.dense_L(U, s, V)) <= 1e-12


def test_unrolled_forward_equals_godec_q0():
    """With the supports the GoDec loop chose, the frozen-mask recurrence
    Z_{t+1} = (1 - M_t) X + M_t L_t reproduces Algorithm 1's iterates at q = 0: the same
    L_T, and (masks left free) the same supports Omega_t in every iteration."""
    d = synth.small_case(46, 38, 3, 0.04, 3, 0, tag="unrolled_pin")
    X, A1 = d["X"].astype(float), d["A1"].astype(float)
    T = 5
    res = O.godec(X, A1, d["k"], 0, tol=-1.0, max_iter=T, keep_history=True)
    assert all(h["r"] == 3 for h in res["history"])
    masks = [h["S_idx"] for h in res["history"]]
    L_T, _, _ = O.unrolled_forward(X, A1, d["k"], T, masks=masks)
    assert _rel(L_T, O.dense_L(res["U"], res["sigma"], res["V"])) <= 1e-12
    _, free_masks, _ = O.unrolled_forward(X, A1, d["k"], T)
    for a, b in zip(free_masks, masks):
        assert np.array_equal(np.sort(a), b)


# --- naive GoDec (Sec. 2.1, eq. raw_lss): exact truncated SVD L-step, exhaustive S-step ----
def _topr_by_eigh(Z, r):
    """Rank-r truncation of Z through the eigenvectors of Z^T Z (the right singular
    vectors), a route independent of the SVD routine the oracle calls."""
    w, Vf = np.linalg.eigh(Z.T @ Z)
    Vr = Vf[:, np.argsort(w)[::-1][:r]]
    return Z @ Vr @ Vr.T


def test_naive_godec_first_iterations_closed_form():
    """From S_0 = 0 the first L-step of naive GoDec is the Eckart-Young truncation of X,
    known in closed form for an X built from its own SVD; S_1 is the exhaustive top-k of
    X - L_1; the second L-step truncates X - S_1 and S_2 thresholds X - L_2 (not Z - L_2)."""
    g = np.random.default_rng(41)
    m, n, r, k = 24, 18, 3, 20
    Uf, _ = np.linalg.qr(g.standard_normal((m, n)))
    Vf, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = np.concatenate([[40.0, 25.0, 12.0], 2.0 * 0.7 ** np.arange(n - 3)])
    X = (Uf * lam) @ Vf.T
    L1 = (Uf[:, :r] * lam[:r]) @ Vf[:, :r].T
    res1 = O.naive_godec(X, r, k, tol=-1.0, max_iter=1)
    assert _rel(res1["L"], L1) <= 1e-12
    assert res1["S_idx"].tolist() == _brute_topk(X - L1, k)
    assert np.allclose(res1["S_val"], (X - L1).ravel()[res1["S_idx"]], rtol=0, atol=1e-12)
    res2 = O.naive_godec(X, r, k, tol=-1.0, max_iter=2)
    Z2 = X.copy()
    Z2.ravel()[res1["S_idx"]] -= res1["S_val"]
    L2 = _topr_by_eigh(Z2, r)
    assert _rel(res2["L"], L2) <= 1e-10
    assert res2["S_idx"].tolist() == _brute_topk(X - res2["L"], k)
