"""Parity of the CUDA path (through the C ABI) with the float64 oracle.

Tolerances (float32 path): relative Frobenius error of L <= 1e-5.  For S
(reading R8): the support equals the exhaustive top-k of the kernel's own
float32 residual (bit-exact against a CPU replica of that residual, or within
the float32 rounding band at full size); S values on the support shared with
the oracle agree to 1e-5; entries whose residual sits within the float32 error
of the k-th magnitude may flip between the float32 and the float64 run, and
their count is reported and bounded.  The hard threshold of a given array is
bit-exact.
"""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_helpers import (GpuRun, lfro_rel, s_common_rel, s_rel,
                         selection_within_band, to_gpu, to_np)

pytestmark = pytest.mark.gpu

TOL_L = 1e-5
TOL_S = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_0302_gb300 as G
    G.library()


# --- streaming products (the power chain of Algorithm 1) ------------------------------
@pytest.mark.parametrize("m,n,r", [(1000, 777, 50), (777, 1000, 3), (64, 64, 1), (2049, 131, 64),
                                   (5, 3000, 8), (3000, 7, 13), (130, 129, 33)])
def test_mul_primitives(m, n, r):
    import paper_1309_0302_gb300 as G
    g = np.random.default_rng(m * 7 + n)
    Z = g.standard_normal((m, n)).astype(np.float32)
    B = g.standard_normal((n, r)).astype(np.float32)
    Cm = g.standard_normal((m, r)).astype(np.float32)
    Y = to_np(G.mul_ZB(to_gpu(Z), to_gpu(B))).astype(np.float64)
    W = to_np(G.mul_ZtC(to_gpu(Z), to_gpu(Cm))).astype(np.float64)
    Yr = Z.astype(np.float64) @ B.astype(np.float64)
    Wr = Z.astype(np.float64).T @ Cm.astype(np.float64)
    assert np.linalg.norm(Y - Yr) <= 1e-5 * np.linalg.norm(Yr)
    assert np.linalg.norm(W - Wr) <= 1e-5 * np.linalg.norm(Wr)


# --- S-step alone: hard threshold with ties and zeros (eq. raw_lss, reading R7) ---------
@pytest.mark.parametrize("seed", range(3))
def test_hard_threshold_ties_zeros(seed):
    import paper_1309_0302_gb300 as G
    g = np.random.default_rng(seed)
    R = g.integers(-4, 5, size=(37, 45)).astype(np.float32)      # heavy ties, ~11% zeros
    for k in [0, 1, 7, 100, 500, 1000, 1400, 37 * 45]:
        idx, val = G.hard_threshold(to_gpu(R), k)
        ri, rv = O.hard_threshold(R.astype(np.float64), k)
        assert np.array_equal(to_np(idx), ri), k
        assert np.array_equal(to_np(val).astype(np.float64), rv), k


def test_hard_threshold_large_exact():
    import paper_1309_0302_gb300 as G
    g = np.random.default_rng(11)
    R = (g.standard_normal((1000, 1203)) * 3).astype(np.float32)
    R[g.random(R.shape) < 0.02] = 0.0
    R.ravel()[g.integers(0, R.size, 5000)] = 2.5                 # a large tie block
    for k in [10000, 40000, 1000 * 1203]:
        idx, val = G.hard_threshold(to_gpu(R), k)
        ri, rv = O.hard_threshold(R.astype(np.float64), k)
        assert np.array_equal(to_np(idx), ri)
        assert np.array_equal(to_np(val).astype(np.float64), rv)


# --- the 500 x 500 workload, whole trajectory with the stop test ------------------------
@pytest.fixture(scope="module")
def c1():
    d = synth.config_c1()
    ref = O.godec(d["X"], d["A1"], d["k"], d["q"], tol=d["tol"], max_iter=d["max_iter"])
    return d, ref


def test_c1_trajectory(c1):
    d, ref = c1
    run = GpuRun(d, tol=d["tol"], max_iter=d["max_iter"])
    iters, rel = run.g.solve()
    assert iters == ref["iters"]
    assert abs(rel - ref["rel_err"][-1]) <= 1e-3 * ref["rel_err"][-1]
    U, s, V = run.factors()
    assert lfro_rel(U, s, V, ref["U"], ref["sigma"], ref["V"]) <= TOL_L
    i, v = run.sparse()
    assert i.size == d["k"] and np.all(np.diff(i) > 0)
    assert s_rel(i, v, ref["S_idx"], ref["S_val"]) <= TOL_S


def test_c1_selection_is_exact_topk_of_kernel_residual(c1):
    """Reading R8(i): the GPU's Omega is exactly the top-k (ties by linear index) of the
    GPU's own float32 residual, read back densely from the same kernel."""
    d, _ = c1
    run = GpuRun(d)
    for t in range(3):
        run.g.iterate(1)
        R = to_np(run.g.residual())
        ri, rv = O.hard_threshold(R.astype(np.float64), d["k"])
        i, v = run.sparse()
        assert np.array_equal(i, ri), t
        assert np.array_equal(v, rv), t


def test_c1_same_step_each_iteration(c1):
    """Reading R8(ii): from the GPU's S_{t-1}, one float64 oracle step must give the
    GPU's L_t and S_t within tolerance (support flips only inside the float32 band)."""
    d, _ = c1
    run = GpuRun(d)
    S_prev = (np.zeros(0, np.int64), np.zeros(0))
    for t in range(4):
        run.g.iterate(1)
        st = O.godec_step(d["X"], d["A1"], S_prev[0], S_prev[1], d["k"], d["q"])
        U, s, V = run.factors()
        assert lfro_rel(U, s, V, st["U"], st["sigma"], st["V"]) <= TOL_L, t
        i, v = run.sparse()
        assert s_rel(i, v, st["S_idx"], st["S_val"]) <= TOL_S, t
        S_prev = (i, v)


# --- odd shapes: several tiles, ragged tails, every q ----------------------------------
@pytest.mark.parametrize("m,n,rank,r,q,dens", [
    (777, 555, 6, 7, 1, 0.03), (300, 1200, 10, 12, 0, 0.02), (1000, 250, 4, 4, 2, 0.05),
    (129, 65, 3, 3, 1, 0.05), (2000, 1500, 50, 50, 2, 0.01), (1500, 97, 2, 2, 3, 0.04),
])
def test_odd_shapes_trajectory(m, n, rank, r, q, dens):
    d = synth.small_case(m, n, rank, dens, r, q, tag=f"odd_{m}_{n}")
    ref = O.godec(d["X"], d["A1"], d["k"], q, tol=-1.0, max_iter=5)
    run = GpuRun(d)
    run.g.iterate(5)
    U, s, V = run.factors()
    assert run.g.info()["r_eff"] == ref["r"]
    assert lfro_rel(U, s, V, ref["U"], ref["sigma"], ref["V"]) <= TOL_L
    i, v = run.sparse()
    e_common, flips = s_common_rel(i, v, ref["S_idx"], ref["S_val"])
    assert e_common <= TOL_S
    assert flips <= 1e-3 * d["k"] + 4
    nb, inside = selection_within_band(d["X"], U, s, V, i, d["k"])
    assert inside, nb


# --- rank test of Algorithm 1 ------------------------------------------------------------
@pytest.mark.parametrize("q", [0, 1, 2])
def test_rank_drop_exact_recovery(q):
    g = np.random.default_rng(40 + q)
    X = (g.standard_normal((300, 4)) @ g.standard_normal((4, 260))).astype(np.float32)
    A1 = g.standard_normal((260, 9)).astype(np.float32)
    d = {"X": X, "A1": A1, "r": 9, "k": 0, "q": q}
    run = GpuRun(d)
    run.g.iterate(2)
    info = run.g.info()
    assert info["r_eff"] == 4 and info["rank_drops"] >= 1
    U, s, V = run.factors()
    L = (U * s) @ V.T
    assert np.linalg.norm(L - X) <= 1e-5 * np.linalg.norm(X)


# --- degenerate cases -------------------------------------------------------------------
def test_k_zero_and_k_everything():
    d = synth.small_case(200, 150, 3, 0.05, 3, 1, tag="kedge")
    for k in (0, 200 * 150):
        dd = dict(d, k=k)
        ref = O.godec(d["X"], d["A1"], k, 1, tol=-1.0, max_iter=3)
        run = GpuRun(dd)
        rel = run.g.iterate(3)
        U, s, V = run.factors()
        assert lfro_rel(U, s, V, ref["U"], ref["sigma"], ref["V"]) <= TOL_L
        i, v = run.sparse()
        assert i.size == ref["S_idx"].size
        if k == 0:
            assert abs(rel - ref["rel_err"][-1]) <= 1e-4 * ref["rel_err"][-1]
        else:
            assert rel <= 1e-12


def test_determinism_bitwise():
    d = synth.small_case(900, 700, 8, 0.02, 8, 1, tag="determinism")
    outs = []
    for _ in range(2):
        run = GpuRun(d)
        run.g.iterate(4)
        outs.append(run.factors32() + run.sparse())
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_nonfinite_input_reports_error():
    import paper_1309_0302_gb300 as G
    d = synth.small_case(100, 80, 3, 0.05, 3, 1, tag="nan")
    X = d["X"].copy()
    X[5, 7] = np.nan
    run = GpuRun(dict(d, X=X))
    with pytest.raises(G.GodecError) as e:
        run.g.iterate(1)
    assert e.value.status == 4


def test_run_host_matches_device_path():
    import paper_1309_0302_gb300 as G
    d = synth.small_case(640, 480, 5, 0.03, 5, 2, tag="hostpath")
    run = GpuRun(d)
    run.g.iterate(3)
    U, s, V = run.factors32()
    i, v = run.sparse()
    h = G.run_host(d["X"], d["A1"], d["r"], d["k"], d["q"], 3)
    assert h["r_eff"] == 5
    assert np.array_equal(h["U"], U) and np.array_equal(h["V"], V) and np.array_equal(h["sigma"], s)
    assert np.array_equal(h["S_idx"], i) and np.array_equal(h["S_val"].astype(np.float64), v)


# --- the 10000 x 10000 workload in the bench's launch configuration ------------------------
@pytest.mark.slow
@pytest.mark.parametrize("fp64_factor", [False, True])
def test_c2_full_size_same_step(fp64_factor):
    """Full-size check: GPU iterations 1..3 of the bench workload, then one float64
    oracle step from the GPU's S_2 compared with the GPU's iteration 3; with the default
    float32 Cholesky factors and with float64 ones (GODEC_FLAG_FP64_FACTOR), whose errors
    are printed side by side."""
    import paper_1309_0302_gb300 as G
    d = synth.config_c2()
    run = GpuRun(d, flags=G.FLAG_FP64_FACTOR if fp64_factor else 0)
    run.g.iterate(2)
    i2, v2 = run.sparse()
    assert i2.size == d["k"]
    run.g.iterate(1)
    st = O.godec_step(d["X"], d["A1"], i2, v2, d["k"], d["q"])
    U, s, V = run.factors()
    eL = lfro_rel(U, s, V, st["U"], st["sigma"], st["V"])
    i, v = run.sparse()
    e_common, flips = s_common_rel(i, v, st["S_idx"], st["S_val"])
    e_full = s_rel(i, v, st["S_idx"], st["S_val"])
    nb, inside = selection_within_band(d["X"], U, s, V, i, d["k"])
    info = run.g.info()
    print(f"c2 same-step ({'float64' if fp64_factor else 'float32'} factors): L {eL:.2e}, "
          f"S common {e_common:.2e}, S with flips {e_full:.2e}, flips {flips}, band mismatches {nb}")
    assert eL <= TOL_L
    assert e_common <= TOL_S
    assert flips <= 1e-4 * d["k"]
    assert inside, nb
    assert abs(info["obj"] - st["E2"]) <= 1e-4 * st["E2"]


# --- dense L from the library's own kernel (eq. mlr_app, L = U diag(sigma) V^T) ------------
@pytest.mark.parametrize("m,n,r,q", [(300, 257, 6, 1), (129, 700, 3, 0), (67, 65, 9, 2)])
def test_get_L_dense_matches_factors(m, n, r, q):
    """godec_get_L_dense writes U diag(sigma) V^T of the context's factors: every entry within
    float32 rounding of the float64 product of the factors godec_get_L returns, including the
    ragged tile edges (m, n not multiples of the 64 x 128 tile, odd row stride)."""
    import paper_1309_0302_gb300 as G
    d = synth.small_case(m, n, r, 0.03, r, q, tag=f"dense{m}x{n}")
    g = G.GoDec(to_gpu(d["X"]), to_gpu(d["A1"]), r, d["k"], q)
    try:
        g.iterate(2)
        U, s, V = (to_np(t).astype(np.float64) for t in g.L())
        L = to_np(g.L_dense()).astype(np.float64)
    finally:
        g.close()
    Lr = (U * s) @ V.T
    bound = 4 * r * 2.0 ** -24 * (np.abs(U) * s) @ np.abs(V).T + 1e-30
    assert L.shape == (m, n)
    assert np.all(np.abs(L - Lr) <= bound)
