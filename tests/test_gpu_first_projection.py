"""The chain's first projection from the cached X A1: (X - S) A1 = X A1 - S A1, with X A1
formed once and S A1 summed over the support of S (Algorithm 1's L-step, product L~ A1 with
A1 fixed).  Both ways of forming it, forced with GODEC_FLAG_SPARSE_FIRST and
GODEC_FLAG_DENSE_FIRST, are checked against the float64 oracle; the sparse one also on rows
with more entries than one staging pass holds, rows wider than one bitmap chunk, a rank drop
(A1 loses columns) and bitwise determinism.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_helpers import GpuRun, lfro_rel, s_common_rel, s_rel, selection_within_band, to_np

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


def _flags():
    import paper_1309_0302_gb300 as G
    return {"sparse": G.FLAG_SPARSE_FIRST, "dense": G.FLAG_DENSE_FIRST}


@pytest.mark.parametrize("way", ["sparse", "dense"])
@pytest.mark.parametrize("m,n,rank,r,q,dens", [
    (777, 555, 6, 7, 1, 0.03), (129, 65, 3, 3, 1, 0.05), (2000, 1500, 50, 50, 2, 0.01),
    (1500, 97, 2, 2, 3, 0.04), (600, 900, 5, 5, 0, 0.002),
])
def test_trajectory_both_ways(way, m, n, rank, r, q, dens):
    d = synth.small_case(m, n, rank, dens, r, q, tag=f"fp_{m}_{n}")
    ref = O.godec(d["X"], d["A1"], d["k"], q, tol=-1.0, max_iter=5)
    run = GpuRun(d, flags=_flags()[way])
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


@pytest.mark.parametrize("m,n,dens", [(64, 1200, 1.0), (40, 12000, 0.3), (33, 10241, 0.6)])
def test_sparse_dense_rows_same_step(m, n, dens):
    """Rows with up to n entries (a 16-word step then holds 512 of them, more than one
    staging pass) and rows wider than one bitmap chunk (10240 columns): one float64 oracle
    step from the GPU's S_{t-1} must give the GPU's L_t and S_t."""
    d = synth.small_case(m, n, 3, dens, 3, 1, tag=f"fpd_{m}_{n}")
    run = GpuRun(d, flags=_flags()["sparse"])
    S_prev = (np.zeros(0, np.int64), np.zeros(0))
    for t in range(3):
        run.g.iterate(1)
        st = O.godec_step(d["X"], d["A1"], S_prev[0], S_prev[1], d["k"], d["q"])
        U, s, V = run.factors()
        assert lfro_rel(U, s, V, st["U"], st["sigma"], st["V"]) <= TOL_L, t
        i, v = run.sparse()
        # at these densities the k-th magnitude sits in the noise: entries may flip inside
        # the float32 band, the shared support must agree
        e_common, _ = s_common_rel(i, v, st["S_idx"], st["S_val"])
        assert e_common <= TOL_S, t
        nb, inside = selection_within_band(d["X"], U, s, V, i, d["k"])
        assert inside, (t, nb)
        S_prev = (i, v)


@pytest.mark.parametrize("q", [0, 2])
def test_rank_drop_sparse_first(q):
    """A rank drop zeroes columns of A1 and of the cached X A1; the recovery of an exactly
    rank-4 X from 9 test columns is exact, as with the streamed projection."""
    g = np.random.default_rng(70 + q)
    X = (g.standard_normal((300, 4)) @ g.standard_normal((4, 260))).astype(np.float32)
    A1 = g.standard_normal((260, 9)).astype(np.float32)
    d = {"X": X, "A1": A1, "r": 9, "k": 0, "q": q}
    run = GpuRun(d, flags=_flags()["sparse"])
    run.g.iterate(3)
    info = run.g.info()
    assert info["r_eff"] == 4 and info["rank_drops"] >= 1
    U, s, V = run.factors()
    assert np.linalg.norm((U * s) @ V.T - X) <= 1e-5 * np.linalg.norm(X)
    ref = O.godec(X, A1, 0, q, tol=-1.0, max_iter=3)
    assert lfro_rel(U, s, V, ref["U"], ref["sigma"], ref["V"]) <= TOL_L


def test_sparse_first_bitwise_deterministic():
    d = synth.small_case(900, 700, 8, 0.02, 8, 1, tag="fp_det")
    outs = []
    for _ in range(2):
        run = GpuRun(d, flags=_flags()["sparse"])
        run.g.iterate(4)
        outs.append(run.factors32() + run.sparse())
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_default_way_is_streamed():
    """Without a flag the first projection streams Z at any density: the default run is
    bitwise the run with GODEC_FLAG_DENSE_FIRST."""
    for dens in (0.002, 0.02):
        d = synth.small_case(500, 400, 5, dens, 5, 1, tag=f"fp_def_{dens}")
        outs = []
        for flags in (0, _flags()["dense"]):
            run = GpuRun(d, flags=flags)
            run.g.iterate(3)
            outs.append(run.factors32() + run.sparse())
        for a, b in zip(*outs):
            assert np.array_equal(a, b), dens


def test_reset_reforms_cached_product():
    """godec_reset re-forms X A1 (the caller may change X between runs), so a run after a
    reset repeats the first one bitwise."""
    d = synth.small_case(400, 300, 4, 0.02, 4, 1, tag="fp_reset")
    run = GpuRun(d, flags=_flags()["sparse"])
    run.g.iterate(3)
    a = run.factors32() + run.sparse()
    run.g.reset()
    run.g.iterate(3)
    b = run.factors32() + run.sparse()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
