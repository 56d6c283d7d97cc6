"""Naive GoDec on the GPU (Sec. 2.1, eq. raw_lss: the L-step is the rank-r truncated SVD of
X - S) against the float64 oracle's naive_godec, whose L-step is numpy's exact SVD.

The GPU computes the truncated SVD by warm-started block subspace iteration; on these
workloads (a rank-r part well above the noise) it converges far below the float32 bar
within the first iterations.  Bars as for GoDec (reading R8): L within 1e-5 relative
Frobenius error, S on the common support within 1e-5, support mismatches only inside the
float32 rounding band of the k-th magnitude, the same number of iterations to the stop
test.
"""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_helpers import s_common_rel, selection_within_band, to_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_0302_gb300 as G
    G.library()


def _gpu(d, r, k, q, tol, max_iter, tag, n_iter=None):
    import paper_1309_0302_gb300 as G
    m, n = d["X"].shape
    p = G.naive_columns(m, n, r)
    om = synth.gaussian(1309, tag + "/omega", (n, p)).astype(np.float32)
    g = G.NaiveGoDec(to_gpu(d["X"]), to_gpu(om), r, k, q=q, tol=tol, max_iter=max_iter)
    try:
        if n_iter is None:
            it, rel = g.solve()
        else:
            rel = g.iterate(n_iter)
            it = n_iter
        U, s, V = (to_np(t).astype(np.float64) for t in g.L())
        idx, val = (to_np(t) for t in g.S())
    finally:
        g.close()
    return it, rel, U, s, V, idx, val.astype(np.float64)


def _compare(d, k, ref, U, s, V, idx, val, tag):
    L = (U * s) @ V.T
    eL = np.linalg.norm(L - ref["L"]) / np.linalg.norm(ref["L"])
    e_common, flips = s_common_rel(idx, val, ref["S_idx"], ref["S_val"])
    nb, inside = selection_within_band(d["X"], U, s, V, idx, k)
    print(f"naive {tag}: L {eL:.2e}, S common {e_common:.2e}, flips {flips}, band mismatches {nb}")
    assert eL <= 1e-5
    assert e_common <= 1e-5
    assert inside, nb


def test_naive_c1_solve():
    """The 500 x 500 workload (rank 10, 5 % sparse, noise 1e-3; r = 10) solved to tol 1e-7:
    the same iteration count as the oracle and the same end point."""
    d = synth.config_c1()
    it, rel, U, s, V, idx, val = _gpu(d, 10, d["k"], 2, 1e-7, 50, "naive_c1")
    ref = O.naive_godec(d["X"], 10, d["k"], tol=1e-7, max_iter=50)
    assert it == len(ref["E2_hist"])
    assert abs(rel - ref["E2_hist"][-1] / np.sum(d["X"].astype(np.float64) ** 2)) <= 1e-3 * rel
    _compare(d, d["k"], ref, U, s, V, idx, val, "c1")


@pytest.mark.parametrize("m,n,r", [(700, 333, 5), (260, 900, 12)])
def test_naive_odd_shapes_three_iterations(m, n, r):
    """Ragged shapes (product tiles and residual tiles cut at the edges), three iterations."""
    d = synth.small_case(m, n, r, 0.03, r, 1, tag=f"naive{m}x{n}")
    it, rel, U, s, V, idx, val = _gpu(d, r, d["k"], 2, -1.0, 50, f"naive{m}x{n}", n_iter=3)
    ref = O.naive_godec(d["X"], r, d["k"], tol=-1.0, max_iter=3)
    _compare(d, d["k"], ref, U, s, V, idx, val, f"{m}x{n}")
