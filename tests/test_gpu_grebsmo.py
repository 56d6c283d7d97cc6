"""GreBsmo on the GPU (Sec. 3.2.1, Algorithm 2, eqs. GreBsmoA, GreBsmoD, softt) against the
float64 oracle (oracle/grebsmo.py) with the same random-projection increments (reading
R22: the same seeded test matrices, the same number of power steps).

Bars: the same final rank and number of rank stages; the stage errors within 1e-4
relative; L = U V within 1e-5 relative Frobenius error; the support of S identical (the
cases keep every |X - U V| far from lambda, so no entry sits on the threshold) and its
values within 1e-5 relative.
"""
import numpy as np
import pytest

import oracle.grebsmo as GB
import synth
from gpu_helpers import to_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_0302_gb300 as G
    G.library()


def _case(m, n, rank, dens, s_lo, s_hi, sigma, tag):
    k = int(round(dens * m * n))
    d = synth.lowrank_sparse(m, n, rank, k, s_lo, s_hi, sigma, 1309, tag)
    # the sparse values of lowrank_sparse are uniform in [s_lo, s_hi]: give them random signs
    # of magnitude in [s_lo, s_hi] so that every outlier is far above lambda
    X = d["X"].astype(np.float64)
    sign = np.where(synth.uniform(1309, tag + "/sign", (k,), 0.0, 1.0) < 0.5, -1.0, 1.0)
    X.ravel()[d["S_idx"]] += (sign - 1.0) * d["S_val"]
    return X.astype(np.float32), k


def _run(X, lam, dr, K, tau, r_max, over, q_inc, tag):
    import paper_1309_0302_gb300 as G
    m, n = X.shape
    stages = 1 + -(-(r_max - dr) // dr)
    om = synth.gaussian(1309, tag + "/omega", (stages, n, dr + over)).astype(np.float32)
    ref = GB.grebsmo(X.astype(np.float64), lam=lam, dr=dr, K=K, tau=tau, r_max=r_max,
                     omegas=[om[s].astype(np.float64) for s in range(stages)], q_inc=q_inc)
    g = G.GreBsmo(to_gpu(X), to_gpu(om), lam, dr, K, tau, r_max, oversample=over, q_inc=q_inc)
    try:
        r, errs = g.run()
        U, s, V = (to_np(t).astype(np.float64) for t in g.L())
        idx, val = (to_np(t) for t in g.S())
        info = g.info()
    finally:
        g.close()
    return ref, r, errs, (U * s) @ V.T, idx, val.astype(np.float64), info


def _check(ref, r, errs, L, idx, val, info, K):
    Lr = ref["U"] @ ref["V"]
    eL = np.linalg.norm(L - Lr) / np.linalg.norm(Lr)
    ridx = np.flatnonzero(ref["S"].ravel())
    rval = ref["S"].ravel()[ridx]
    print(f"grebsmo: rank {r} (oracle {ref['r']}), stages {len(errs)}, L {eL:.2e}, "
          f"|S| {idx.size} (oracle {ridx.size}), errors {errs} vs {ref['errors']}")
    assert r == ref["r"]
    assert len(errs) == len(ref["errors"])
    assert np.allclose(errs, ref["errors"], rtol=1e-4, atol=1e-12)
    assert eL <= 1e-5
    assert np.array_equal(idx, ridx)
    assert np.linalg.norm(val - rval) <= 1e-5 * np.linalg.norm(rval)
    assert info["iter"] == K * len(errs)
    assert info["nnz"] == ridx.size


def test_grebsmo_finds_the_rank():
    """Low rank 3, 2 % outliers of magnitude 20-30, noise 1e-3, lambda = 3 (between the
    low-rank entries and the outliers): the greedy increments stop at rank 3 once the error
    falls to the shrinkage floor, on a 300 x 257 matrix (ragged product tiles)."""
    X, k = _case(300, 257, 3, 0.02, 20.0, 30.0, 1e-3, "greb_rank")
    lam = 3.0
    floor = k * lam ** 2 / float(np.sum(X.astype(np.float64) ** 2))
    out = _run(X, lam, 1, 10, 1.5 * floor, 8, 6, 4, "greb_rank")
    _check(*out, K=10)
    assert out[1] == 3


def test_grebsmo_without_sparse_part_is_the_truncated_svd():
    """lambda above every entry: S stays empty and U V is the rank-r_max truncation the
    oracle's increments build (dr = 2, three stages), on a tall 1100 x 300 matrix."""
    g = np.random.default_rng(2)
    m, n = 1100, 300
    Uf, _ = np.linalg.qr(g.standard_normal((m, 12)))
    Vf, _ = np.linalg.qr(g.standard_normal((n, 12)))
    X = ((Uf * (100.0 * 0.6 ** np.arange(12))) @ Vf.T).astype(np.float32)
    out = _run(X, 1e6, 2, 8, 0.0, 6, 6, 6, "greb_svd")
    _check(*out, K=8)
    assert out[4].size == 0


def test_grebsmo_wide_many_stages():
    """A wide 257 x 1030 matrix, rank 6 built in increments of dr = 2 with 3 % outliers."""
    X, k = _case(257, 1030, 6, 0.03, 15.0, 25.0, 1e-3, "greb_wide")
    lam = 2.0
    floor = k * lam ** 2 / float(np.sum(X.astype(np.float64) ** 2))
    out = _run(X, lam, 2, 8, 1.5 * floor, 10, 6, 4, "greb_wide")
    _check(*out, K=8)
