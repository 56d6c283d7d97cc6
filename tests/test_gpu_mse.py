"""MSE training on the GPU (Sec. 4.2.1, Algorithm 4 with the q = 0 BRP blocks) against the
float64 oracle (oracle/mse.py), both fed the same Gaussian test matrix at every block step.

Bars: the sum of the blocks within 1e-5 relative Frobenius error; the support of S equal
(the outliers stand far above the residual of the other entries) and its values within
1e-5; each label's subspace within 1e-4 of the oracle's (sine of the largest principal
angle); the objective history within 1e-4 relative (it is the squared norm of a small
float32 residual, as for GoDec's objective).
"""
import numpy as np
import pytest

import oracle.mse as MS
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


def _multilabel(n, p, k, r, K, noise, tag):
    """Synthetic multi-label data of the kind Algorithm 4 models (the real multi-label
    datasets are not reproduced): every sample carries each label with probability 0.35
    (at least one), label i adds a rank-r component with its own row space, plus K
    outliers of magnitude 5-10 and Gaussian noise."""
    u = synth.uniform(1309, tag + "/labels", (n, k), 0.0, 1.0)
    Y = (u < 0.35).astype(np.int32)
    Y[Y.sum(axis=1) == 0, 0] = 1
    X = np.zeros((n, p))
    for i in range(k):
        B = np.linalg.qr(synth.gaussian(1309, tag + f"/basis{i}", (p, r)))[0].T
        rows = np.flatnonzero(Y[:, i])
        X[rows] += synth.gaussian(1309, tag + f"/coef{i}", (rows.size, r)) @ B * 3.0
    pos = synth.sample_positions(1309, tag + "/outliers", n * p, K)
    mag = synth.uniform(1309, tag + "/mag", (K,), 5.0, 10.0)
    sgn = np.where(synth.uniform(1309, tag + "/sgn", (K,), 0.0, 1.0) < 0.5, -1.0, 1.0)
    X.ravel()[pos] += mag * sgn
    X += noise * synth.gaussian(1309, tag + "/noise", (n, p))
    return X.astype(np.float32), Y


class _Fixed:
    """Stands in for the oracle's random generator: hands out the given test matrices in
    the order Algorithm 4 draws them."""

    def __init__(self, mats):
        self._it = iter(mats)

    def standard_normal(self, shape):
        a = next(self._it)
        assert a.shape == tuple(shape)
        return a


def _sin_angle(A, B):
    """Sine of the largest principal angle between the row spaces of A and B."""
    Qa, _ = np.linalg.qr(A.T)
    Qb, _ = np.linalg.qr(B.T)
    s = np.linalg.svd(Qa.T @ Qb, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - s.min() ** 2)))


@pytest.mark.parametrize("n,p,k,r,K,iters", [(1500, 300, 4, 3, 2000, 6), (701, 129, 3, 2, 500, 4)])
def test_mse_matches_oracle(n, p, k, r, K, iters):
    import paper_1309_0302_gb300 as G
    tag = f"mse{n}x{p}"
    X, Y = _multilabel(n, p, k, r, K, 1e-3, tag)
    ranks = [r] * k
    A1s = synth.gaussian(1309, tag + "/A1", (iters, k, p, r)).astype(np.float32)
    ref = MS.mse_train(X.astype(np.float64), Y, ranks, K, iters,
                       brp_rng=_Fixed([A1s[t, i].astype(np.float64) for t in range(iters) for i in range(k)]))
    out = G.mse_train(to_gpu(X), Y, ranks, K, iters, to_gpu(A1s))
    Ls = to_np(out["Lsum"]).astype(np.float64)
    Lr = sum(ref["L"])
    eL = np.linalg.norm(Ls - Lr) / np.linalg.norm(Lr)
    idx, val = to_np(out["S_idx"]), to_np(out["S_val"]).astype(np.float64)
    ridx = np.flatnonzero(ref["S"].ravel())
    angles = [_sin_angle(to_np(out["C"])[i, :r].astype(np.float64), ref["C"][i]) for i in range(k)]
    h = np.array(out["history"])
    eh = np.max(np.abs(h - np.array(ref["history"])) / np.array(ref["history"]))
    print(f"mse {n}x{p}: sum of blocks {eL:.2e}, |S| {idx.size} (oracle {ridx.size}), subspace sines "
          f"{max(angles):.2e}, history {eh:.2e}: {h.tolist()} vs {ref['history']}")
    assert eL <= 1e-5
    assert np.array_equal(idx, ridx)
    assert np.linalg.norm(val - ref["S"].ravel()[ridx]) <= 1e-5 * np.linalg.norm(ref["S"].ravel()[ridx])
    assert max(angles) <= 1e-4
    assert eh <= 1e-4
