"""LinGoDec on the GPU (Sec. 4.3, eqs. LinGoDec and NLinGoDec with readings R20, R21) against
the float64 oracle (oracle/lingodec.py) after the same number of alternations.

Bars: W within 1e-5 relative Frobenius error; S on the common support within 1e-5 of
||W F^T||_F (S = R - lambda sgn R is formed from the float32 residual R = X - W F^T, whose
rounding scales with the low-rank part, about 20 times the outliers here, not with S);
support mismatches only at entries whose residual lies within float32 rounding of lambda
(a threshold decision taken in two precisions); the relative error within 1e-5.
"""
import numpy as np
import pytest

import oracle.lingodec as LG
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


def _recipe(m, n, d, r, rho, sigma, tag):
    """The paper's synthetic LinGoDec data: W a product of two Gaussians, Gaussian item
    features, a Bernoulli(rho) support with +-1 values, Gaussian noise."""
    W = synth.gaussian(1309, tag + "/Wa", (m, r)) @ synth.gaussian(1309, tag + "/Wb", (r, d))
    F = synth.gaussian(1309, tag + "/F", (n, d))
    u = synth.uniform(1309, tag + "/supp", (m, n), 0.0, 1.0)
    sgn = np.where(synth.uniform(1309, tag + "/sign", (m, n), 0.0, 1.0) < 0.5, -1.0, 1.0)
    S = np.where(u < rho, sgn, 0.0)
    X = W @ F.T + S + sigma * synth.gaussian(1309, tag + "/G", (m, n))
    return X.astype(np.float32), F.astype(np.float32)


@pytest.mark.parametrize("m,n,d,r,iters", [(600, 400, 20, 5, 10), (257, 1031, 12, 3, 6)])
def test_lingodec_matches_oracle(m, n, d, r, iters):
    import paper_1309_0302_gb300 as G
    X, F = _recipe(m, n, d, r, 0.05, 1e-3, f"lingo{m}x{n}")
    lam = 0.25
    ref = LG.lingodec(X.astype(np.float64), F.astype(np.float64), r, lam, iters)
    g = G.LinGoDec(to_gpu(X), to_gpu(F), r, lam)
    try:
        rel = g.iterate(iters)
        W = to_np(g.W()).astype(np.float64)
        idx, val = (to_np(t) for t in g.S())
        info = g.info()
    finally:
        g.close()
    eW = np.linalg.norm(W - ref["W"]) / np.linalg.norm(ref["W"])
    Sr = ref["S"].ravel()
    ridx = np.flatnonzero(Sr)
    common, ia, ib = np.intersect1d(idx, ridx, return_indices=True)
    eS = np.linalg.norm(val[ia].astype(np.float64) - Sr[common]) / np.linalg.norm(ref["W"] @ F.astype(np.float64).T)
    diff = np.setxor1d(idx, ridx)
    R = (X.astype(np.float64) - ref["W"] @ F.astype(np.float64).T).ravel()
    near = np.abs(np.abs(R[diff]) - lam) <= 1e-5 * (1.0 + np.abs(X.ravel()[diff]))
    Rr = X.astype(np.float64) - ref["W"] @ F.astype(np.float64).T - ref["S"]
    rel_ref = float(np.sum(Rr * Rr) / np.sum(X.astype(np.float64) ** 2))
    print(f"lingodec {m}x{n}: W {eW:.2e}, S common (of ||W F^T||) {eS:.2e}, support mismatches {diff.size} "
          f"(all near lambda: {bool(np.all(near))}), rel err {rel:.6e} vs {rel_ref:.6e}")
    assert eW <= 1e-5
    assert eS <= 1e-5
    assert np.all(near)
    assert abs(rel - rel_ref) <= 1e-5 * rel_ref
    assert info["iter"] == iters
