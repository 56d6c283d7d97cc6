"""Parity of the precision form (float16 chain + one float32 correction) with the oracle.

The oracle of this form is the float64 L-step of Algorithm 1 (O.godec_step) followed by the
same tangent-space correction in float64 (O.tangent_refine, reading R11, pinned in
test_oracle.py): the GPU's corrected L must match it to 1e-5 (relative Frobenius).  The
float16 chain alone (flag FLAG_NO_REFINE) must match the plain float64 L-step to 1e-3.
Inputs are seeded low-rank + sparse + noise matrices of the C3 shape class (tall, small r).
"""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_helpers import lfro_rel, to_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_0302_gb300 as G
    G.library()


def _first_step(d, flags):
    import paper_1309_0302_gb300 as G
    g = G.GoDec(to_gpu(d["X"]), to_gpu(d["A1"]), d["r"], d["k"], d["q"], tol=0.0, max_iter=4,
                precision=G.PREC_BF16_REFINE, flags=flags)
    g.iterate(1)
    U, s, V = g.L()
    idx, val = g.S()
    g.close()
    return to_np(U).astype(np.float64), to_np(s).astype(np.float64), to_np(V).astype(np.float64), to_np(idx), to_np(val)


@pytest.mark.parametrize("m,n,rank,r,q", [(3000, 400, 3, 3, 2), (2048, 512, 6, 6, 1), (4800, 200, 3, 3, 2),
                                          (1500, 700, 12, 12, 0)])
def test_precision_form_first_iteration(m, n, rank, r, q):
    import paper_1309_0302_gb300 as G
    d = synth.small_case(m, n, rank, 0.02, r, q, tag=f"prec{m}x{n}")
    X64 = d["X"].astype(np.float64)
    st = O.godec_step(X64, d["A1"].astype(np.float64), np.zeros(0, np.int64), np.zeros(0), d["k"], q)
    Ur, sr, Vr = O.tangent_refine(X64, st["U"], st["V"])
    # corrected: within 1e-5 of the float64 L-step + float64 correction
    U, s, V, idx, val = _first_step(d, 0)
    err = lfro_rel(U, s, V, Ur, sr, Vr)
    # float16 chain alone: within 1e-3 of the plain float64 L-step
    U0, s0, V0, _, _ = _first_step(d, G.FLAG_NO_REFINE)
    err0 = lfro_rel(U0, s0, V0, st["U"], st["sigma"], st["V"])
    print(f"precision form {m}x{n} r={r} q={q}: corrected {err:.2e}, chain only {err0:.2e}")
    assert err <= 1e-5
    assert err0 <= 1e-3


@pytest.mark.slow
def test_precision_form_c3_full_size():
    """C3 (76800 x 1000 video matrix, r = 3, k = 1.2e6, q = 2), two iterations: L against
    the float64 L-step + correction (<= 1e-5), the support of S against the exhaustive
    top-k of the float64 residual built from the GPU's own L (mismatches only inside the
    rounding band), S values on the common support, and the second iteration from the
    GPU's S_1 (the 16-bit copies of X - S after the scatter)."""
    import paper_1309_0302_gb300 as G
    from gpu_helpers import s_common_rel, selection_within_band
    d = synth.config_c3()
    X64, A64, k, q = d["X"].astype(np.float64), d["A1"].astype(np.float64), d["k"], d["q"]
    g = G.GoDec(to_gpu(d["X"]), to_gpu(d["A1"]), d["r"], k, q, tol=0.0, max_iter=4,
                precision=G.PREC_BF16_REFINE)
    try:
        errs = []
        S_idx, S_val = np.zeros(0, np.int64), np.zeros(0)
        for it in range(2):
            g.iterate(1)
            U, s, V = (to_np(t).astype(np.float64) for t in g.L())
            idx, val = (to_np(t) for t in g.S())
            st = O.godec_step(X64, A64, S_idx, S_val, k, q)
            Z = X64.copy()
            Z.ravel()[S_idx] -= S_val
            Ur, sr, Vr = O.tangent_refine(Z, st["U"], st["V"])
            del Z
            errs.append(lfro_rel(U, s, V, Ur, sr, Vr))
            nmis, inband = selection_within_band(d["X"], U, s, V, idx, k, chunk_rows=4096)
            R = X64 - (Ur * sr) @ Vr.T
            oi, ov = O.hard_threshold(R, k)
            del R
            serr, _ = s_common_rel(idx, val.astype(np.float64), oi, ov)
            print(f"C3 precision form iteration {it + 1}: L {errs[-1]:.2e}, S common {serr:.2e}, "
                  f"support mismatches {nmis} (in band: {inband})")
            assert idx.size == k
            assert inband
            assert serr <= 1e-5
            S_idx, S_val = idx.astype(np.int64), val.astype(np.float64)
        assert max(errs) <= 1e-5
    finally:
        g.close()
