"""The timeout path of the device pipelines, exercised without faulting or hanging the
GPU: godec_check_timeout runs one bounded wait that nothing completes (an mbarrier no
thread arrives on, polled with the helper every pipeline wait uses, ~2 ms at most), which
gives up and flags the context as a pipeline wait does.  The call must return
GODEC_ERR_TIMEOUT, leave the iteration count and the factors as they were, and the
context must then iterate exactly as an untouched one.
"""
import numpy as np
import pytest

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


def _ctx(d):
    import paper_1309_0302_gb300 as G
    return G.GoDec(to_gpu(d["X"]), to_gpu(d["A1"]), d["r"], d["k"], d["q"], tol=-1.0, max_iter=50)


def test_bounded_wait_reports_timeout_and_context_recovers():
    import paper_1309_0302_gb300 as G
    d = synth.small_case(300, 260, 5, 0.03, 5, 1, tag="timeout")
    g, ref = _ctx(d), _ctx(d)
    try:
        g.iterate(2)
        ref.iterate(2)
        before = g.info()
        U0, s0, V0 = (to_np(t) for t in g.L())
        with pytest.raises(G.GodecError) as e:
            g.check_timeout(1000)
        assert e.value.status == 5
        assert "gave up" in str(e.value)
        after = g.info()
        assert after["iter"] == before["iter"]
        U1, s1, V1 = (to_np(t) for t in g.L())
        assert np.array_equal(U0, U1) and np.array_equal(s0, s1) and np.array_equal(V0, V1)
        # the context goes on as if nothing happened
        rel = g.iterate(2)
        rel_ref = ref.iterate(2)
        assert g.info()["iter"] == ref.info()["iter"] == 4
        assert abs(rel - rel_ref) <= 1e-9 * rel_ref   # the objective's float64 sums are atomic: last bits only
        for a, b in zip(g.L(), ref.L()):
            assert np.array_equal(to_np(a), to_np(b))
        ia, va = (to_np(t) for t in g.S())
        ib, vb = (to_np(t) for t in ref.S())
        assert np.array_equal(ia, ib) and np.array_equal(va, vb)
    finally:
        g.close()
        ref.close()


def test_timeout_self_test_rejects_bad_polls():
    import paper_1309_0302_gb300 as G
    d = synth.small_case(200, 200, 4, 0.03, 4, 0, tag="timeout_args")
    g = _ctx(d)
    try:
        for polls in (0, (1 << 20) + 1):
            with pytest.raises(G.GodecError) as e:
                g.check_timeout(polls)
            assert e.value.status == 1
        g.iterate(1)   # still usable
    finally:
        g.close()
