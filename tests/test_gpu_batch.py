"""Parity of the batched form (godec_batch_*) with the float64 oracle.

Every problem of a batch runs Algorithm 1 on its own matrix; the batch only changes how
the iterations are launched (one CUDA graph per batch iteration, SM budgets from the
autotuner).  So each problem is held to the plain form's bar (reading R8(ii)): from the
GPU's S_{t-1}, one float64 oracle step must give the GPU's L_t within 1e-5 and S_t with
support flips only inside the float32 rounding band.  Problems of uneven m, n, r and q
in one batch, a rank drop inside the batch graph (the problem finishes that iteration
on its own), the tuner's bookkeeping, and C4 at full size.
"""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_helpers import lfro_rel, s_common_rel, selection_within_band, to_gpu, to_np

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


SHAPES = [(300, 257, 4, 4, 1), (130, 700, 7, 7, 1), (512, 384, 12, 12, 2), (1000, 260, 2, 2, 0),
          (257, 1200, 32, 32, 1), (640, 640, 20, 20, 1)]


def _problems(shapes, dens=0.03):
    return [synth.small_case(m, n, rank, dens, r, q, tag=f"batch{j}") for j, (m, n, rank, r, q) in enumerate(shapes)]


def _batch(ds, tune=True):
    import paper_1309_0302_gb300 as G
    return G.GoDecBatch([to_gpu(d["X"]) for d in ds], [to_gpu(d["A1"]) for d in ds], [d["r"] for d in ds],
                        [d["k"] for d in ds], [d["q"] for d in ds], tune=tune)


def _state(p):
    U, s, V = (to_np(t).astype(np.float64) for t in p.L())
    i, v = p.S()
    return U, s, V, to_np(i), to_np(v).astype(np.float64)


def _same_step(d, S_prev, U, s, V, i, v):
    st = O.godec_step(d["X"], d["A1"], S_prev[0], S_prev[1], d["k"], d["q"])
    eL = lfro_rel(U, s, V, st["U"], st["sigma"], st["V"])
    e_common, flips = s_common_rel(i, v, st["S_idx"], st["S_val"])
    return eL, e_common, flips


@pytest.mark.parametrize("tune", [True, False])
def test_batch_same_step(tune):
    ds = _problems(SHAPES)
    b = _batch(ds, tune)
    try:
        prev = [(np.zeros(0, np.int64), np.zeros(0)) for _ in ds]
        for t in range(3):
            b.iterate(1)
            for j, d in enumerate(ds):
                U, s, V, i, v = _state(b.problem(j))
                eL, ec, flips = _same_step(d, prev[j], U, s, V, i, v)
                nb, inside = selection_within_band(d["X"], U, s, V, i, d["k"])
                assert eL <= TOL_L, (t, j, eL)
                assert ec <= TOL_S, (t, j, ec)
                assert inside, (t, j, nb)
                prev[j] = (i.astype(np.int64), v)
    finally:
        b.close()


def test_batch_equals_single_problem_runs():
    """The same problems run one by one through godec_init contexts: L within float32
    rounding of the batch's after 4 iterations (grid sizes and the normaliser path change
    only the order of float32 sums)."""
    import paper_1309_0302_gb300 as G
    ds = _problems(SHAPES[:4])
    b = _batch(ds)
    try:
        b.iterate(4)
        for j, d in enumerate(ds):
            U, s, V, _, _ = _state(b.problem(j))
            g = G.GoDec(to_gpu(d["X"]), to_gpu(d["A1"]), d["r"], d["k"], d["q"], tol=-1.0, max_iter=10)
            g.iterate(4)
            U2, s2, V2 = (to_np(t).astype(np.float64) for t in g.L())
            g.close()
            assert lfro_rel(U, s, V, U2, s2, V2) <= 1e-5, j
            assert b.problem(j).info()["iter"] == 4
    finally:
        b.close()


def test_batch_rank_drop_inside_graph():
    """Problem 1 has true rank 4 but r = 9 and no sparse part: the rank test lowers r in
    the batch graph; that problem finishes the iteration on its own graphs and the next
    batch launch is captured again with its new r.  The others are unaffected."""
    g = np.random.default_rng(41)
    X = (g.standard_normal((300, 4)) @ g.standard_normal((4, 260))).astype(np.float32)
    A1 = g.standard_normal((260, 9)).astype(np.float32)
    drop = {"X": X, "A1": A1, "r": 9, "k": 0, "q": 1}
    ds = [_problems(SHAPES[:1])[0], drop, _problems(SHAPES[5:6])[0]]
    b = _batch(ds)
    try:
        b.iterate(3)
        info = b.problem(1).info()
        assert info["r_eff"] == 4 and info["rank_drops"] >= 1 and info["iter"] == 3
        U, s, V, _, _ = _state(b.problem(1))
        assert np.linalg.norm((U * s) @ V.T - X) <= 1e-5 * np.linalg.norm(X)
        for j in (0, 2):
            assert b.problem(j).info()["iter"] == 3
        b.iterate(1)
        assert all(b.problem(j).info()["iter"] == 4 for j in range(3))
    finally:
        b.close()


def test_batch_tuning_and_reset():
    import torch
    ds = _problems(SHAPES[:3])
    b = _batch(ds)
    try:
        t = b.tuning()
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        assert all(ms > 0 for ms in t["policy_ms"])
        assert t["policy"] == int(np.argmin(t["policy_ms"]))
        assert all(4 <= x <= nsm for x in t["sm"]) or t["policy"] == 0
        b.iterate(2)
        b.reset()
        assert all(b.problem(j).info()["iter"] == 0 for j in range(3))
        b.iterate(1)
        U, s, V, i, v = _state(b.problem(0))
        eL, ec, _ = _same_step(ds[0], (np.zeros(0, np.int64), np.zeros(0)), U, s, V, i, v)
        assert eL <= TOL_L and ec <= TOL_S
    finally:
        b.close()


def test_batch_rejects_bad_arguments():
    import paper_1309_0302_gb300 as G
    d = _problems(SHAPES[:1])[0]
    with pytest.raises(G.GodecError):   # k above m n in problem 0
        G.GoDecBatch([to_gpu(d["X"])], [to_gpu(d["A1"])], [d["r"]], [10 ** 9], [1])
    with pytest.raises(ValueError):
        G.GoDecBatch([to_gpu(d["X"])], [], [d["r"]], [d["k"]], [1])
    b = _batch([d])
    try:
        with pytest.raises(IndexError):
            b.problem(1)
    finally:
        b.close()


@pytest.mark.slow
def test_batch_c4_full_size():
    """C4: 64 problems (m, n log-uniform in [256, 4096], r in 2..32, 2-5 % sparse, q = 1),
    tuned budgets; iterations 1 and 2 of six of them (smallest, largest and four others)
    against one float64 oracle step each from the GPU's previous S."""
    ds = synth.config_c4()
    b = _batch(ds)
    try:
        sizes = [d["X"].size for d in ds]
        pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 5, 17, 33, 60})
        prev = {j: (np.zeros(0, np.int64), np.zeros(0)) for j in pick}
        for t in range(2):
            b.iterate(1)
            for j in pick:
                d = ds[j]
                U, s, V, i, v = _state(b.problem(j))
                eL, ec, flips = _same_step(d, prev[j], U, s, V, i, v)
                print(f"C4 problem {j} {d['X'].shape} r={d['r']} iteration {t + 1}: L {eL:.2e}, "
                      f"S common {ec:.2e}, flips {flips}")
                assert eL <= TOL_L and ec <= TOL_S
                assert flips <= max(4, 1e-4 * d["k"])
                prev[j] = (i.astype(np.int64), v)
        print("C4 tuning:", b.tuning()["policy_ms"], "policy", b.tuning()["policy"])
    finally:
        b.close()
