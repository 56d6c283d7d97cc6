"""Parity of the differentiated form (godec_backward, q = 0) with the float64 oracle.

The GPU runs T iterations of Algorithm 1 at q = 0; its supports Omega_1 .. Omega_{T-1}
are then frozen (reading R14) and the gradient of ||L_T - L*||_F^2 with respect to X
comes from godec_backward.  The oracle takes the same supports and computes its float64
reverse-mode gradient (itself pinned by central finite differences and a forward-mode
dot-product test in test_oracle.py).  Tolerance: relative Frobenius error of dX <= 1e-4
(float32 arithmetic through a T-step chain of r x r solves: errors of order
u32 cond(Y2) per step), L_T within 1e-5.  The cases take r equal to the rank of the
low-rank part: above it, Y2 has singular values at the noise level, the gradient's
dependence on them is ill-conditioned and no float32 tolerance holds.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL_DX = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_0302_gb300 as G
    G.library()


def _case(m, n, rank, density, r, T, seed):
    torch = pytest.importorskip("torch")
    d = synth.small_case(m, n, rank, density, r, 0, tag=f"bw{seed}")
    g = np.random.default_rng(seed)
    Us, Vs = g.standard_normal((m, r)), g.standard_normal((n, r))
    X = torch.from_numpy(d["X"]).cuda()
    A1 = torch.from_numpy(d["A1"]).cuda()
    return d, X, A1, Us, Vs


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("m,n,rank,r,T,seed", [(256, 192, 4, 4, 3, 1), (300, 257, 6, 6, 4, 2),
                                               (130, 129, 3, 3, 1, 3), (512, 384, 10, 10, 2, 4)])
def test_backward_matches_oracle(m, n, rank, r, T, seed):
    torch = pytest.importorskip("torch")
    import paper_1309_0302_gb300 as G
    d, X, A1, Us, Vs = _case(m, n, rank, 0.02, r, T, seed)
    k = d["k"]
    Lstar = Us @ Vs.T
    Xg = X.clone().requires_grad_(True)
    L = G.unrolled_godec(Xg, A1, r, k, T)
    loss = ((L - torch.from_numpy(Lstar).float().cuda()) ** 2).sum()
    loss.backward()
    dX = Xg.grad.cpu().numpy().astype(np.float64)
    # the same supports in the oracle (the last one does not enter the loss)
    gpu = G.GoDec(X, A1, r, k, 0, tol=0.0, max_iter=T)
    masks = []
    for _ in range(T):
        gpu.iterate(1)
        masks.append(gpu.S()[0].cpu().numpy())
    gpu.close()
    X64, A64 = d["X"].astype(np.float64), d["A1"].astype(np.float64)
    Lo, _, _ = O.unrolled_forward(X64, A64, k, T, masks)
    assert _rel(L.detach().cpu().numpy().astype(np.float64), Lo) <= 1e-5
    ref = O.unrolled_vjp(X64, A64, k, T, Lstar, masks)
    err = _rel(dX, ref)
    print(f"dX rel err {err:.2e}")
    assert err <= TOL_DX


def test_backward_finite_differences_64_directions():
    """The GPU adjoint against central differences of the loss (h = 1e-3, 64 random
    directions), the loss evaluated in float64 on the GPU's own supports: the directional
    derivatives dX . v agree with the differences to 1e-4 (relative, over all 64)."""
    torch = pytest.importorskip("torch")
    import paper_1309_0302_gb300 as G
    m, n, r, T = 256, 192, 4, 3
    d, X, A1, Us, Vs = _case(m, n, 4, 0.02, r, T, 11)
    k = d["k"]
    Lstar = Us @ Vs.T
    Xg = X.clone().requires_grad_(True)
    L = G.unrolled_godec(Xg, A1, r, k, T)
    ((L - torch.from_numpy(Lstar).float().cuda()) ** 2).sum().backward()
    dX = Xg.grad.cpu().numpy().astype(np.float64)
    gpu = G.GoDec(X, A1, r, k, 0, tol=0.0, max_iter=T)
    masks = []
    for _ in range(T):
        gpu.iterate(1)
        masks.append(gpu.S()[0].cpu().numpy())
    gpu.close()
    X64, A64 = d["X"].astype(np.float64), d["A1"].astype(np.float64)
    g = np.random.default_rng(12)
    fd, dots = [], []
    for _ in range(64):
        v = g.standard_normal((m, n))
        h = 1e-3
        fd.append((O.unrolled_loss(X64 + h * v, A64, k, T, Lstar, masks)
                   - O.unrolled_loss(X64 - h * v, A64, k, T, Lstar, masks)) / (2 * h))
        dots.append(np.sum(dX * v))
    fd, dots = np.array(fd), np.array(dots)
    err = float(np.linalg.norm(fd - dots) / np.linalg.norm(fd))
    print(f"finite differences, 64 directions: rel err {err:.2e}")
    assert err <= 1e-4


def test_backward_lowrank_equals_dense():
    torch = pytest.importorskip("torch")
    import paper_1309_0302_gb300 as G
    m, n, r, T = 256, 200, 5, 3
    d, X, A1, Us, Vs = _case(m, n, 5, 0.02, r, T, 7)
    k = d["k"]
    gpu = G.GoDec(X, A1, r, k, 0, tol=0.0, max_iter=T)
    sup = []
    for t in range(T):
        gpu.iterate(1)
        if t < T - 1:
            sup.append(gpu.S()[0].clone())
    gpu.close()
    g = np.random.default_rng(9)
    gU = torch.from_numpy(g.standard_normal((m, 7)).astype(np.float32)).cuda()
    gV = torch.from_numpy(g.standard_normal((n, 7)).astype(np.float32)).cuda()
    dX1 = G.backward(X, A1, T, sup, gU=gU, gV=gV).cpu().numpy()
    dX2 = G.backward(X, A1, T, sup, gL=gU @ gV.T).cpu().numpy()
    assert _rel(dX1, dX2) <= 1e-5


def test_backward_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    import paper_1309_0302_gb300 as G
    X = torch.zeros((128, 128), device="cuda")
    A1 = torch.ones((128, 4), device="cuda")
    gU = torch.ones((128, 2), device="cuda")
    with pytest.raises(ValueError):
        G.backward(X, A1, 2, [], gU=gU, gV=gU)           # T - 1 supports missing (binding)
    with pytest.raises(G.GodecError):                    # r above 64 (library)
        G.backward(X, torch.ones((128, 65), device="cuda"), 1, [], gU=gU, gV=gU)
    with pytest.raises(ValueError):                      # float64 gradient factors
        G.backward(X, A1, 1, [], gU=gU.double(), gV=gU.double())


@pytest.mark.parametrize("dense", [False, True])
def test_backward_rebuilt_iterates_match_kept(dense):
    """GODEC_BACKWARD_REBUILD (the iterates rebuilt in the backward sweep from X and the
    checkpoints) gives the gradient of the default, which keeps them from the forward sweep;
    only the float atomics of the sparse products may differ in the last bits."""
    torch = pytest.importorskip("torch")
    import paper_1309_0302_gb300 as G
    d, X, A1, Us, Vs = _case(300, 257, 6, 0.02, 6, 4, 5)
    r, k, T = d["r"], d["k"], 4
    gpu = G.GoDec(X, A1, r, k, 0, tol=0.0, max_iter=T)
    sup = []
    for t in range(T):
        gpu.iterate(1)
        if t < T - 1:
            sup.append(gpu.S()[0].clone())
    U, s, V = gpu.L()
    gpu.close()
    gU = torch.cat([2.0 * U * s, -2.0 * torch.from_numpy(Us).float().cuda()], 1).contiguous()
    gV = torch.cat([V, torch.from_numpy(Vs).float().cuda()], 1).contiguous()
    kw = {"gL": (gU @ gV.T).contiguous()} if dense else {"gU": gU, "gV": gV}
    kept = G.backward(X, A1, T, sup, **kw).cpu().numpy().astype(np.float64)
    rebuilt = G.backward(X, A1, T, sup, rebuild=True, **kw).cpu().numpy().astype(np.float64)
    assert np.isfinite(kept).all() and np.abs(kept).max() > 0
    assert _rel(rebuilt, kept) <= 1e-5


@pytest.mark.slow
def test_backward_c5_full_size():
    """C5 (4096 x 4096, r = 20, k = 2 %, q = 0, T = 10, loss ||L_T - L*||^2 with a rank-20
    L*): the GPU gradient (low-rank dL/dL_T = [2 U sigma | -2 U*] [V | V*]^T) against the
    float64 oracle gradient on the GPU's supports."""
    torch = pytest.importorskip("torch")
    import paper_1309_0302_gb300 as G
    d = synth.config_c5()
    m, n, r, k, T = 4096, 4096, d["r"], d["k"], d["T"]
    X = torch.from_numpy(d["X"]).cuda()
    A1 = torch.from_numpy(d["A1"]).cuda()
    gpu = G.GoDec(X, A1, r, k, 0, tol=0.0, max_iter=T)
    masks, sup = [], []
    for t in range(T):
        gpu.iterate(1)
        idx = gpu.S()[0]
        masks.append(idx.cpu().numpy())
        if t < T - 1:
            sup.append(idx.clone())
    U, s, V = gpu.L()
    gpu.close()
    Us = torch.from_numpy(d["Ustar"]).float().cuda()
    Vs = torch.from_numpy(d["Vstar"]).float().cuda()
    gU = torch.cat([2.0 * U * s, -2.0 * Us], dim=1).contiguous()
    gV = torch.cat([V, Vs], dim=1).contiguous()
    dX = G.backward(X, A1, T, sup, gU=gU, gV=gV).cpu().numpy().astype(np.float64)
    Lstar = d["Ustar"].astype(np.float64) @ d["Vstar"].astype(np.float64).T
    ref = O.unrolled_vjp(d["X"].astype(np.float64), d["A1"].astype(np.float64), k, T, Lstar, masks)
    err = _rel(dX, ref)
    print(f"C5 dX rel err {err:.2e}")
    assert err <= TOL_DX
