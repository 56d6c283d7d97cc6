"""Shared helpers of the GPU tests (not a test module)."""
import numpy as np


def to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_np(t):
    return t.detach().cpu().numpy()


def lfro_rel(Ua, sa, Va, Ub, sb, Vb):
    """||Ua diag(sa) Va^T - Ub diag(sb) Vb^T||_F / ||Ub diag(sb) Vb^T||_F from the factors."""
    Aa, Ab = Ua * sa, Ub * sb
    aa = np.sum((Aa.T @ Aa) * (Va.T @ Va))
    bb = np.sum((Ab.T @ Ab) * (Vb.T @ Vb))
    ab = np.sum((Aa.T @ Ab) * (Va.T @ Vb))
    return float(np.sqrt(max(aa + bb - 2.0 * ab, 0.0)) / np.sqrt(bb))


def s_rel(ia, va, ib, vb):
    """Relative Frobenius distance of two sparse matrices given as COO."""
    u = np.union1d(ia, ib)
    A = np.zeros(u.size)
    B = np.zeros(u.size)
    A[np.searchsorted(u, ia)] = va
    B[np.searchsorted(u, ib)] = vb
    nb = np.linalg.norm(B)
    return float(np.linalg.norm(A - B) / (nb if nb > 0 else 1.0))


def fma32(a, b, c):
    """float32 fused multiply-add emulated in float64 (the product is exact)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


class GpuRun:
    def __init__(self, d, tol=1e-7, max_iter=50, rank_tol=0.0, flags=0):
        import paper_1309_0302_gb300 as G
        self.d = d
        self.g = G.GoDec(to_gpu(d["X"]), to_gpu(d["A1"]), d["r"], d["k"], d["q"], tol=tol,
                         max_iter=max_iter, rank_tol=rank_tol, flags=flags)

    def factors(self):
        U, s, V = self.g.L()
        return to_np(U).astype(np.float64), to_np(s).astype(np.float64), to_np(V).astype(np.float64)

    def factors32(self):
        U, s, V = self.g.L()
        return to_np(U), to_np(s), to_np(V)

    def sparse(self):
        i, v = self.g.S()
        return to_np(i), to_np(v).astype(np.float64)


def s_common_rel(ia, va, ib, vb):
    """Relative error of S values on the common support (reading R8(iii))."""
    common, xa, xb = np.intersect1d(ia, ib, return_indices=True)
    nb = np.linalg.norm(vb)
    return float(np.linalg.norm(va[xa] - vb[xb]) / (nb if nb > 0 else 1.0)), int(ia.size + ib.size - 2 * common.size)


def selection_within_band(X, U, s, V, idx, k, chunk_rows=500):
    """Reading R8(ii): compare the GPU support with the exhaustive top-k of the float64
    residual built from the GPU's own L factors.  Every mismatch must lie within the
    rounding band of the kernel's residual, b = 16 u32 (|x| + sum_l |U_il s_l V_jl|),
    u32 = 2^-24: the two-term float16 split of each L factor is exact to 2^-22 (4 u32)
    per factor, the dropped low x low term adds 4 u32, the tensor core's float32
    accumulation over 64 K-terms at most 4 u32 more, and forming X - L one rounding.
    Returns (number of mismatches, all inside the band)."""
    m, n = X.shape
    Us = U * s
    R = np.empty((m, n))
    B = np.empty((m, n))
    for r0 in range(0, m, chunk_rows):
        r1 = min(m, r0 + chunk_rows)
        R[r0:r1] = X[r0:r1].astype(np.float64) - Us[r0:r1] @ V.T
        B[r0:r1] = np.abs(X[r0:r1]) + np.abs(Us[r0:r1]) @ np.abs(V.T)
    a = np.abs(R).ravel()
    kk = min(k, a.size)
    tau = np.partition(a, a.size - kk)[a.size - kk]
    ref = np.flatnonzero(a >= tau)
    diff = np.setxor1d(ref, idx)
    band = 16.0 * 2.0 ** -24 * B.ravel()[diff]
    return int(diff.size), bool(np.all(np.abs(a[diff] - tau) <= band + 1e-7 * tau))
