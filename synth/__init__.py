"""Seeded synthetic inputs for GoDec-BRP workloads.

This module is the ONLY code shared by the CPU oracle (``oracle/``) and the
CUDA path (``paper_1309_0302_gb300``): it draws the data matrix X, the random
test matrix A1 and the ground truth, and holds none of the method's arithmetic.

Random numbers come from one counter-based generator written from its
published definition: output i of stream ``key`` is SplitMix64's finaliser
applied to ``key + (i + 1) * 0x9E3779B97F4A7C15`` (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014).  Uniform
doubles take the top 53 bits; normals use the cosine branch of Box-Muller
with two counters per draw.  Every array has its own stream, keyed by the
base seed and the array's name, so any slice can be regenerated alone.

Workload shapes follow the paper's synthetic experiment (Sec. 5.1: L = A B
with Gaussian factors, S on a uniformly drawn support, G = 1e-3 x Gaussian)
and, for the video-shaped case, a synthetic stand-in for the surveillance
sequences of Sec. 5.2 (no frame of any real video is reproduced).
"""
from __future__ import annotations

import math
import zlib

import numpy as np

__all__ = [
    "Stream", "gaussian", "uniform", "sample_positions", "lowrank_sparse",
    "config_c1", "config_c2", "config_c3", "config_c4", "config_c5",
    "small_case",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (variant 13 of Stafford's mix functions)."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """A counter-based stream of 64-bit words, keyed by (seed, name)."""

    def __init__(self, seed: int, name: str):
        with np.errstate(over="ignore"):
            base = np.array([(seed * 0x9E3779B97F4A7C15 + zlib.crc32(name.encode()))
                             & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
            self.key = _mix64(base)[0]

    def u64(self, start: int, count: int) -> np.ndarray:
        ctr = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        with np.errstate(over="ignore"):
            return _mix64(self.key + ctr * _GOLDEN)

    def uniform(self, start: int, count: int) -> np.ndarray:
        """Doubles in [0, 1) from counters start .. start+count-1."""
        return (self.u64(start, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, start: int, count: int) -> np.ndarray:
        """Standard normals; draw i uses counters 2(start+i) and 2(start+i)+1."""
        out = np.empty(count, dtype=np.float64)
        for c0 in range(0, count, _CHUNK):
            c = min(_CHUNK, count - c0)
            u = self.uniform(2 * (start + c0), 2 * c).reshape(c, 2)
            u1 = 1.0 - u[:, 0]                      # (0, 1]
            out[c0:c0 + c] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u[:, 1])
        return out


def gaussian(seed: int, name: str, shape, start: int = 0) -> np.ndarray:
    n = int(np.prod(shape))
    return Stream(seed, name).normal(start, n).reshape(shape)


def uniform(seed: int, name: str, shape, lo: float, hi: float) -> np.ndarray:
    n = int(np.prod(shape))
    return lo + (hi - lo) * Stream(seed, name).uniform(0, n).reshape(shape)


def sample_positions(seed: int, name: str, total: int, k: int) -> np.ndarray:
    """k distinct positions of [0, total) drawn uniformly, returned ascending.

    Uniform draws are de-duplicated in draw order, so the first k distinct
    values form a uniformly random k-subset.
    """
    if k < 0 or k > total:
        raise ValueError("need 0 <= k <= total")
    if k == 0:
        return np.zeros(0, dtype=np.int64)
    st = Stream(seed, name)
    drawn = np.zeros(0, dtype=np.int64)
    start, batch = 0, k + k // 4 + 1024
    while True:
        idx = np.minimum((st.uniform(start, batch) * total).astype(np.int64), total - 1)
        start += batch
        drawn = np.concatenate([drawn, idx])
        uniq, first = np.unique(drawn, return_index=True)
        if uniq.size >= k:
            keep = np.sort(first)[:k]
            return np.sort(drawn[keep])
        batch = max(1024, 2 * (k - uniq.size))


def lowrank_sparse(m: int, n: int, rank: int, k: int, s_lo: float, s_hi: float,
                   sigma: float, seed: int, tag: str, r_a1: int | None = None,
                   row_block: int = 512) -> dict:
    """X = U V^T + S + G with Gaussian factors, k uniform sparse entries and noise.

    X is formed in float64 and rounded once to float32; both paths use that
    float32 array (the oracle promotes it to float64).  A1 (n x r_a1) is
    N(0, 1), drawn in float64 and rounded to float32 for the same reason.
    """
    U = gaussian(seed, tag + "/U", (m, rank))
    V = gaussian(seed, tag + "/V", (n, rank))
    pos = sample_positions(seed, tag + "/omega", m * n, k)
    sval = uniform(seed, tag + "/svals", (k,), s_lo, s_hi)
    X = np.empty((m, n), dtype=np.float32)
    noise = Stream(seed, tag + "/G")
    for r0 in range(0, m, row_block):
        r1 = min(m, r0 + row_block)
        blk = U[r0:r1] @ V.T
        if sigma != 0.0:
            blk += sigma * noise.normal(r0 * n, (r1 - r0) * n).reshape(r1 - r0, n)
        lo, hi = np.searchsorted(pos, [r0 * n, r1 * n])
        p = pos[lo:hi] - r0 * n
        blk.reshape(-1)[p] += sval[lo:hi]
        X[r0:r1] = blk.astype(np.float32)
    r_a1 = rank if r_a1 is None else r_a1
    A1 = gaussian(seed, tag + "/A1", (n, r_a1)).astype(np.float32)
    return {"X": X, "A1": A1, "U": U, "V": V, "S_idx": pos, "S_val": sval}


def config_c1(seed: int = 1309) -> dict:
    """500 x 500, rank 10, k = 12500 (5 %) U[-10, 10], noise 1e-3; r=10, q=1."""
    d = lowrank_sparse(500, 500, 10, 12500, -10.0, 10.0, 1e-3, seed, "c1")
    d.update(r=10, k=12500, q=1, tol=1e-7, max_iter=50, name="c1_500x500_r10_q1")
    return d


def config_c2(seed: int = 1309) -> dict:
    """10000 x 10000, rank 50, k = 1e6 (1 %) U[-20, 20], noise 1e-2; r=50, q=2."""
    d = lowrank_sparse(10000, 10000, 50, 1000000, -20.0, 20.0, 1e-2, seed, "c2")
    d.update(r=50, k=1000000, q=2, tol=1e-7, max_iter=30, name="c2_10000x10000_r50_q2")
    return d


def small_case(m: int, n: int, rank: int, density: float, r: int, q: int,
               seed: int = 1309, s_amp: float = 10.0, sigma: float = 1e-3,
               tag: str | None = None) -> dict:
    """A small C1/C2-shaped case used for parity tests at odd sizes."""
    k = int(round(density * m * n))
    tag = tag or f"small_{m}x{n}_{rank}_{r}_{q}"
    d = lowrank_sparse(m, n, rank, k, -s_amp, s_amp, sigma, seed, tag, r_a1=r)
    d.update(r=r, k=k, q=q, tol=1e-7, max_iter=50, name=tag)
    return d


def config_c3(seed: int = 1309, frames: int = 1000, width: int = 320, height: int = 240) -> dict:
    """Video-shaped tall matrix: rows are pixels (i = y*width + x), columns frames.

    Background: three smooth cosine fields b_c in [0, 1/3] times slowly
    varying gains g_c(t) = 1 + 0.2 sin(2 pi t / T_c + phi_c).  Foreground:
    20 textured 24 x 24 blobs (values U[0.3, 1]) that translate 1-3 px per
    frame with integer velocities and reflect at the borders; a later blob
    overwrites an earlier one where they overlap; the blob value is added to
    the background.  Noise N(0, 1e-3^2).  r = 3, k = 1.2e6, q = 2.
    """
    m, n = width * height, frames
    p = uniform(seed, "c3/bg", (3, 6), 0.0, 1.0)
    ys, xs = np.divmod(np.arange(m), width)
    B = np.empty((m, 3))
    G = np.empty((n, 3))
    t = np.arange(n)
    for c in range(3):
        fx, fy = 0.2 + 1.3 * p[c, 0], 0.2 + 1.3 * p[c, 1]
        phi, psi = 2 * math.pi * p[c, 2], 2 * math.pi * p[c, 3]
        period = 200.0 + 800.0 * p[c, 4]
        B[:, c] = (0.5 + 0.5 * np.cos(2 * math.pi * (fx * xs / width + fy * ys / height) + phi)) / 3.0
        G[:, c] = 1.0 + 0.2 * np.sin(2 * math.pi * t / period + psi)
    X = B @ G.T
    S = np.zeros((m, n))
    nb, bs = 20, 24
    tex = uniform(seed, "c3/tex", (nb, bs, bs), 0.3, 1.0)
    st = uniform(seed, "c3/blobs", (nb, 4), 0.0, 1.0)
    for b in range(nb):
        x = int(st[b, 0] * (width - bs + 1))
        y = int(st[b, 1] * (height - bs + 1))
        speed = 1 + int(st[b, 2] * 3)                    # 1..3 px per frame
        ang = int(st[b, 3] * 8)                          # one of 8 directions
        vx = [1, 1, 0, -1, -1, -1, 0, 1][ang] * speed
        vy = [0, 1, 1, 1, 0, -1, -1, -1][ang] * speed
        for f in range(n):
            rows = ((y + np.arange(bs))[:, None] * width + (x + np.arange(bs))[None, :]).ravel()
            S[rows, f] = tex[b].ravel()
            x, vx = _reflect(x + vx, vx, width - bs)
            y, vy = _reflect(y + vy, vy, height - bs)
    X += S
    X += 1e-3 * gaussian(seed, "c3/G", (m, n))
    A1 = gaussian(seed, "c3/A1", (n, 3)).astype(np.float32)
    return {"X": X.astype(np.float32), "A1": A1, "B": B, "G": G, "S_dense_nnz": int((S != 0).sum()),
            "r": 3, "k": 1200000, "q": 2, "tol": 1e-7, "max_iter": 30,
            "name": f"c3_video_{m}x{n}_r3_q2"}


def _reflect(p: int, v: int, hi: int):
    if p < 0:
        return -p, -v
    if p > hi:
        return 2 * hi - p, -v
    return p, v


def config_c4(seed: int = 1309, count: int = 64) -> list[dict]:
    """64 independent matrices of uneven shape for the batched form (q = 1)."""
    u = uniform(seed, "c4/shape", (count, 4), 0.0, 1.0)
    out = []
    for i in range(count):
        m = int(round(math.exp(math.log(256) + u[i, 0] * (math.log(4096) - math.log(256)))))
        n = int(round(math.exp(math.log(256) + u[i, 1] * (math.log(4096) - math.log(256)))))
        r = 2 + int(u[i, 2] * 31)                        # U{2..32}
        rho = 0.02 + 0.03 * u[i, 3]
        k = int(round(rho * m * n))
        d = lowrank_sparse(m, n, r, k, -10.0, 10.0, 1e-3, seed, f"c4/{i}")
        d.update(r=r, k=k, q=1, tol=1e-7, max_iter=40, name=f"c4_{i}_{m}x{n}_r{r}")
        out.append(d)
    return out


def config_c5(seed: int = 1309) -> dict:
    """4096 x 4096 rank 20, 2 % sparse U[-10, 10], noise 1e-3; q = 0, T = 10,
    loss ||L_T - L*||_F^2 with L* = U* V*^T a seeded rank-20 target."""
    k = int(0.02 * 4096 * 4096)
    d = lowrank_sparse(4096, 4096, 20, k, -10.0, 10.0, 1e-3, seed, "c5")
    d["Ustar"] = gaussian(seed, "c5/Ustar", (4096, 20))
    d["Vstar"] = gaussian(seed, "c5/Vstar", (4096, 20))
    d.update(r=20, k=k, q=0, T=10, name="c5_4096x4096_r20_T10")
    return d
