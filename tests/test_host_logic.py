"""Host logic of the library, checked on the CPU (no device work): the stream-K geometry
that sizes the product's partial-slot and completion buffers, against a brute-force
walk of the CTA ranges, and the batched form's budget rule, against its definition."""
import math

import numpy as np
import pytest

import paper_1309_0302_gb300 as G

SHAPES = [(1, 1), (128, 64), (129, 65), (10000, 10000), (10000, 1000), (76800, 1000), (1000, 76800),
          (256, 4096), (4096, 257), (333, 12345), (5, 100000)]


@pytest.mark.parametrize("nsm", [1, 4, 16, 17, 40, 152])
def test_tc_geometry_against_brute_force(nsm):
    for rows, K in SHAPES:
        g = G.tc_geometry(rows, K, nsm)
        tiles, ks = math.ceil(rows / 128), math.ceil(K / 64)
        S = tiles * ks
        ncta = nsm - 4 if nsm > 16 else nsm
        assert (g["tiles"], g["ks"], g["S"], g["G"]) == (tiles, ks, S, min(S, ncta))
        Gc = g["G"]
        lo = [c * S // Gc for c in range(Gc)]
        hi = [(c + 1) * S // Gc for c in range(Gc)]
        assert lo[0] == 0 and hi[-1] == S and all(hi[c] == lo[c + 1] for c in range(Gc - 1))
        # the kernel's owner of stage s: ((s + 1) G - 1) / S
        owner = np.repeat(np.arange(Gc), np.diff(np.r_[lo, S]))
        s_all = np.arange(S, dtype=np.int64)
        assert np.array_equal(((s_all + 1) * Gc - 1) // S, owner)
        # CTAs sharing each tile (partial slots) and tiles each CTA touches (completions owed)
        per_tile = [len(set(owner[t * ks:(t + 1) * ks])) for t in range(tiles)]
        per_cta = [((hi[c] - 1) // ks - lo[c] // ks + 1) if hi[c] > lo[c] else 0 for c in range(Gc)]
        assert max(per_tile) == g["maxseg"], (rows, K, nsm)
        assert max(per_cta) <= g["maxpend"], (rows, K, nsm)


def test_tc_geometry_rejects_bad_arguments():
    for args in [(0, 10, 4), (10, 0, 4), (10, 10, 0)]:
        with pytest.raises(G.GodecError):
            G.tc_geometry(*args)


def test_batch_budget_rule():
    g = np.random.default_rng(3)
    shapes = [(int(round(math.exp(math.log(256) + u * math.log(16)))),
               int(round(math.exp(math.log(256) + v * math.log(16))))) for u, v in g.uniform(size=(64, 2))]
    W = sum(m * n for m, n in shapes)
    prev = None
    for k in range(5):
        b = G.batch_budgets(shapes, 152, k)
        if k == 0:
            assert b == [152] * 64
            continue
        want = [max(4, min(152, math.ceil(2 ** (k - 1) * 152 * m * n / W))) for m, n in shapes]
        assert b == want
        if prev is not None:
            assert all(x >= y for x, y in zip(b, prev))      # more oversubscription, more SMs
        prev = b
    assert G.batch_budgets([(300, 300)], 2, 1) == [2]         # never more than the device has
    with pytest.raises(G.GodecError):
        G.batch_budgets(shapes, 152, 5)
