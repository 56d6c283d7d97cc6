"""The benchmark's accounting, checked on the CPU: the algorithmic bytes of one iteration
(the measurement rule behind `iteration_roofline`) against the counts stated for the C2
workload, built up here term by term, and the whole-job throughput of N replicas."""
import bench


def test_iteration_bytes_c2():
    """C2 (10^4 x 10^4, r = 50, k = 10^6, q = 2): 6q+3 = 15 passes over the 400 MB matrix
    (6q+2 chain products with X A1 cached, one S-step pass), 6q+2 reads and one write of
    the 12-byte COO S, and the skinny operands in and out of the 15 products."""
    m = n = 10_000
    r, k, q = 50, 1_000_000, 2
    passes = 6 * q + 3
    matrix = passes * 4 * m * n                      # 6.0 GB
    sparse = (6 * q + 2) * 12 * k + 12 * k           # 0.18 GB
    skinny = passes * 2 * 4 * (m + n) * r            # 0.12 GB
    total = bench.iteration_bytes(m, n, r, k, q)
    assert total == matrix + sparse + skinny
    assert abs(total - 6.3e9) <= 0.01 * 6.3e9        # the 6.3 GB per iteration stated for C2


def test_iteration_bytes_scales_with_the_power_scheme():
    """Each extra power step q adds six passes over the matrix and six reads of S."""
    m, n, r, k = 3000, 2000, 10, 5000
    d = bench.iteration_bytes(m, n, r, k, 3) - bench.iteration_bytes(m, n, r, k, 2)
    assert d == 6 * 4 * m * n + 6 * 12 * k + 6 * 2 * 4 * (m + n) * r


def test_job_value_counts_every_replica_over_the_slowest_rank():
    assert bench.job_value(1, 30, 60.0) == 500.0
    assert bench.job_value(4, 30, 60.0) == 2000.0
