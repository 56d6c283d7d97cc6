"""Plain CPU float64 oracle for GoDec by bilateral random projection.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never calls into it and it shares no code with the CUDA
library: the only common module is ``synth`` (seeded inputs).

Everything here is numpy in float64, written step by step from the paper
(Zhou & Tao, "Unmixing Incoherent Structures of Big Data by Randomized or
Greedy Decomposition", arXiv:1309.0302): Algorithm 1 (GoDec by BRP), eq.
(lr_app) and eq. (mlr_app) of Sec. 3.1, the entry-wise hard threshold of eq.
(raw_lss), and the objective of eq. (ls_app).  Library primitives used as
single steps: matrix product, Householder QR, SVD, solve, partition.
``oracle.grebsmo`` holds GreBsmo (Sec. 3.2.1, Algorithm 2), ``oracle.lingodec`` LinGoDec
(Sec. 4.3) and ``oracle.mse`` MSE training (Sec. 4.2.1, Algorithm 4), the same way.
"""
from .godec import (  # noqa: F401
    ltilde_times, ltilde_t_times, numerical_rank, brp_literal, brp_stable,
    hard_threshold, godec, godec_step, naive_godec, tangent_refine,
    unrolled_forward, unrolled_vjp, unrolled_jvp, unrolled_loss, dense_L,
    RANK_TOL,
)
