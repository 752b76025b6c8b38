"""Host logic of bench.py that needs no GPU."""
import os

import bench
import pytest

CSRC = os.path.join(bench.ROOT, "paper_2602_23967_b300", "csrc")


def test_code_of_strips_comments_and_blank_lines():
    src = "int a = 1;  // one\n\n/* block\n   comment */ int b = 2;\n   // only a comment\nint c;\n"
    assert bench.code_of(src) == "int a = 1;\n int b = 2;\nint c;"


def _read(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def test_kernel_hash_follows_code_not_comments():
    base = bench.kernel_sources_sha256()
    assert bench.kernel_sources_sha256(_read) == base
    first = bench.KERNEL_SOURCES[0]

    def with_comment(name):
        text = _read(name)
        return text + "\n// a remark that changes no code\n" if name == first else text

    def with_code(name):
        text = _read(name)
        return text + "\nstatic const int kUnused = 1;\n" if name == first else text

    assert bench.kernel_sources_sha256(with_comment) == base
    assert bench.kernel_sources_sha256(with_code) != base


def test_job_throughput_counts_every_rank():
    # 2 ranks x 4096 instances x 5 steps in 10 s of the slowest rank
    assert bench.job_throughput(2, 4096, 5, 10_000.0) == 2 * 4096 * 5 / 10.0


def test_bench_fp64_kkt_equals_the_oracle_evaluator():
    # the benchmark's host-side KKT check (no oracle import in the timed legs)
    # computes the same residuals as the oracle's evaluator (Sec. 4.2)
    import numpy as np

    import bench
    import oracle
    from paper_2602_23967_b300 import workloads as W

    rng = np.random.default_rng(1)
    for qp in (W.random_qp(seed=2), W.mpc_qp(seed=3), W.lasso_qp(rows=200, cols=30, density=0.1, seed=4),
               W.factor_portfolio(n=500, k=10, seed=5)):
        x = rng.standard_normal(qp.n)
        y = rng.standard_normal(qp.m)
        Qx = qp.Q @ x if qp.Q is not None else np.zeros(qp.n)
        ref = oracle.kkt(qp.n, qp.m, x, y, qp.A @ x, qp.A.T @ y, Qx, qp.c, qp.lc, qp.uc, qp.lv, qp.uv)
        assert bench.fp64_kkt(qp, x, y) == pytest.approx(max(ref[:3]), rel=1e-12)
