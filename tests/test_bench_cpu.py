"""Host logic of bench.py that needs no GPU."""
import os

import bench

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
