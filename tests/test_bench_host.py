"""Host-side accounting of bench.py that its roofline figures rest on: the
algorithmic bytes of the per-atom velocity correlator pushed one at a time
and in blocks (the blocked count must reduce to the per-push count for
blocks of one, and save exactly the re-read older samples otherwise)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


@pytest.fixture(scope="module")
def bench():
    import bench as b

    return b


def test_blocked_bytes_reduce_to_per_push(bench):
    for done, t_end in ((0, 40), (5, 1005), (17, 50)):
        per_push = sum(bench.vacf_bytes_per_push(t, 8, 16, 2, 1000, 4) for t in range(done + 1, t_end + 1))
        assert bench.vacf_bytes_blocked(done, t_end, 8, 16, 2, 1000, 4, block=1) == per_push


def test_blocked_bytes_save_the_older_reads(bench):
    # steady state (every block-0 lag formed): a push one at a time reads 15
    # older samples, a block of 8 reads them once
    done, t_end, ns, esz = 1000, 1000 + 8 * 50, 1000, 4
    per_push = sum(bench.vacf_bytes_per_push(t, 8, 16, 2, ns, esz) for t in range(done + 1, t_end + 1))
    blocked = bench.vacf_bytes_blocked(done, t_end, 8, 16, 2, ns, esz, block=8)
    blocks = (t_end - done) // 8
    assert per_push - blocked == blocks * (8 * 15 - 15) * ns * esz


def test_timed_bytes_count_whole_blocks(bench):
    class A:
        warmup, steps = 5, 1003

    # pushes 1..5 wait after the warm-up call; the timed call's passes apply
    # pushes 1..1008 (126 whole blocks) and leave 1009 and 1010 waiting
    got = bench.vacf_timed_bytes(A, 8, 16, 2, 100, pre=0)
    assert got == bench.vacf_bytes_blocked(0, 1008, 8, 16, 2, 300, 4, 8)

    class B:
        warmup, steps = 5, 20

    assert bench.vacf_timed_bytes(B, 8, 16, 2, 100, pre=0) == bench.vacf_bytes_blocked(0, 24, 8, 16, 2, 300, 4, 8)
    # after the bench's untimed fill of 256 steps the timed call of 20 steps
    # (warm-up 5) applies pushes 257 .. 280: blocks 33 to 35 in steady state
    assert bench.vacf_timed_bytes(B, 8, 16, 2, 100, pre=256) == bench.vacf_bytes_blocked(256, 280, 8, 16, 2, 300,
                                                                                           4, 8)
