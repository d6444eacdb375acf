"""Host-side logic of bench.py that needs no GPU."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_bench_fed_cycle_length_matches_the_oracle():
    """bench.py counts the explicit steps of the FED detection from the
    level times with its own cycle-length rule; it must agree with the
    oracle's cycle (Eq. 5) for every level gap of the workload."""
    import oracle
    import bench
    s0 = 1.6
    t = [0.5 * (s0 * 2.0 ** (i / 4)) ** 2 for i in range(16)]
    for a, b in zip(t, t[1:]):
        assert bench.fed_cycle_length(b - a) == len(oracle.fed_tau(b - a))
    assert sum(bench.fed_cycle_length(b - a) for a, b in zip(t, t[1:])) == 166
