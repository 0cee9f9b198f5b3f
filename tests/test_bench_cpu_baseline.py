"""The all-cores oracle baseline of bench.py: one spawned process per host
core, each one coarse step of its own copy of the workload; the rate counts the
cell updates of all of them over the longest step."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_all_cores_rate_counts_every_process():
    sys.path.insert(0, ROOT)
    import bench
    rate, cores, t = bench.cpu_oracle_rate_all_cores(32, 16)
    assert cores == len(os.sched_getaffinity(0))
    assert t > 0.0
    # each process advances the 32^3 cells once: the rate is their sum over the longest step
    assert abs(rate * t - cores * 32 ** 3) <= 1e-6 * cores * 32 ** 3
