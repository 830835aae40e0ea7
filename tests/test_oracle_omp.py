"""The multi-core CPU baseline (the oracle's step with its per-fish loops on
OpenMP threads, the parallelisation the paper studies in Sec. 2.3) against
the serial oracle: the same per-fish state and maxima bit for bit, and the
barycentre sums to rounding, whatever the thread count."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("swim_mode,feed_mode,init_mode", [(0, 0, 0), (1, 0, 1), (0, 1, 0),
                                                           (1, 1, 1)])
def test_openmp_run_equals_serial_run(precision, swim_mode, feed_mode, init_mode):
    cfg = oracle.Config(n_fish=2999, seed=11, school_id=5, swim_mode=swim_mode,
                        feed_mode=feed_mode, init_weight_mode=init_mode)
    start = oracle.init(cfg, precision)
    ref = start.copy()
    ref_stats = oracle.run(cfg, ref, 3, 30)
    for threads in (1, 2, 4, 7):
        got = start.copy()
        stats = oracle.run_omp(cfg, got, 3, 30, threads=threads)
        assert got.tobytes() == ref.tobytes()
        for k in ("max_abs_delta", "eat_max_diff"):
            assert np.array_equal(stats[k], ref_stats[k])
        # both sides are compensated binary64 sums of exact products
        assert np.all(np.abs(stats["sum_w"] - ref_stats["sum_w"]) <= 1e-15 * ref_stats["sum_w"])
        for s, a in (("sum_wx", "sum_abs_wx"), ("sum_wy", "sum_abs_wy")):
            assert np.all(np.abs(stats[s] - ref_stats[s]) <= 1e-15 * ref_stats[a])


def test_openmp_run_splits_like_one_run():
    cfg = oracle.Config(n_fish=513, seed=3)
    one = oracle.init(cfg, "f32")
    two = one.copy()
    oracle.run_omp(cfg, one, 0, 12, threads=3)
    oracle.run_omp(cfg, two, 0, 5, threads=3)
    oracle.run_omp(cfg, two, 5, 7, threads=3)
    assert one.tobytes() == two.tobytes()


def test_openmp_run_refuses_the_collective_movements():
    cfg = oracle.Config(n_fish=64, seed=1, collective_mode=1)
    school = oracle.init(cfg, "f32")
    with pytest.raises(ValueError):
        oracle.run_omp(cfg, school, 0, 1)


def test_bench_multicore_baseline_reports_its_threads():
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    rate, seconds, steps, threads = bench.cpu_openmp_rate(4096, 2, seconds=0.2)
    assert rate > 0 and seconds > 0 and steps >= 1
    assert threads == len(os.sched_getaffinity(0))
    host = bench.host_cpu()
    assert host["usable"] == threads and host["nproc"] >= threads and host["model"]
