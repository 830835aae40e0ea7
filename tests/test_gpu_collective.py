"""GPU parity of the collective movements (fish-school search variant,
collective_mode 1) against the CPU oracle: the whole per-fish state bit for
bit, the maxima exactly and the barycentre sums within the mode's tolerance.
The school sums that feed back into positions are exact fixed-point sums on
both sides, so no reduction order can move a fish."""
import numpy as np
import pytest

import oracle
import paper_2507_20173_gb300 as fsb
from fsb_testutil import assert_state_equal, assert_stats_match, oracle_config, oracle_precision

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_20173_gb300 import build
    build.build()
    fsb.lib()


def coll_cfg(n, seed, **kw):
    base = dict(collective_mode=1, step_vol=0.3, step=2.0, init_weight_mode=1)
    base.update(kw)
    return fsb.fsb_config_init(n, seed, **base)


def run_pair(cfg, steps, calls=None, timing=False):
    school = fsb.School.create(cfg)
    if timing:
        fsb.fsb_set_kernel_timing(school.handle, True)
    calls = calls or [steps]
    stats = np.concatenate([school.step(c, stats=True) for c in calls])
    got = school.read()
    assert fsb.fsb_handle_path(school.handle) == fsb.FSB_PATH_STREAM
    school.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg, oracle_precision(cfg))
    ref_stats = oracle.run(ocfg, ref, 0, steps)
    return got, stats, ref, ref_stats


@pytest.mark.parametrize("n", [1, 2, 3, 64, 777, 4099, 100_003])
def test_collective_school_matches_the_oracle(n):
    cfg = coll_cfg(n, 40 + n)
    got, stats, ref, ref_stats = run_pair(cfg, 7)
    assert_state_equal(got, ref, "collective n=%d" % n)
    assert_stats_match(stats, ref_stats, cfg.precision, "collective n=%d" % n)


@pytest.mark.parametrize("precision", [fsb.FSB_FP32, fsb.FSB_FP32_KAHAN, fsb.FSB_FP64_ACC,
                                       fsb.FSB_FP64_STATE])
def test_collective_every_precision(precision):
    cfg = coll_cfg(20_001, 5, precision=precision)
    got, stats, ref, ref_stats = run_pair(cfg, 6, calls=[2, 4])
    assert_state_equal(got, ref, "collective precision %d" % precision)
    assert_stats_match(stats, ref_stats, precision, "collective precision %d" % precision)


@pytest.mark.parametrize("swim_mode,feed_mode", [(1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("step_vol", [0.0, 1.5])
def test_collective_with_the_other_variants(swim_mode, feed_mode, step_vol):
    cfg = coll_cfg(9_999, 8, swim_mode=swim_mode, feed_mode=feed_mode, step_vol=step_vol)
    got, stats, ref, ref_stats = run_pair(cfg, 5)
    assert_state_equal(got, ref, "collective modes %d/%d" % (swim_mode, feed_mode))
    assert_stats_match(stats, ref_stats, cfg.precision, "collective")


def test_collective_many_blocks_and_split_calls():
    """A million fish over hundreds of blocks: every block's exact partial
    folds to the oracle's sums, across calls of 1, 3 and 2 steps."""
    cfg = coll_cfg(1_000_003, 77, step_vol=0.5)
    got, stats, ref, ref_stats = run_pair(cfg, 6, calls=[1, 3, 2])
    assert_state_equal(got, ref, "collective 1e6")
    assert_stats_match(stats, ref_stats, cfg.precision, "collective 1e6")


def test_collective_timed_and_long_calls():
    """The timed path (each step's two passes bracketed by events) and a call
    longer than one captured graph give the same trajectory."""
    cfg = coll_cfg(3_001, 12)
    got, stats, ref, ref_stats = run_pair(cfg, 4, timing=True)
    assert_state_equal(got, ref, "collective timed")
    cfg = coll_cfg(257, 13, step=0.5)
    got, stats, ref, ref_stats = run_pair(cfg, 2100)     # beyond one whole-call graph
    assert_state_equal(got, ref, "collective 2100 steps")
    assert_stats_match(stats, ref_stats, cfg.precision, "collective 2100 steps")


def test_collective_refused_where_it_does_not_run():
    cfg = coll_cfg(5000, 1, path=fsb.FSB_PATH_RESIDENT)
    with pytest.raises(fsb.FsbError) as e:
        fsb.School.create(cfg)
    assert e.value.status == fsb.FSB_ERR_UNSUPPORTED
    tmpl = coll_cfg(1, 0)
    ts = [torch.zeros(100, device="cuda") for _ in range(4)]
    state = fsb.FsbStateDev(*(t.data_ptr() for t in ts))
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_run_batch(tmpl, np.array([0, 50, 100], np.uint64), np.array([1, 2], np.uint64),
                          state, 2, init=True)
    assert e.value.status == fsb.FSB_ERR_UNSUPPORTED
    stats = np.zeros(2, fsb.STATS_DTYPE)
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_step_static(coll_cfg(100, 1), state, 0, 2, stats,
                            torch.cuda.current_stream().cuda_stream)
    assert e.value.status == fsb.FSB_ERR_UNSUPPORTED
    s = fsb.School.create(coll_cfg(5000, 1))
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_set_fault_injection(s.handle, 0, 1, 0)
    assert e.value.status == fsb.FSB_ERR_UNSUPPORTED
    s.destroy()
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_autotune(coll_cfg(5000, 1), 3)
    assert e.value.status == fsb.FSB_ERR_UNSUPPORTED
