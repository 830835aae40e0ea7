"""GPU parity of the two model variants against the CPU oracle:
swim_mode 1 (the move's half-width scales with the fish's weight, a reading
of the paper's weight-dependent movement) and feed_mode 1 (feeding normalised by
the paper's eat() value max(prev - cur)), on every path that runs them."""
import numpy as np
import pytest

import oracle
import paper_2507_20173_gb300 as fsb
from fsb_testutil import assert_state_equal, assert_stats_match, oracle_config, oracle_precision
from test_gpu_batch import check_batch, make_state, read_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = [(1, 0), (0, 1), (1, 1)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_20173_gb300 import build
    build.build()
    fsb.lib()


def run_and_compare(cfg, steps, tuning=None, calls=None):
    school = fsb.School.create(cfg)
    if tuning:
        fsb.fsb_set_tuning(school.handle, **tuning)
    calls = calls or [steps]
    stats = np.concatenate([school.step(n, stats=True) for n in calls])
    got = school.read()
    path = fsb.fsb_handle_path(school.handle)
    school.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg, oracle_precision(cfg))
    ref_stats = oracle.run(ocfg, ref, 0, steps)
    assert_state_equal(got, ref, "modes %d/%d" % (cfg.swim_mode, cfg.feed_mode))
    assert_stats_match(stats, ref_stats, cfg.precision, "modes %d/%d" % (cfg.swim_mode,
                                                                         cfg.feed_mode))
    return path


@pytest.mark.parametrize("swim_mode,feed_mode", MODES)
@pytest.mark.parametrize("kernel,block", [(1, 256), (2, 512), (2, 256), (3, 512)])
@pytest.mark.parametrize("n", [7, 4099, 100_003])
def test_streaming_variants(swim_mode, feed_mode, kernel, block, n):
    cfg = fsb.fsb_config_init(n, 77 + n, path=fsb.FSB_PATH_STREAM, swim_mode=swim_mode,
                              feed_mode=feed_mode, init_weight_mode=1, step=3.0)
    run_and_compare(cfg, 9, tuning={"stream_kernel": kernel, "stream_block": block},
                    calls=[4, 5])


@pytest.mark.parametrize("swim_mode,feed_mode", MODES)
def test_binary64_state_variants(swim_mode, feed_mode):
    cfg = fsb.fsb_config_init(20_001, 5, precision=fsb.FSB_FP64_STATE, swim_mode=swim_mode,
                              feed_mode=feed_mode, init_weight_mode=1, step=2.0)
    run_and_compare(cfg, 11)


@pytest.mark.parametrize("swim_mode,feed_mode", MODES)
@pytest.mark.parametrize("n", [5000, 300_001])
def test_resident_variants(swim_mode, feed_mode, n):
    """The resident kernel runs both variants; with the weight-scaled swim it
    swims each step after the previous step's eat instead of beside the grid
    barrier."""
    cfg = fsb.fsb_config_init(n, 3, path=fsb.FSB_PATH_RESIDENT, swim_mode=swim_mode,
                              feed_mode=feed_mode, init_weight_mode=1, step=2.0)
    assert run_and_compare(cfg, 13, calls=[6, 7]) == fsb.FSB_PATH_RESIDENT


@pytest.mark.parametrize("fpt", [4, 8, 12, 16])
def test_resident_weighted_swim_every_fish_per_thread(fpt):
    cfg = fsb.fsb_config_init(200_000, 11, path=fsb.FSB_PATH_RESIDENT, swim_mode=1,
                              init_weight_mode=1, step=3.0)
    assert run_and_compare(cfg, 9, tuning={"resident_fpt": fpt},
                           calls=[4, 5]) == fsb.FSB_PATH_RESIDENT


@pytest.mark.parametrize("swim_mode,feed_mode", MODES)
def test_batch_variants(swim_mode, feed_mode):
    sizes = np.array([1, 31, 600, 8193, 20000, 4096, 65536], dtype=np.uint64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    seeds = (500 + np.arange(sizes.size)).astype(np.uint64)
    tmpl = fsb.fsb_config_init(1, 0, swim_mode=swim_mode, feed_mode=feed_mode,
                               init_weight_mode=1, step=2.5)
    ts, state = make_state(offsets[-1])
    steps = 7
    stats = np.zeros(sizes.size * steps, fsb.STATS_DTYPE)
    fsb.fsb_run_batch(tmpl, offsets, seeds, state, steps, init=True, stats=stats)
    check_batch(tmpl, offsets, seeds, read_state(ts), stats, steps, tmpl.precision)


@pytest.mark.parametrize("swim_mode,feed_mode", MODES)
def test_allocation_free_step_variants(swim_mode, feed_mode):
    n = 30_011
    cfg = fsb.fsb_config_init(n, 21, swim_mode=swim_mode, feed_mode=feed_mode, init_weight_mode=1,
                              step=2.0)
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    mine = [torch.from_numpy(np.ascontiguousarray(ref[f])).cuda()
            for f in ("x", "y", "weight", "prevObjective")]
    state = fsb.FsbStateDev(*(t.data_ptr() for t in mine))
    stats = np.zeros(8, fsb.STATS_DTYPE)
    fsb.fsb_step_static(cfg, state, 0, 8, stats, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref_stats = oracle.run(ocfg, ref, 0, 8)
    got = {k: t.cpu().numpy() for k, t in zip(("x", "y", "w", "prev"), mine)}
    got["cur"] = np.sqrt(got["x"] * got["x"] + got["y"] * got["y"])
    assert_state_equal(got, ref, "static variants")
    assert_stats_match(stats, ref_stats, cfg.precision, "static variants")
