"""GPU parity of stream kernels 4 and 5, the streaming step blocked over k
steps (a maxima pass swims the next k steps from the state to find their
max |delta| and eat() values, then a step pass eats and swims them again --
kernel 5 loads the positions the maxima pass kept instead): the per-fish
state bit for bit and both maxima exactly against the oracle, the
barycentre sums within the mode's tolerance, and at the benchmark's size the
same bits as the one-pass-per-step kernel."""
import numpy as np
import pytest

import oracle
import paper_2507_20173_gb300 as fsb
from fsb_testutil import assert_state_equal, assert_stats_match, oracle_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_20173_gb300 import build
    build.build()
    fsb.lib()


def blocked_school(cfg, k, kernel=4):
    s = fsb.School.create(cfg)
    fsb.fsb_set_tuning(s.handle, stream_kernel=kernel, stream_block_steps=k)
    t = fsb.fsb_get_tuning(s.handle)
    assert (t["stream_kernel"], t["stream_block_steps"]) == (kernel, k)
    return s


def run_pair(cfg, k, calls, kernel=4):
    s = blocked_school(cfg, k, kernel)
    stats = np.concatenate([s.step(c, stats=True) for c in calls])
    got = s.read()
    s.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run(ocfg, ref, 0, sum(calls))
    return got, stats, ref, ref_stats


@pytest.mark.parametrize("kernel", [4, 5])
@pytest.mark.parametrize("k", [2, 4, 8])
@pytest.mark.parametrize("steps", [1, 2, 5, 9])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 33, 4097, 100_003, 1_000_003])
def test_blocked_school_matches_the_oracle(n, steps, k, kernel):
    """Whole and partial pairs (steps - 1 not a multiple of k), ragged tails
    (n % 4), schools smaller than one group, grids of one block and many."""
    cfg = fsb.fsb_config_init(n, 900 + n, path=fsb.FSB_PATH_STREAM, step=1.5,
                              init_weight_mode=1, school_id=3)
    got, stats, ref, ref_stats = run_pair(cfg, k, [steps], kernel)
    where = "blocked kernel %d k=%d n=%d T=%d" % (kernel, k, n, steps)
    assert_state_equal(got, ref, where)
    assert_stats_match(stats, ref_stats, cfg.precision, where)


@pytest.mark.parametrize("kernel", [4, 5])
@pytest.mark.parametrize("precision", [fsb.FSB_FP32, fsb.FSB_FP32_KAHAN, fsb.FSB_FP64_ACC])
@pytest.mark.parametrize("feed_mode", [0, 1])
def test_blocked_every_binary32_mode_and_paper_feeding(precision, feed_mode, kernel):
    cfg = fsb.fsb_config_init(50_001, 17, path=fsb.FSB_PATH_STREAM, precision=precision,
                              feed_mode=feed_mode, init_weight_mode=1)
    got, stats, ref, ref_stats = run_pair(cfg, 4, [3, 10, 1], kernel)
    where = "blocked kernel %d precision %d feed %d" % (kernel, precision, feed_mode)
    assert_state_equal(got, ref, where)
    assert_stats_match(stats, ref_stats, precision, where)


@pytest.mark.parametrize("kernel", [4, 5])
def test_blocked_timed_and_long_calls(kernel):
    """The timed path brackets each pair of passes with events (one unit per
    pair), and a call longer than one captured graph launches the pairs
    directly; both give the oracle's trajectory."""
    cfg = fsb.fsb_config_init(3001, 5, path=fsb.FSB_PATH_STREAM)
    s = blocked_school(cfg, 4, kernel)
    fsb.fsb_set_kernel_timing(s.handle, True)
    stats = s.step(10, stats=True)
    ms, launches = fsb.fsb_kernel_time(s.handle)
    assert launches == 3 and ms > 0.0      # pairs of 4, 4 and 1 steps
    fsb.fsb_set_kernel_timing(s.handle, False)
    stats = np.concatenate([stats, s.step(2100, stats=True)])
    got = s.read()
    s.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run(ocfg, ref, 0, 2110)
    assert_state_equal(got, ref, "blocked long call")
    assert_stats_match(stats, ref_stats, cfg.precision, "blocked long call")


@pytest.mark.parametrize("kernel", [4, 5])
def test_blocked_resume_from_checkpoint(kernel):
    cfg = fsb.fsb_config_init(10_007, 8, path=fsb.FSB_PATH_STREAM)
    s = blocked_school(cfg, 8, kernel)
    s.step(6)
    mid = s.read()
    s.destroy()
    init = {"x": mid["x"], "y": mid["y"], "w": mid["w"], "prev_objective": mid["prev"]}
    r = fsb.School.create(cfg, init=init, start_step=6)
    fsb.fsb_set_tuning(r.handle, stream_kernel=kernel, stream_block_steps=8)
    stats = r.step(11, stats=True)
    got = r.read()
    r.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    oracle.run(ocfg, ref, 0, 6)
    ref_stats = oracle.run(ocfg, ref, 6, 11)
    assert_state_equal(got, ref, "blocked resume")
    assert_stats_match(stats, ref_stats, cfg.precision, "blocked resume")


@pytest.mark.parametrize("kernel", [4, 5])
@pytest.mark.parametrize("fields", [dict(precision=fsb.FSB_FP64_STATE), dict(swim_mode=1),
                                    dict(collective_mode=1)])
def test_blocked_refused_where_positions_or_state_do_not_allow_it(fields, kernel):
    """The blocked passes need binary32 state and positions that do not
    depend on weights (no weight-scaled swim, no collective movements)."""
    cfg = fsb.fsb_config_init(4096, 1, path=fsb.FSB_PATH_STREAM, **fields)
    s = fsb.School.create(cfg)
    before = fsb.fsb_get_tuning(s.handle)
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_set_tuning(s.handle, stream_kernel=kernel)
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    assert fsb.fsb_get_tuning(s.handle) == before
    s.destroy()


@pytest.mark.parametrize("kernel", [4, 5])
def test_blocked_swim_steps_the_scaled_move_allows(kernel):
    """The blocked passes form the move as v * (step * 2^-23), exact only for
    a step of 0 or of at least 2^-103: a still school (step 0) runs them and
    matches the oracle; a step between is refused (kernel 1 runs it)."""
    cfg = fsb.fsb_config_init(4099, 3, path=fsb.FSB_PATH_STREAM, step=0.0)
    got, stats, ref, ref_stats = run_pair(cfg, 4, [6], kernel)
    assert_state_equal(got, ref, "blocked, step 0")
    assert_stats_match(stats, ref_stats, cfg.precision, "blocked, step 0")
    tiny = fsb.School.create(fsb.fsb_config_init(4096, 1, path=fsb.FSB_PATH_STREAM, step=1e-35))
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_set_tuning(tiny.handle, stream_kernel=kernel)
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    tiny.destroy()


@pytest.mark.parametrize("kernel", [4, 5])
def test_blocked_needs_aligned_state_and_a_valid_block(kernel):
    n = 1000
    ts = [torch.zeros(n + 1, dtype=torch.float32, device="cuda")[1:] for _ in range(4)]
    cfg = fsb.fsb_config_init(n, 1, path=fsb.FSB_PATH_STREAM)
    h = fsb.fsb_create(cfg, fsb.FsbStateDev(*(t.data_ptr() for t in ts)), None, 0, None)
    with pytest.raises(fsb.FsbError):
        fsb.fsb_set_tuning(h, stream_kernel=kernel)
    fsb.fsb_destroy(h)
    s = fsb.School.create(cfg)
    for bad in (dict(stream_block_steps=3), dict(stream_block_steps=16),
                dict(stream_block=512)):
        with pytest.raises(fsb.FsbError) as e:
            fsb.fsb_set_tuning(s.handle, stream_kernel=kernel, **bad)
        assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    s.destroy()


def test_kernel5_switches_back_and_forth_and_reports_a_failed_allocation():
    """Kernel 5's position slots are kept across tunings (a larger k grows
    them); a school whose slots cannot be allocated keeps its tuning."""
    cfg = fsb.fsb_config_init(20_001, 4, path=fsb.FSB_PATH_STREAM)
    s = fsb.School.create(cfg)
    stats = [s.step(3, stats=True)]
    for kernel, k in ((5, 2), (4, 4), (5, 8), (1, 0), (5, 4)):
        fsb.fsb_set_tuning(s.handle, stream_kernel=kernel, stream_block_steps=k)
        stats.append(s.step(5, stats=True))
    got = s.read()
    s.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run(ocfg, ref, 0, 28)
    assert_state_equal(got, ref, "kernel 5 retuned")
    assert_stats_match(np.concatenate(stats), ref_stats, cfg.precision, "kernel 5 retuned")
    # leave about 6 GB: a school of 2^27 fish takes 2 GB, its slots for
    # k = 8 would take 8 GB
    free, _ = torch.cuda.mem_get_info()
    if free < 8 * (1 << 30):
        pytest.skip("needs 8 GB of free device memory")
    hog = torch.empty(free - 6 * (1 << 30), dtype=torch.uint8, device="cuda")
    s = fsb.School.create(fsb.fsb_config_init(1 << 27, 1, path=fsb.FSB_PATH_STREAM))
    before = fsb.fsb_get_tuning(s.handle)
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_set_tuning(s.handle, stream_kernel=5, stream_block_steps=8)
    assert e.value.status == fsb.FSB_ERR_OOM
    assert fsb.fsb_get_tuning(s.handle) == before
    s.step(2)                            # still runs on its old tuning
    s.destroy()
    del hog
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kernel,k", [(4, 4), (4, 8), (5, 4), (5, 8)])
def test_full_size_blocked_agrees_bitwise_with_one_pass_per_step(kernel, k):
    """N = 2^28, seed 2, T = 100 (the benchmark's school): the blocked
    passes leave the same bits in every fish as the vector-load kernel, with
    the same exact maxima, and barycentre sums equal within the tolerance."""
    n, steps, seed = 1 << 28, 100, 2
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 40 * (1 << 30):
        pytest.skip("needs ~40 GB of free device memory")
    out = []
    for kern in (kernel, 1):
        s = fsb.School.create(fsb.fsb_config_init(n, seed, path=fsb.FSB_PATH_STREAM))
        if kern != 1:
            fsb.fsb_set_tuning(s.handle, stream_kernel=kern, stream_block_steps=k)
        stats = s.step(steps, stats=True)
        state = [t.clone() for t in s.tensors]
        s.destroy()
        out.append((state, stats))
    (a, sa), (b, sb) = out
    for name, ta, tb in zip(("x", "y", "w", "prev"), a, b):
        bad = int((ta.view(torch.int32) != tb.view(torch.int32)).sum())
        assert bad == 0, "%s differs in %d fish" % (name, bad)
    assert np.array_equal(sa["max_abs_delta"], sb["max_abs_delta"])
    assert np.array_equal(sa["eat_max_diff"], sb["eat_max_diff"])
    # each within 1e-5 of its normaliser (sum w; sum |w x| <= 100 sum w)
    assert np.all(np.abs(sa["sum_w"] - sb["sum_w"]) <= 2e-5 * sb["sum_w"])
    for key in ("sum_wx", "sum_wy"):
        assert np.all(np.abs(sa[key] - sb[key]) <= 2e-5 * 100.0 * sb["sum_w"]), key


def test_library_choice_is_kernel5_for_large_streaming_schools():
    """The library's streaming kernel: 5 with 8 steps per pair for a school
    of at least 2^22 fish that allows it (binary32, default swim) when its
    slots (64 B per fish) take at most half of the free device memory;
    kernel 1 otherwise."""
    def chosen(n, **fields):
        s = fsb.School.create(fsb.fsb_config_init(n, 1, path=fsb.FSB_PATH_STREAM, **fields))
        t = fsb.fsb_get_tuning(s.handle)
        s.destroy()
        return t["stream_kernel"], t["stream_block_steps"]
    torch.cuda.empty_cache()
    assert chosen(1 << 22) == (5, 8)
    assert chosen((1 << 22) - 1)[0] == 1
    assert chosen(1 << 22, precision=fsb.FSB_FP64_STATE)[0] == 1
    assert chosen(1 << 22, swim_mode=1)[0] == 1
    assert chosen(1 << 22, step=1e-35)[0] == 1
    # set_tuning with every field 0 is the library's choice again
    s = fsb.School.create(fsb.fsb_config_init(1 << 22, 1, path=fsb.FSB_PATH_STREAM))
    fsb.fsb_set_tuning(s.handle, stream_kernel=1)
    fsb.fsb_set_tuning(s.handle)
    assert fsb.fsb_get_tuning(s.handle)["stream_kernel"] == 5
    s.destroy()
    # not enough free memory for the slots: kernel 1
    free, _ = torch.cuda.mem_get_info()
    if free < 8 * (1 << 30):
        pytest.skip("needs 8 GB of free device memory")
    hog = torch.empty(free - 6 * (1 << 30), dtype=torch.uint8, device="cuda")
    try:
        assert chosen(1 << 26)[0] == 1       # 1 GB of state, 4 GB of slots: > half of what is left
    finally:
        del hog
        torch.cuda.empty_cache()
