"""GPU parity of the resident (on-chip) single-school path against the CPU
oracle, its grid-barrier failure detection, and the N = 2^20, T = 1000
school the resident kernel is built for."""
import numpy as np
import pytest

import oracle
import paper_2507_20173_gb300 as fsb
from fsb_testutil import (BARY_TOL, assert_state_equal, assert_stats_match, oracle_config)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def resident_cfg(n, seed, **kw):
    return fsb.fsb_config_init(n, seed, path=fsb.FSB_PATH_RESIDENT, **kw)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_20173_gb300 import build
    build.build()
    fsb.lib()


def run_pair(cfg, steps, calls=None):
    school = fsb.School.create(cfg)
    assert fsb.fsb_handle_path(school.handle) == fsb.FSB_PATH_RESIDENT
    calls = calls or [steps]
    stats = np.concatenate([school.step(n, stats=True) for n in calls])
    got = school.read()
    school.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run(ocfg, ref, 0, steps)
    return got, stats, ref, ref_stats


@pytest.mark.parametrize("precision", [fsb.FSB_FP32, fsb.FSB_FP32_KAHAN, fsb.FSB_FP64_ACC])
def test_small_school_every_step(precision):
    cfg = resident_cfg(10_000, 0, precision=precision)
    got, stats, ref, ref_stats = run_pair(cfg, 100)
    assert_state_equal(got, ref, "resident N=10000")
    assert_stats_match(stats, ref_stats, precision, "resident N=10000")


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 1023, 1024, 1025, 4095, 4096, 4097,
                               8191, 8193, 65537, 300_001])
def test_ragged_sizes_and_grid_shapes(n):
    """Sizes that give one block, several blocks, partial warps and partial
    fish-per-thread slots."""
    cfg = resident_cfg(n, 7 + n, school_id=11, step=3.0, init_weight_mode=1)
    steps = 6 if n > 100_000 else 11
    got, stats, ref, ref_stats = run_pair(cfg, steps)
    assert_state_equal(got, ref, "resident N=%d" % n)
    assert_stats_match(stats, ref_stats, cfg.precision, "resident N=%d" % n)


def test_split_calls_and_resume_across_paths():
    """Calls of different length equal one call, and a school advanced on
    the resident path resumes bit-exactly on the streaming path."""
    cfg = resident_cfg(20_000, 3)
    got, stats, ref, ref_stats = run_pair(cfg, 12, calls=[1, 4, 7])
    assert_state_equal(got, ref, "resident split")
    assert_stats_match(stats, ref_stats, cfg.precision, "resident split")
    scfg = fsb.fsb_config_init(20_000, 3, path=fsb.FSB_PATH_STREAM)
    b = fsb.School.create(scfg, init={"x": got["x"], "y": got["y"], "w": got["w"],
                                      "prev_objective": got["prev"]}, start_step=12)
    b.step(5)
    end = b.read()
    b.destroy()
    oracle.run(oracle_config(cfg), ref, 12, 5)
    assert_state_equal(end, ref, "resident -> stream resume")


def test_runs_are_deterministic():
    cfg = resident_cfg(200_000, 9)
    outs = []
    for _ in range(2):
        s = fsb.School.create(cfg)
        outs.append((s.step(20, stats=True), s.read()))
        s.destroy()
    assert np.array_equal(outs[0][0], outs[1][0])
    for k in ("x", "y", "w", "prev"):
        assert np.array_equal(outs[0][1][k], outs[1][1][k])


def test_fp64_state_is_not_resident():
    cfg = resident_cfg(1000, 1, precision=fsb.FSB_FP64_STATE)
    with pytest.raises(fsb.FsbError) as e:
        fsb.School.create(cfg)
    assert e.value.status == fsb.FSB_ERR_UNSUPPORTED


def test_auto_path_picks_resident_for_small_binary32_schools():
    s = fsb.School.create(fsb.fsb_config_init(100_000, 1))
    assert fsb.fsb_handle_path(s.handle) == fsb.FSB_PATH_RESIDENT
    s.destroy()
    s = fsb.School.create(fsb.fsb_config_init(1 << 24, 1))
    assert fsb.fsb_handle_path(s.handle) == fsb.FSB_PATH_STREAM
    s.destroy()


@pytest.mark.parametrize("n,block", [(1000, 32), (10_000, 32), (30_000, 64), (60_000, 128),
                                     (100_000, 192), (1 << 20, 512)])
def test_default_block_spreads_small_schools_over_the_sms(n, block):
    """A school that fits at four fish per thread takes the smallest block
    (a multiple of 32 fish threads) that puts it on at most one block per SM;
    a larger one keeps a pair for every thread of 512."""
    s = fsb.School.create(fsb.fsb_config_init(n, 1))
    t = fsb.fsb_get_tuning(s.handle)
    s.destroy()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if sms != 152:
        pytest.skip("block table measured for 152 SMs")
    assert t["resident_block"] == block
    assert t["resident_fpt"] == (4 if n <= 152 * 2048 else 16)


def test_missing_barrier_arrival_times_out_without_hanging():
    """Failure detection without a GPU fault: one block withholds its
    arrival at a grid barrier (set from the host).  Every bounded wait runs
    out after 50 ms, the call reports FSB_ERR_TIMEOUT, the state is the state
    before the call, and the context stays usable."""
    cfg = resident_cfg(300_000, 4)
    s = fsb.School.create(cfg)
    s.step(3)
    before = s.read()
    fsb.fsb_set_fault_injection(s.handle, 1, 2, 50_000_000)
    with pytest.raises(fsb.FsbError) as e:
        s.step(5, stats=True)
    assert e.value.status == fsb.FSB_ERR_TIMEOUT
    # the state was not written back by the failed call
    x = np.empty(cfg.n_fish, np.float32)
    with pytest.raises(fsb.FsbError):
        fsb.fsb_read_state(s.handle, x)          # the latched status is reported
    assert np.array_equal(x, before["x"])
    s.destroy()
    # the device still works
    t = torch.ones(1000, device="cuda")
    assert float(t.sum().item()) == 1000.0
    ok = fsb.School.create(fsb.fsb_config_init(5000, 1, path=fsb.FSB_PATH_RESIDENT))
    ok.step(2)
    ok.destroy()


def test_resident_school_2p20_t1000():
    """N = 2^20, seed 1, T = 1000 in the launch configuration the resident
    benchmark runs: full state against the oracle at T = 100, then sampled
    fish followed one by one to T = 1000, and the last step's max and sums
    against the whole read-back state."""
    n, seed = 1 << 20, 1
    cfg = fsb.fsb_config_init(n, seed)
    s = fsb.School.create(cfg)
    assert fsb.fsb_handle_path(s.handle) == fsb.FSB_PATH_RESIDENT
    start = s.read()
    st100 = s.step(100, stats=True)
    mid = s.read()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run(ocfg, ref, 0, 100)
    assert_state_equal(mid, ref, "2^20 T=100")
    assert_stats_match(st100, ref_stats, cfg.precision, "2^20 T=100")
    st900 = s.step(900, stats=True)
    got = s.read()
    s.destroy()
    assert got["step"] == 1000
    M = np.concatenate([st100["max_abs_delta"], st900["max_abs_delta"]])
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[0, 1, n - 2, n - 1], rng.integers(0, n, 3000)]))
    for i in idx:
        fish = np.zeros(1, oracle.FISH_F32)
        fish["x"], fish["y"] = start["x"][i], start["y"][i]
        fish["weight"] = start["w"][i]
        fish["prevObjective"] = start["prev"][i]
        fish["currentObjective"] = start["cur"][i]
        xs, ys, ds, fish = oracle.track_fish(ocfg, int(i), 0, 1000, fish)
        assert xs[-1] == got["x"][i] and ys[-1] == got["y"][i], i
        assert fish["prevObjective"][0] == got["prev"][i], i
        assert np.all(np.abs(ds) <= M), i
        ws = oracle.eat_fish(ocfg, float(start["w"][i]), ds, M)
        assert ws[-1] == got["w"][i], i
    assert st900["max_abs_delta"][-1] == np.max(np.abs(got["cur"] - got["prev"]))
    w64 = got["w"].astype(np.float64)
    x64 = got["x"].astype(np.float64)
    assert abs(st900["sum_wx"][-1] - np.sum(w64 * x64)) / np.sum(w64 * np.abs(x64)) \
        <= BARY_TOL[cfg.precision]


def test_resident_school_2p20_t1000_every_step():
    """N = 2^20, seed 1, T = 1000 in the launch configuration the resident
    benchmark runs, against the whole school advanced by the oracle's step on
    every host core (run_omp, pinned equal to run bit for bit): every step's
    max|delta| and eat() value exactly, every step's barycentre sums within
    the mode's tolerance, and every fish's final state bit for bit."""
    n, seed, steps = 1 << 20, 1, 1000
    cfg = fsb.fsb_config_init(n, seed)
    s = fsb.School.create(cfg)
    assert fsb.fsb_handle_path(s.handle) == fsb.FSB_PATH_RESIDENT
    stats = s.step(steps, stats=True)
    got = s.read()
    s.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run_omp(ocfg, ref, 0, steps)
    assert_stats_match(stats, ref_stats, cfg.precision, "2^20 every step")
    assert_state_equal(got, ref, "2^20 T=1000")
