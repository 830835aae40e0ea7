"""GPU parity of the streaming path (C ABI) against the CPU oracle.

Per-fish state (x, y, weight, prevObjective, currentObjective) and max|delta|
must be bit-exact; the paper's eat() statistic max(prev - cur) too; the
barycentre sums within the tolerance of the arithmetic mode.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2507_20173_gb300 as fsb
from fsb_testutil import (BARY_TOL, assert_state_equal, assert_stats_match, bary_errors,
                          oracle_config, oracle_precision)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

def stream_cfg(n, seed, **kw):
    """Configuration pinned to the streaming path."""
    return fsb.fsb_config_init(n, seed, path=fsb.FSB_PATH_STREAM, **kw)


PRECISIONS = [fsb.FSB_FP32, fsb.FSB_FP32_KAHAN, fsb.FSB_FP64_ACC, fsb.FSB_FP64_STATE]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_20173_gb300 import build
    build.build()
    fsb.lib()


def run_pair(cfg, steps, calls=None):
    """GPU and oracle side by side; returns (gpu state, gpu stats, oracle
    school, oracle stats)."""
    school = fsb.School.create(cfg)
    calls = calls or [steps]
    stats = np.concatenate([school.step(n, stats=True) for n in calls])
    got = school.read()
    school.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg, oracle_precision(cfg))
    ref_stats = oracle.run(ocfg, ref, 0, steps)
    return got, stats, ref, ref_stats


@pytest.mark.parametrize("precision", [fsb.FSB_FP32_KAHAN, fsb.FSB_FP64_STATE])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 4095, 4096, 4097, 10000])
def test_init_matches_oracle(n, mode, precision):
    cfg = stream_cfg(n, 0xABCDEF0123 + n, init_weight_mode=mode,
                              precision=precision, school_id=n % 7)
    school = fsb.School.create(cfg)
    got = school.read()
    school.destroy()
    assert got["step"] == 0
    ref = oracle.init(oracle_config(cfg), oracle_precision(cfg))
    assert_state_equal(got, ref, "init N=%d" % n)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_small_school_every_step(precision):
    """N = 10,000, seed 0, T = 100: stats of every step and the final state."""
    cfg = stream_cfg(10_000, 0, precision=precision)
    got, stats, ref, ref_stats = run_pair(cfg, 100)
    assert_state_equal(got, ref, "N=10000 T=100")
    assert got["step"] == 100
    assert_stats_match(stats, ref_stats, precision, "N=10000")


def test_small_school_state_after_each_step():
    cfg = stream_cfg(10_000, 0)
    school = fsb.School.create(cfg)
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    for t in range(1, 21):
        school.step(1)
        ref_stats = oracle.run(ocfg, ref, t - 1, 1)
        got = school.read()
        assert_state_equal(got, ref, "step %d" % t)
        st = np.zeros(1, fsb.STATS_DTYPE)
        fsb.fsb_last_stats(school.handle, st, 1)
        assert_stats_match(st, ref_stats, cfg.precision, "step %d" % t)
    school.destroy()


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 32, 33, 511, 512, 513, 4095, 4096, 4097])
def test_ragged_sizes(n):
    cfg = stream_cfg(n, 99 + n, school_id=3, step=2.5)
    got, stats, ref, ref_stats = run_pair(cfg, 9)
    assert_state_equal(got, ref, "N=%d" % n)
    assert_stats_match(stats, ref_stats, cfg.precision, "N=%d" % n)


@pytest.mark.parametrize("precision", [fsb.FSB_FP32_KAHAN, fsb.FSB_FP64_STATE])
def test_unaligned_buffers_take_the_scalar_path(precision):
    """Buffers offset by one element are not 16-byte aligned, so the library
    runs its scalar kernel; results are the same."""
    n, steps = 1003, 12
    cfg = stream_cfg(n, 5, precision=precision)
    dt = torch.float64 if precision == fsb.FSB_FP64_STATE else torch.float32
    big = [torch.empty(n + 1, dtype=dt, device="cuda") for _ in range(4)]
    bufs = fsb.FsbStateDev(*(b[1:].data_ptr() for b in big))
    h = fsb.fsb_create(cfg, bufs, None, 0, torch.cuda.current_stream().cuda_stream)
    stats = np.zeros(steps, fsb.STATS_DTYPE)
    fsb.fsb_step(h, steps, stats)
    npdt = np.float64 if precision == fsb.FSB_FP64_STATE else np.float32
    got = {k: np.empty(n, npdt) for k in ("x", "y", "w", "prev", "cur")}
    fsb.fsb_read_state(h, got["x"], got["y"], got["w"], got["prev"], got["cur"])
    fsb.fsb_destroy(h)
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg, oracle_precision(cfg))
    ref_stats = oracle.run(ocfg, ref, 0, steps)
    assert_state_equal(got, ref, "unaligned")
    assert_stats_match(stats, ref_stats, precision, "unaligned")


# (kernel, block, blocks per SM, stages): vector loads with 1 / 3 / 4
# guaranteed blocks per SM, bulk-copy ring with 2 / 3 / 4 stages
VARIANTS = [(1, 256, 0, 0), (1, 256, 3, 0), (1, 256, 4, 0), (1, 512, 0, 0),
            (2, 256, 0, 2), (2, 256, 0, 3), (2, 256, 0, 4), (2, 512, 0, 2), (2, 512, 0, 4),
            (3, 256, 0, 2), (3, 256, 0, 3), (3, 512, 0, 2), (3, 512, 0, 3), (3, 512, 1, 2)]


@pytest.mark.parametrize("kernel,block,per_sm,stages", VARIANTS)
@pytest.mark.parametrize("n", [1, 33, 2047, 2048, 2049, 4096 * 3 + 5, 1_000_003])
def test_stream_kernel_variants(kernel, block, per_sm, stages, n):
    """Every launch shape of the streaming pass: whole tiles, a ragged tail,
    fewer tiles than blocks."""
    cfg = stream_cfg(n, 1234 + n, step=1.5, init_weight_mode=1)
    school = fsb.School.create(cfg)
    fsb.fsb_set_tuning(school.handle, stream_kernel=kernel, stream_block=block,
                       stream_blocks_per_sm=per_sm, stream_stages=stages)
    t = fsb.fsb_get_tuning(school.handle)
    assert (t["stream_kernel"], t["stream_block"]) == (kernel, block)
    stats = school.step(7, stats=True)
    got = school.read()
    school.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run(ocfg, ref, 0, 7)
    assert_state_equal(got, ref, "variant %d/%d N=%d" % (kernel, block, n))
    assert_stats_match(stats, ref_stats, cfg.precision, "variant %d/%d N=%d" % (kernel, block, n))


def test_autotuner_choice_reproduces_the_oracle():
    """The native autotuner measures every launch shape of both paths; the
    winner, applied to a new school, still gives the oracle's trajectory."""
    n, steps = 300_000, 6
    cfg = fsb.fsb_config_init(n, 5)
    r = fsb.fsb_autotune(cfg, 10)
    assert r["candidates"] >= 8 and r["fish_steps_per_s"] > 0
    run = fsb.fsb_config_init(n, 5, path=r["path"])
    s = fsb.School.create(run)
    fsb.fsb_set_tuning(s.handle, **r["tuning"])
    stats = s.step(steps, stats=True)
    got = s.read()
    s.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run(ocfg, ref, 0, steps)
    assert_state_equal(got, ref, "autotuned")
    assert_stats_match(stats, ref_stats, cfg.precision, "autotuned")


@pytest.mark.parametrize("kernel", [2, 3])
def test_bulk_copy_kernel_needs_binary32_aligned_state(kernel):
    s = fsb.School.create(stream_cfg(1000, 1, precision=fsb.FSB_FP64_STATE))
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_set_tuning(s.handle, stream_kernel=kernel)
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    assert fsb.fsb_get_tuning(s.handle)["stream_kernel"] == 1
    s.destroy()


def test_warp_specialised_ring_takes_two_or_three_stages():
    s = fsb.School.create(stream_cfg(5000, 1))
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_set_tuning(s.handle, stream_kernel=3, stream_stages=4)
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    fsb.fsb_set_tuning(s.handle, stream_kernel=3, stream_stages=3)
    t = fsb.fsb_get_tuning(s.handle)
    assert (t["stream_kernel"], t["stream_stages"]) == (3, 3)
    s.destroy()


def test_split_calls_equal_one_call():
    cfg = stream_cfg(3001, 17)
    got, stats, ref, ref_stats = run_pair(cfg, 10, calls=[3, 1, 6])
    assert_state_equal(got, ref, "split")
    assert_stats_match(stats, ref_stats, cfg.precision, "split")


def test_long_call_uses_chunked_graphs():
    """More steps than one captured graph holds (2048): chunk graphs plus
    direct launches must give the same trajectory."""
    cfg = stream_cfg(67, 23, step=1.0)
    got, stats, ref, ref_stats = run_pair(cfg, 2048 + 700)
    assert_state_equal(got, ref, "long call")
    assert_stats_match(stats, ref_stats, cfg.precision, "long call")


def test_library_owned_buffers_and_side_stream():
    cfg = stream_cfg(2500, 8)
    s = torch.cuda.Stream()
    h = fsb.fsb_create(cfg, None, None, 0, s.cuda_stream)
    stats = np.zeros(15, fsb.STATS_DTYPE)
    fsb.fsb_step(h, 15, stats)
    got = {k: np.empty(2500, np.float32) for k in ("x", "y", "w", "prev", "cur")}
    assert fsb.fsb_read_state(h, got["x"], got["y"], got["w"], got["prev"], got["cur"]) == 15
    fsb.fsb_destroy(h)
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run(ocfg, ref, 0, 15)
    assert_state_equal(got, ref, "library buffers")
    assert_stats_match(stats, ref_stats, cfg.precision, "library buffers")


@pytest.mark.parametrize("precision", [fsb.FSB_FP32_KAHAN, fsb.FSB_FP64_STATE])
def test_resume_from_host_checkpoint(precision):
    cfg = stream_cfg(4321, 77, precision=precision, init_weight_mode=1)
    a = fsb.School.create(cfg)
    a.step(13)
    mid = a.read()
    a.step(11)
    end_a = a.read()
    a.destroy()
    b = fsb.School.create(cfg, init={"x": mid["x"], "y": mid["y"], "w": mid["w"],
                                     "prev_objective": mid["prev"]}, start_step=mid["step"])
    b.step(11)
    end_b = b.read()
    b.destroy()
    assert end_b["step"] == end_a["step"] == 24
    for k in ("x", "y", "w", "prev", "cur"):
        assert np.array_equal(end_a[k], end_b[k]), k


def test_runs_are_deterministic():
    cfg = stream_cfg(50_000, 4)
    outs = []
    for _ in range(2):
        s = fsb.School.create(cfg)
        st = s.step(30, stats=True)
        outs.append((st, s.read()))
        s.destroy()
    assert np.array_equal(outs[0][0], outs[1][0])
    for k in ("x", "y", "w", "prev"):
        assert np.array_equal(outs[0][1][k], outs[1][1][k])


def test_kernel_timing_counts_fused_launches():
    cfg = stream_cfg(100_000, 1)
    s = fsb.School.create(cfg)
    fsb.fsb_set_kernel_timing(s.handle, True)
    s.step(9)
    ms, n = fsb.fsb_kernel_time(s.handle)
    assert n == 8 and ms > 0.0
    fsb.fsb_set_kernel_timing(s.handle, False)
    s.destroy()


def test_argument_errors():
    cfg = stream_cfg(10, 1)
    s = fsb.School.create(cfg)
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_step(s.handle, 0)
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    s.destroy()
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_create(stream_cfg(10, 1), None, None, 0xFFFFFFFF, None)
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG


def test_still_school_never_eats():
    cfg = stream_cfg(777, 2, step=0.0, init_weight_mode=1)
    got, stats, ref, ref_stats = run_pair(cfg, 5)
    assert np.all(stats["max_abs_delta"] == 0.0)
    assert_state_equal(got, ref, "still")


def test_full_size_stream_school_sampled():
    """N = 2^28, seed 2, T = 100 in the launch configuration the benchmark
    times.  Sampled fish are followed by the oracle one by one (positions do
    not depend on weights; weights follow from the GPU's verified maxima);
    the last step's max|delta|, eat() statistic and barycentre sums are
    checked against the whole read-back state."""
    n, steps, seed = 1 << 28, 100, 2
    free, _ = torch.cuda.mem_get_info()
    if free < 12 * (1 << 30):
        pytest.skip("needs ~12 GB of free device memory")
    cfg = stream_cfg(n, seed)
    s = fsb.School.create(cfg)
    start = s.read()
    stats = s.step(steps, stats=True)
    got = s.read()
    s.destroy()
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([
        np.arange(0, 4096), np.arange(n - 4096, n),
        (np.arange(1, 200) * (n // 200)), rng.integers(0, n, 20000)])).astype(np.int64)
    ocfg = oracle_config(cfg)
    for i in idx:
        fish = np.zeros(1, oracle.FISH_F32)
        fish["x"], fish["y"] = start["x"][i], start["y"][i]
        fish["weight"] = start["w"][i]
        fish["prevObjective"] = start["prev"][i]
        fish["currentObjective"] = start["cur"][i]
        xs, ys, ds, fish = oracle.track_fish(ocfg, int(i), 0, steps, fish)
        assert xs[-1] == got["x"][i] and ys[-1] == got["y"][i], i
        assert fish["prevObjective"][0] == got["prev"][i], i
        assert fish["currentObjective"][0] == got["cur"][i], i
        assert np.all(np.abs(ds) <= stats["max_abs_delta"]), i
        ws = oracle.eat_fish(ocfg, float(start["w"][i]), ds, stats["max_abs_delta"])
        assert ws[-1] == got["w"][i], i
    delta = got["cur"] - got["prev"]
    assert stats["max_abs_delta"][-1] == np.max(np.abs(delta))
    assert stats["eat_max_diff"][-1] == np.max(got["prev"] - got["cur"])
    w64 = got["w"].astype(np.float64)
    ref_w = np.sum(w64)
    ref_x = np.sum(w64 * got["x"].astype(np.float64))
    abs_x = np.sum(w64 * np.abs(got["x"].astype(np.float64)))
    assert abs(stats["sum_w"][-1] - ref_w) / ref_w <= BARY_TOL[cfg.precision]
    assert abs(stats["sum_wx"][-1] - ref_x) / abs_x <= BARY_TOL[cfg.precision]


def host_free_bytes():
    return os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")


def test_full_size_stream_school_every_step():
    """N = 2^28, seed 2, T = 100 in the launch configuration the benchmark
    times, against the whole school advanced by the oracle's step on every
    host core (run_omp: run's per-fish arithmetic and maxima, pinned equal to
    run bit for bit): every step's max|delta| and eat() value exactly, every
    step's barycentre sums within the mode's tolerance, and every fish's final
    state bit for bit.  No GPU value feeds the oracle."""
    n, steps, seed = 1 << 28, 100, 2
    free, _ = torch.cuda.mem_get_info()
    if free < 12 * (1 << 30) or host_free_bytes() < 24 * (1 << 30):
        pytest.skip("needs ~12 GB of free device memory and ~24 GB of host memory")
    cfg = stream_cfg(n, seed)
    s = fsb.School.create(cfg)
    stats = s.step(steps, stats=True)
    got = s.read()
    s.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run_omp(ocfg, ref, 0, steps)
    assert_stats_match(stats, ref_stats, cfg.precision, "2^28 every step")
    assert_state_equal(got, ref, "2^28 T=100")


@pytest.mark.parametrize("kernel,stages", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_full_size_launch_shapes_agree_bitwise(kernel, stages):
    """The per-fish state is exact whatever the launch shape, so at the
    benchmark's size (N = 2^28, seed 2) the bulk-copy ring kernels and the
    vector-load kernel must leave the same bits in every fish after 100
    steps, with the same exact maxima; a stage refilled before all of its
    reads were performed would show up here as a handful of moved fish."""
    n, steps, seed = 1 << 28, 100, 2
    free, _ = torch.cuda.mem_get_info()
    if free < 12 * (1 << 30):
        pytest.skip("needs ~12 GB of free device memory")
    out = []
    for k, block, st in ((kernel, 512, stages), (1, 256, 2)):
        s = fsb.School.create(stream_cfg(n, seed))
        fsb.fsb_set_tuning(s.handle, stream_kernel=k, stream_block=block, stream_stages=st)
        stats = s.step(steps, stats=True)
        state = [t.clone() for t in s.tensors]
        s.destroy()
        out.append((state, stats))
    (a, sa), (b, sb) = out
    for name, ta, tb in zip(("x", "y", "w", "prev"), a, b):
        bad = int((ta.view(torch.int32) != tb.view(torch.int32)).sum())
        assert bad == 0, "%s differs in %d fish between launch shapes" % (name, bad)
    assert np.array_equal(sa["max_abs_delta"], sb["max_abs_delta"])
    assert np.array_equal(sa["eat_max_diff"], sb["eat_max_diff"])


@pytest.mark.parametrize("precision", [fsb.FSB_FP32_KAHAN, fsb.FSB_FP64_STATE])
def test_read_state_objective_over_chunks(precision):
    """fsb_read_state derives currentObjective chunk by chunk (2^22 fish per
    chunk).  With a ragged last chunk every fish must still hold the
    correctly rounded sqrt(x*x + y*y) of its read-back position (Sec. 2.1.1),
    which numpy computes here in the state's precision, one rounding per
    operation."""
    n = 2 * (1 << 22) + 12345
    s = fsb.School.create(stream_cfg(n, 31, precision=precision))
    s.step(3)
    got = s.read()
    s.destroy()
    x, y = got["x"], got["y"]
    want = np.sqrt(x * x + y * y)
    assert want.dtype == x.dtype
    bad = np.nonzero(got["cur"] != want)[0]
    assert bad.size == 0, "cur differs at %d fish, first %d" % (bad.size, bad[0])


@pytest.mark.parametrize("kernel", [2, 3])
@pytest.mark.parametrize("pass_index", [0, 2, 4])
def test_withheld_copy_times_out_without_hanging(kernel, pass_index):
    """Failure detection without a GPU fault: one block withholds the first
    bulk copy of its ring in one pass of a call (set from the host).  Its
    bounded wait runs out after 50 ms, every other block gives up, the passes
    behind it do nothing, the call reports FSB_ERR_TIMEOUT, and the context
    stays usable."""
    import time
    s = fsb.School.create(stream_cfg(1 << 22, 8))
    fsb.fsb_set_tuning(s.handle, stream_kernel=kernel)
    s.step(2)
    fsb.fsb_set_fault_injection(s.handle, 5, pass_index, 50_000_000)
    t0 = time.perf_counter()
    with pytest.raises(fsb.FsbError) as e:
        s.step(4, stats=True)                   # passes 0 (swim) .. 4 (settle)
    assert e.value.status == fsb.FSB_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    with pytest.raises(fsb.FsbError) as e:
        s.read()                                # the latched status is reported
    assert e.value.status == fsb.FSB_ERR_TIMEOUT
    s.destroy()
    t = torch.ones(1000, device="cuda")
    assert float(t.sum().item()) == 1000.0
    cfg = stream_cfg(50_001, 3)
    ok = fsb.School.create(cfg)
    fsb.fsb_set_tuning(ok.handle, stream_kernel=kernel)
    stats = ok.step(3, stats=True)
    got = ok.read()
    ok.destroy()
    ref = oracle.init(oracle_config(cfg))
    ref_stats = oracle.run(oracle_config(cfg), ref, 0, 3)
    assert_state_equal(got, ref, "after a failed handle")
    assert_stats_match(stats, ref_stats, cfg.precision, "after a failed handle")


def test_fault_injection_needs_a_copy_ring_kernel():
    s = fsb.School.create(stream_cfg(10_000, 1))
    fsb.fsb_set_tuning(s.handle, stream_kernel=1)
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_set_fault_injection(s.handle, 0, 1, 0)
    assert e.value.status == fsb.FSB_ERR_UNSUPPORTED
    fsb.fsb_set_tuning(s.handle, stream_kernel=2)
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_set_fault_injection(s.handle, 100000, 1, 0)
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    fsb.fsb_set_fault_injection(s.handle, -1, 0, 0)   # clearing is always fine
    s.step(2)
    s.destroy()


@pytest.mark.parametrize("precision", [fsb.FSB_FP32_KAHAN, fsb.FSB_FP64_STATE])
@pytest.mark.parametrize("offset", [0, 1])
def test_pinned_host_transfers_match_the_copy_engine_path(precision, offset):
    """Pinned host arrays are read and written by kernels (vector groups when
    every array is 16-byte aligned, one fish per thread otherwise); pageable
    ones by the copy engines.  Both routes give the same bits, and a school
    resumed from a pinned checkpoint runs as one resumed from pageable
    memory."""
    n = 100_003
    cfg = stream_cfg(n, 77, precision=precision, init_weight_mode=1)
    dt = torch.float64 if precision == fsb.FSB_FP64_STATE else torch.float32
    s = fsb.School.create(cfg)
    s.step(5)
    want = s.read()                                   # pageable: copy engines
    pinned = [torch.empty(n + offset, dtype=dt).pin_memory()[offset:] for _ in range(5)]
    views = [t.numpy() for t in pinned]
    assert fsb.fsb_read_state(s.handle, *views) == 5  # pinned: kernels
    for k, v in zip(("x", "y", "w", "prev", "cur"), views):
        assert np.array_equal(v, want[k]), k
    # only some fields, with currentObjective computed on the way out
    for t in pinned:
        t.zero_()
    fsb.fsb_read_state(s.handle, None, views[1], None, None, views[4])
    assert np.array_equal(views[1], want["y"]) and np.array_equal(views[4], want["cur"])
    assert not views[0].any()
    s.destroy()
    # resume from the pinned arrays, and from pageable copies of them
    out = []
    for src in (views[:4], [np.array(v) for v in views[:4]]):
        r = fsb.School.create(cfg, init=dict(zip(("x", "y", "w", "prev_objective"), src)),
                              start_step=5)
        st = r.step(3, stats=True)
        out.append((r.read(), st))
        r.destroy()
    (a, sa), (b, sb) = out
    for k in ("x", "y", "w", "prev", "cur"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(sa["max_abs_delta"], sb["max_abs_delta"])
