"""fsb_step_static: the allocation-free entry point, for callers that cannot
let a library allocate device memory at call time (hosts that own all GPU
memory through their own arena, latency-bound pipelines where cudaMalloc's
device-wide synchronisation would stall other streams).

It is checked against the regular entry point (fsb_create + fsb_step) on two
calls in a row, through the C ABI: the same state bit-for-bit, the same
maxima, and barycentre sums within the tolerance of the arithmetic mode
(normalised, as every parity test here, by the sum of |w x| from the
oracle).  Its throughput is taken once beside fsb_step's.  This file is
collected last so a failure here never hides another test.
"""
import numpy as np
import pytest

import oracle
import paper_2507_20173_gb300 as fsb
from fsb_testutil import BARY_TOL, oracle_config, oracle_precision

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_20173_gb300 import build
    build.build()
    fsb.lib()


def read_tensors(ts):
    return [t.cpu().numpy() for t in ts]


@pytest.mark.parametrize("precision", [fsb.FSB_FP32_KAHAN, fsb.FSB_FP64_STATE])
@pytest.mark.parametrize("n", [4097, 300_001])
def test_static_step_matches_regular_entry_point(n, precision):
    cfg = fsb.fsb_config_init(n, 31337 + n, precision=precision, init_weight_mode=1,
                              school_id=2)
    stream = torch.cuda.current_stream()
    ref = fsb.School.create(cfg, stream=stream)
    start = ref.read()
    dt = torch.float64 if precision == fsb.FSB_FP64_STATE else torch.float32
    # caller-owned copies of the same initial state for the static path
    mine = [torch.from_numpy(np.ascontiguousarray(start[k])).to("cuda", dt)
            for k in ("x", "y", "w", "prev")]
    state = fsb.FsbStateDev(*(t.data_ptr() for t in mine))
    # the normalisers of the sum errors: sum |w x|, sum |w y| of each step
    ocfg = oracle_config(cfg)
    norm = oracle.run(ocfg, oracle.init(ocfg, oracle_precision(cfg)), 0, 12)
    step = 0
    for n_steps in (7, 5):                       # two calls in a row
        want = ref.step(n_steps, stats=True)
        got = np.zeros(n_steps, fsb.STATS_DTYPE)
        fsb.fsb_step_static(cfg, state, step, n_steps, got, stream.cuda_stream)
        torch.cuda.synchronize()
        o = norm[step:step + n_steps]
        step += n_steps
        assert np.array_equal(got["max_abs_delta"], want["max_abs_delta"])
        assert np.array_equal(got["eat_max_diff"], want["eat_max_diff"])
        for k, d in (("sum_w", np.abs(o["sum_w"])), ("sum_wx", o["sum_abs_wx"]),
                     ("sum_wy", o["sum_abs_wy"])):
            err = np.abs(got[k] - want[k]) / d
            assert err.max() <= BARY_TOL[precision], (k, err.max())
        r = ref.read()
        for k, t in zip(("x", "y", "w", "prev"), read_tensors(mine)):
            assert np.array_equal(t, r[k]), (n_steps, k)
    ref.destroy()


def test_static_step_runs_at_the_regular_rate():
    """Calls of 20 steps on 2^26 fish, timed with CUDA events beside fsb_step
    on the same school: the static path runs fsb_step's kernels in fsb_step's
    launch shape, so it keeps its rate (the loose bound allows for the launch
    cost of its uncaptured passes).  Each entry point runs one untimed call
    of the same length first."""
    n, steps = 1 << 26, 20
    cfg = fsb.fsb_config_init(n, 5, path=fsb.FSB_PATH_STREAM)
    stream = torch.cuda.current_stream()
    ref = fsb.School.create(cfg, stream=stream)
    # the kernels the static path runs (the library's choice for this size
    # is stream kernel 5, which needs scratch the static path does not have)
    fsb.fsb_set_tuning(ref.handle, stream_kernel=1)
    st0 = ref.read()
    ts = [torch.from_numpy(st0[k]).to("cuda") for k in ("x", "y", "w", "prev")]
    del st0
    state = fsb.FsbStateDev(*(t.data_ptr() for t in ts))
    calls = {"fsb_step": lambda k: fsb.fsb_step(ref.handle, steps),
             "fsb_step_static": lambda k: fsb.fsb_step_static(cfg, state, k * steps, steps,
                                                              None, stream.cuda_stream)}
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = {}
    for name, call in calls.items():
        call(0)
        torch.cuda.synchronize()
        a.record(stream)
        call(1)
        b.record(stream)
        torch.cuda.synchronize()
        times[name] = a.elapsed_time(b)
    ref.destroy()
    rate = {k: n * steps / (v / 1e3) for k, v in times.items()}
    print("fish-steps/s: fsb_step %.3e, fsb_step_static %.3e" % (rate["fsb_step"],
                                                                  rate["fsb_step_static"]))
    assert rate["fsb_step_static"] >= 0.8 * rate["fsb_step"], rate


def test_static_step_rejects_runs_beyond_its_scratch():
    cfg = fsb.fsb_config_init(1000, 1)
    ts = [torch.zeros(1000, dtype=torch.float32, device="cuda") for _ in range(4)]
    state = fsb.FsbStateDev(*(t.data_ptr() for t in ts))
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_step_static(cfg, state, 0, 4097, None, s)
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    assert "4096" in fsb.fsb_last_error()
    # the step counter must stay below 2^32, also for a start near 2^64
    for start in ((1 << 32) - 5, (1 << 64) - 2):
        with pytest.raises(fsb.FsbError) as e:
            fsb.fsb_step_static(cfg, state, start, 10, None, s)
        assert e.value.status == fsb.FSB_ERR_INVALID_ARG
