"""fsb_step_static: the allocation-free entry point, for callers that cannot
let a library allocate device memory at call time (hosts that own all GPU
memory through their own arena, latency-bound pipelines where cudaMalloc's
device-wide synchronisation would stall other streams).

It is checked against the regular entry point (fsb_create + fsb_step) on two
calls in a row, through the C ABI: the same state bit-for-bit, the same
maxima, and barycentre sums within the tolerance of the arithmetic mode.
This file is collected last so a failure here never hides another test.
"""
import numpy as np
import pytest

import paper_2507_20173_gb300 as fsb
from fsb_testutil import BARY_TOL

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
    step = 0
    for n_steps in (7, 5):                       # two calls in a row
        want = ref.step(n_steps, stats=True)
        got = np.zeros(n_steps, fsb.STATS_DTYPE)
        fsb.fsb_step_static(cfg, state, step, n_steps, got, stream.cuda_stream)
        torch.cuda.synchronize()
        step += n_steps
        assert np.array_equal(got["max_abs_delta"], want["max_abs_delta"])
        assert np.array_equal(got["eat_max_diff"], want["eat_max_diff"])
        for k in ("sum_w", "sum_wx", "sum_wy"):
            err = np.abs(got[k] - want[k]) / np.maximum(np.abs(want[k]), 1.0)
            assert err.max() <= BARY_TOL[precision], (k, err.max())
        r = ref.read()
        for k, t in zip(("x", "y", "w", "prev"), read_tensors(mine)):
            assert np.array_equal(t, r[k]), (n_steps, k)
    ref.destroy()


def test_static_step_rejects_runs_beyond_its_scratch():
    cfg = fsb.fsb_config_init(1000, 1)
    ts = [torch.zeros(1000, dtype=torch.float32, device="cuda") for _ in range(4)]
    state = fsb.FsbStateDev(*(t.data_ptr() for t in ts))
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_step_static(cfg, state, 0, 4097, None, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    assert "4096" in fsb.fsb_last_error()
