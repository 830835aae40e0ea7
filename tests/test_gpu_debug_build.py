"""The debug library (build.py debug=True: the run-time invariant checks of
fsb_check.cuh compiled in) runs the resident, batched and streaming paths on
small ragged cases with no check failing, and still matches the oracle bit
for bit.  It runs in a child process, which loads libfsb_debug.so instead of
the release library this test session uses."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys
import numpy as np
sys.path.insert(0, os.path.join(os.environ["FSB_ROOT"], "tests"))
sys.path.insert(0, os.environ["FSB_ROOT"])
import oracle
import paper_2507_20173_gb300 as fsb
from paper_2507_20173_gb300 import build
from fsb_testutil import assert_state_equal, assert_stats_match, oracle_config
import torch

fsb.LIB_PATH = build.build(debug=True)
fsb.lib()

def single(n, path, steps, **kw):
    cfg = fsb.fsb_config_init(n, 11 + n, path=path, **kw)
    school = fsb.School.create(cfg)
    stats = school.step(steps, stats=True)   # synchronises: latched checks surface here
    got = school.read()
    school.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run(ocfg, ref, 0, steps)
    assert_state_equal(got, ref, "debug %d path %d" % (n, path))
    assert_stats_match(stats, ref_stats, cfg.precision, "debug %d path %d" % (n, path))

for n in (1, 33, 4097, 300001):
    single(n, fsb.FSB_PATH_RESIDENT, 7, init_weight_mode=1)
single(4097, fsb.FSB_PATH_RESIDENT, 5, swim_mode=1)
for n in (5, 4097, 100003):
    single(n, fsb.FSB_PATH_STREAM, 5)

sizes = np.array([65536, 33000, 20000, 9000, 8192, 700, 1, 2, 4097], dtype=np.uint64)
offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
seeds = (77 + np.arange(sizes.size)).astype(np.uint64)
tmpl = fsb.fsb_config_init(1, 0, init_weight_mode=1)
ts = [torch.zeros(int(offsets[-1]), dtype=torch.float32, device="cuda") for _ in range(4)]
state = fsb.FsbStateDev(*(t.data_ptr() for t in ts))
steps = 5
stats = np.zeros(sizes.size * steps, fsb.STATS_DTYPE)
fsb.fsb_run_batch(tmpl, offsets, seeds, state, steps, init=True, stats=stats)
x, y, w, pv = (t.cpu().numpy() for t in ts)
for k in range(sizes.size):
    lo, hi = int(offsets[k]), int(offsets[k + 1])
    ocfg = oracle.Config(n_fish=hi - lo, seed=int(seeds[k]), school_id=k, init_weight_mode=1)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run(ocfg, ref, 0, steps)
    sub = {"x": x[lo:hi], "y": y[lo:hi], "w": w[lo:hi], "prev": pv[lo:hi],
           "cur": np.sqrt(x[lo:hi] * x[lo:hi] + y[lo:hi] * y[lo:hi])}
    assert_state_equal(sub, ref, "debug batch school %d" % k)
    assert_stats_match(stats[k * steps:(k + 1) * steps], ref_stats, tmpl.precision,
                       "debug batch school %d" % k)
print("debug library: every check held")
'''


def test_debug_library_checks_hold_and_matches_the_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, FSB_ROOT=ROOT)
    proc = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True,
                          timeout=1200)
    assert proc.returncode == 0, proc.stdout[-2000:] + proc.stderr[-4000:]
    assert "every check held" in proc.stdout


ERRORS_CHILD = r'''
import os, sys
import numpy as np
sys.path.insert(0, os.environ["FSB_ROOT"])
import paper_2507_20173_gb300 as fsb
from paper_2507_20173_gb300 import build
import torch

fsb.LIB_PATH = build.build(debug=True)
fsb.lib()

def expect(status, call):
    try:
        call()
    except fsb.FsbError as e:
        assert e.status == status, (e.status, status, str(e))
        return
    assert status == fsb.FSB_OK, "expected %s" % fsb.fsb_strerror(status)

n = 4096
cfg = fsb.fsb_config_init(n, 3, path=fsb.FSB_PATH_STREAM)
good = fsb.School.create(cfg)
st = good.read()
good.destroy()
bad = {k: st[k].copy() for k in ("x", "y", "w", "prev")}
bad["x"][17] = np.float32(3 * cfg.pond_half)     # a fish outside the pond

# the handle path reports the latched status at its synchronising call
s = fsb.School.create(cfg, init={"x": bad["x"], "y": bad["y"], "w": bad["w"],
                                 "prev_objective": bad["prev"]})
expect(fsb.FSB_ERR_STATE, lambda: s.step(3, stats=True))
s.destroy()

# the allocation-free path: an asynchronous call (no or device statistics)
# returns OK, and the next synchronising call (host statistics) reports the
# carried status once
stream = torch.cuda.current_stream().cuda_stream
ts = [torch.from_numpy(bad[k]).cuda() for k in ("x", "y", "w", "prev")]
state = fsb.FsbStateDev(*(t.data_ptr() for t in ts))
host = np.zeros(3, fsb.STATS_DTYPE)
dev = torch.zeros(3 * fsb.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
expect(fsb.FSB_OK, lambda: fsb.fsb_step_static(cfg, state, 0, 3, None, stream))
expect(fsb.FSB_OK, lambda: fsb.fsb_step_static(cfg, state, 3, 3, dev.data_ptr(), stream))
expect(fsb.FSB_ERR_STATE, lambda: fsb.fsb_step_static(cfg, state, 6, 3, host, stream))
expect(fsb.FSB_OK, lambda: fsb.fsb_step_static(cfg, state, 9, 3, host, stream))
# a synchronising call that fails itself reports its own status
ts[0][17] = 3 * cfg.pond_half
expect(fsb.FSB_ERR_STATE, lambda: fsb.fsb_step_static(cfg, state, 12, 3, host, stream))
expect(fsb.FSB_OK, lambda: fsb.fsb_step_static(cfg, state, 15, 3, host, stream))
print("device errors reported")
'''


def test_debug_library_reports_a_state_outside_the_pond():
    """The debug build checks that every fish a streaming pass reads lies in
    the pond (the method never leaves it).  A school with one fish outside is
    reported as FSB_ERR_STATE: by fsb_step when it synchronises, and by
    fsb_step_static at the first call given host statistics, whether the
    failing call was that one or an earlier asynchronous one."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, FSB_ROOT=ROOT)
    proc = subprocess.run([sys.executable, "-c", ERRORS_CHILD], env=env, capture_output=True,
                          text=True, timeout=1200)
    assert proc.returncode == 0, proc.stdout[-2000:] + proc.stderr[-4000:]
    assert "device errors reported" in proc.stdout
