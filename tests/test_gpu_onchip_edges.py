"""Edge cases of the on-chip (resident and batched) per-pair passes against
the CPU oracle: swim steps on either side of the threshold below which the
paired swim keeps the two-rounding form of (2u - 1) * s (s * 2^-23 must be
exact to fold it; such a step runs the kernels' variant copies, which
choose the form per pair), tiny ponds whose objectives underflow,
subnormal positions, and both model variants, bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2507_20173_gb300 as fsb
from fsb_testutil import assert_state_equal, assert_stats_match, oracle_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (pond half-width P, swim step s): s = 2^-103 is the smallest step whose
# s * 2^-23 is normal (folded form); 1.5 * 2^-104 and a subnormal step take
# the two-rounding form; P = 2^-100 keeps positions within reach of s.
EDGE_PHYSICS = [
    (2.0 ** -100, 2.0 ** -103),
    (2.0 ** -100, 1.5 * 2.0 ** -104),
    (2.0 ** -120, 3.0e-40),
    (1.0e-30, 1.0e-30),
    (100.0, 0.0),
    (100.0, 1.0e30),
    (3.0, 0.7),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_20173_gb300 import build
    build.build()
    fsb.lib()


@pytest.mark.parametrize("pond,step", EDGE_PHYSICS)
@pytest.mark.parametrize("variant", [{}, {"swim_mode": 1}, {"feed_mode": 1}])
def test_resident_edge_physics(pond, step, variant):
    cfg = fsb.fsb_config_init(5001, 17, path=fsb.FSB_PATH_RESIDENT, pond_half=pond, step=step,
                              init_weight_mode=1, **variant)
    school = fsb.School.create(cfg)
    assert fsb.fsb_handle_path(school.handle) == fsb.FSB_PATH_RESIDENT
    stats = school.step(7, stats=True)
    got = school.read()
    school.destroy()
    ocfg = oracle_config(cfg)
    ref = oracle.init(ocfg)
    ref_stats = oracle.run(ocfg, ref, 0, 7)
    what = "resident P=%g s=%g %s" % (pond, step, variant)
    assert_state_equal(got, ref, what)
    assert_stats_match(stats, ref_stats, cfg.precision, what)


@pytest.mark.parametrize("pond,step", EDGE_PHYSICS)
def test_batch_edge_physics(pond, step):
    sizes = np.array([3, 4097, 9001], dtype=np.uint64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    seeds = np.array([5, 6, 7], dtype=np.uint64)
    tmpl = fsb.fsb_config_init(1, 0, pond_half=pond, step=step, init_weight_mode=1)
    ts = [torch.zeros(int(offsets[-1]), dtype=torch.float32, device="cuda") for _ in range(4)]
    state = fsb.FsbStateDev(*(t.data_ptr() for t in ts))
    steps = 6
    stats = np.zeros(sizes.size * steps, fsb.STATS_DTYPE)
    fsb.fsb_run_batch(tmpl, offsets, seeds, state, steps, init=True, stats=stats)
    x, y, w, pv = (t.cpu().numpy() for t in ts)
    for k in range(sizes.size):
        lo, hi = int(offsets[k]), int(offsets[k + 1])
        ocfg = oracle.Config(n_fish=hi - lo, seed=int(seeds[k]), school_id=k, init_weight_mode=1,
                             pond_half=pond, step=step, w0=tmpl.w0, w_min=tmpl.w_min,
                             w_max=tmpl.w_max)
        ref = oracle.init(ocfg)
        ref_stats = oracle.run(ocfg, ref, 0, steps)
        sub = {"x": x[lo:hi], "y": y[lo:hi], "w": w[lo:hi], "prev": pv[lo:hi],
               "cur": np.sqrt(x[lo:hi] * x[lo:hi] + y[lo:hi] * y[lo:hi])}
        what = "batch school %d P=%g s=%g" % (k, pond, step)
        assert_state_equal(sub, ref, what)
        assert_stats_match(stats[k * steps:(k + 1) * steps], ref_stats, tmpl.precision, what)
