"""GPU parity of the batched path (many schools of uneven size in one
persistent launch) against the CPU oracle, school by school."""
import numpy as np
import pytest

import oracle
import paper_2507_20173_gb300 as fsb
from fsb_testutil import assert_state_equal, assert_stats_match
from paper_2507_20173_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# fish one block holds and fish one warp of a packed team holds (library
# constants, read once the library is loaded)
BF = TF = 0


def edge_sizes():
    return [1, 2, 31, 257, 512, 4097, BF // 2, BF // 2 + 1, BF - 1, BF, BF + 1, 12000, 20000,
            40000, 65536, 8 * BF, 3, 700]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_20173_gb300 import build
    build.build()
    fsb.lib()
    global BF, TF
    limits = fsb.fsb_batch_limits()
    BF, TF = limits["block_fish"], limits["team_fish"]
    assert BF > 0 and TF > 0 and limits["max_cluster"] == 8


def team_warps(n):
    """Warps of the packed team a school of n fish runs on (TF fish per
    warp; 0: not packed, more than half a block)."""
    n = int(n)
    if n > 8 * TF:
        return 0
    w = 1
    while w * TF < n:
        w *= 2
    return w


def make_state(total):
    ts = [torch.zeros(int(total), dtype=torch.float32, device="cuda") for _ in range(4)]
    return ts, fsb.FsbStateDev(*(t.data_ptr() for t in ts))


def read_state(ts):
    x, y, w, pv = (t.cpu().numpy() for t in ts)
    cur = None
    return {"x": x, "y": y, "w": w, "prev": pv}


def oracle_school(tmpl, n, seed, school_id, steps, **kw):
    cfg = oracle.Config(n_fish=int(n), seed=int(seed), school_id=int(school_id),
                        init_weight_mode=tmpl.init_weight_mode, pond_half=tmpl.pond_half,
                        step=tmpl.step, w0=tmpl.w0, w_min=tmpl.w_min, w_max=tmpl.w_max,
                        swim_mode=tmpl.swim_mode, feed_mode=tmpl.feed_mode)
    school = oracle.init(cfg)
    stats = oracle.run(cfg, school, 0, steps) if steps else None
    return school, stats


def check_batch(tmpl, offsets, seeds, got, stats, steps, precision):
    for k in range(seeds.size):
        lo, hi = int(offsets[k]), int(offsets[k + 1])
        ref, ref_stats = oracle_school(tmpl, hi - lo, seeds[k], k, steps)
        sub = {"x": got["x"][lo:hi], "y": got["y"][lo:hi], "w": got["w"][lo:hi],
               "prev": got["prev"][lo:hi],
               "cur": np.sqrt(got["x"][lo:hi] * got["x"][lo:hi] +
                              got["y"][lo:hi] * got["y"][lo:hi])}
        ref_cmp = ref.copy()
        # currentObjective is derived on the device by fsb_read_state for a
        # single school; here it is recomputed in binary32 by numpy (each
        # operation correctly rounded), matching the stored positions
        assert_state_equal(sub, ref_cmp, "school %d (N=%d)" % (k, hi - lo))
        if steps:
            assert_stats_match(stats[k * steps:(k + 1) * steps], ref_stats, precision,
                               "school %d" % k)


@pytest.mark.parametrize("cluster", [1, 2, 3, 4, 5, 6, 7, 8])
def test_edge_size_batch_every_cluster_size(cluster):
    """Every school on clusters of `cluster` blocks (1: every school on a
    block of its own, none packed)."""
    sizes = np.array(edge_sizes(), dtype=np.uint64)
    if cluster * BF < sizes.max():
        sizes = np.minimum(sizes, cluster * BF)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    seeds = (1000 + np.arange(sizes.size)).astype(np.uint64)
    tmpl = fsb.fsb_config_init(1, 0, step=2.0, init_weight_mode=1)
    ts, state = make_state(offsets[-1])
    b = fsb.fsb_batch_create(tmpl, offsets, seeds, state, init=True)
    fsb.fsb_batch_set_cluster(b, cluster)
    info = fsb.fsb_batch_info(b)
    assert info["cluster"] == cluster and info["n_clusters"] >= 1
    steps = 6
    stats = np.zeros(sizes.size * steps, fsb.STATS_DTYPE)
    fsb.fsb_batch_step(b, steps, stats)
    fsb.fsb_batch_destroy(b)
    check_batch(tmpl, offsets, seeds, read_state(ts), stats, steps, tmpl.precision)


def test_single_block_clusters_for_small_schools():
    sizes = np.array([1, 5, 100, 8192, 4000, 333], dtype=np.uint64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    seeds = (7 + np.arange(sizes.size)).astype(np.uint64)
    tmpl = fsb.fsb_config_init(1, 0)
    ts, state = make_state(offsets[-1])
    b = fsb.fsb_batch_create(tmpl, offsets, seeds, state, init=True)
    assert fsb.fsb_batch_info(b)["cluster"] == 1
    stats = np.zeros(sizes.size * 9, fsb.STATS_DTYPE)
    fsb.fsb_batch_step(b, 9, stats)
    fsb.fsb_batch_destroy(b)
    check_batch(tmpl, offsets, seeds, read_state(ts), stats, 9, tmpl.precision)


def test_init_only_and_split_calls():
    sizes = np.array([300, 9000, 17], dtype=np.uint64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    seeds = np.array([5, 6, 2 ** 40 + 3], dtype=np.uint64)
    tmpl = fsb.fsb_config_init(1, 0)
    ts, state = make_state(offsets[-1])
    b = fsb.fsb_batch_create(tmpl, offsets, seeds, state, init=True)
    fsb.fsb_batch_step(b, 0)
    torch.cuda.synchronize()
    check_batch(tmpl, offsets, seeds, read_state(ts), None, 0, tmpl.precision)
    s1 = np.zeros(sizes.size * 3, fsb.STATS_DTYPE)
    s2 = np.zeros(sizes.size * 4, fsb.STATS_DTYPE)
    fsb.fsb_batch_step(b, 3, s1)
    fsb.fsb_batch_step(b, 4, s2)
    assert fsb.fsb_batch_info(b)["step"] == 7
    fsb.fsb_batch_destroy(b)
    got = read_state(ts)
    stats = np.concatenate([np.concatenate([s1[k * 3:(k + 1) * 3], s2[k * 4:(k + 1) * 4]])
                            for k in range(sizes.size)])
    check_batch(tmpl, offsets, seeds, got, stats, 7, tmpl.precision)


def test_batch_school_equals_single_school_run():
    sizes = np.array([1000, 20000, 4096], dtype=np.uint64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    seeds = np.array([11, 12, 13], dtype=np.uint64)
    tmpl = fsb.fsb_config_init(1, 0)
    ts, state = make_state(offsets[-1])
    fsb.fsb_run_batch(tmpl, offsets, seeds, state, 10, init=True)
    torch.cuda.synchronize()
    got = read_state(ts)
    for k in range(3):
        cfg = fsb.fsb_config_init(int(sizes[k]), int(seeds[k]), school_id=k)
        s = fsb.School.create(cfg)
        s.step(10)
        one = s.read()
        s.destroy()
        lo, hi = int(offsets[k]), int(offsets[k + 1])
        for f in ("x", "y", "w", "prev"):
            assert np.array_equal(one[f], got[f][lo:hi]), (k, f)


@pytest.mark.parametrize("precision", [fsb.FSB_FP32, fsb.FSB_FP64_ACC])
def test_ragged_ensemble_sample(precision):
    """A 64-school sample of the log-uniform [256, 65536] ensemble."""
    wl = workloads.ragged_batch(64, 256, 65536, seed=3)
    offsets, seeds = wl.offsets(), wl.seeds()
    tmpl = fsb.fsb_config_init(1, 0, precision=precision)
    ts, state = make_state(offsets[-1])
    steps = 8
    stats = np.zeros(seeds.size * steps, fsb.STATS_DTYPE)
    fsb.fsb_run_batch(tmpl, offsets, seeds, state, steps, init=True, stats=stats)
    check_batch(tmpl, offsets, seeds, read_state(ts), stats, steps, precision)


def test_batch_argument_errors():
    tmpl = fsb.fsb_config_init(1, 0)
    big = 8 * BF + 1                             # more than a cluster of 8 holds
    ts, state = make_state(big)
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_batch_create(tmpl, np.array([0, big], np.uint64), np.array([1], np.uint64),
                             state, init=True)
    assert e.value.status == fsb.FSB_ERR_UNSUPPORTED
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_batch_create(tmpl, np.array([0, 10, 10], np.uint64), np.array([1, 2], np.uint64),
                             state, init=True)
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    t64 = fsb.fsb_config_init(1, 0, precision=fsb.FSB_FP64_STATE)
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_batch_create(t64, np.array([0, 10], np.uint64), np.array([1], np.uint64),
                             state, init=True)
    assert e.value.status == fsb.FSB_ERR_UNSUPPORTED
    b = fsb.fsb_batch_create(tmpl, np.array([0, BF + 1], np.uint64), np.array([1], np.uint64),
                             state, init=True)
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_batch_set_cluster(b, 1)          # BF + 1 fish do not fit one block
    assert e.value.status == fsb.FSB_ERR_UNSUPPORTED
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_batch_set_cluster(b, 9)          # beyond the widest cluster
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    fsb.fsb_batch_step(b, 2)
    fsb.fsb_batch_destroy(b)


def test_default_plan_runs_each_school_on_the_cluster_that_holds_it():
    """With no forced cluster size every school goes to the queue of the
    smallest cluster (1 to 8 blocks of BF fish) that holds it (one of at
    most half a block to the smallest packed team of warps), one
    concurrent launch per size, largest first, single blocks on the SMs left
    over; the result is still every school's single-school trajectory."""
    sizes = np.array([65536, 40000, 33000, 32768, 20000, 16385, 16384, 9000, 8193, 8192, 5000,
                      700, 31, 1, 2, 64000, 12000, 30000, 4096], dtype=np.uint64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    seeds = (3000 + np.arange(sizes.size)).astype(np.uint64)
    tmpl = fsb.fsb_config_init(1, 0, step=1.5, init_weight_mode=1)
    ts, state = make_state(offsets[-1])
    b = fsb.fsb_batch_create(tmpl, offsets, seeds, state, init=True)
    plan = fsb.fsb_batch_plan(b)
    need = [max(1, -(-int(n) // BF)) for n in sizes]   # blocks of BF fish that hold it
    packed = [team_warps(n) for n in sizes]
    assert plan["queue_schools"] == {c: sum(1 for k, m in enumerate(need)
                                            if m == c and not packed[k])
                                     for c in range(8, 0, -1)}
    assert plan["packed_schools"] == {w: packed.count(w) for w in (8, 4, 2, 1)}
    clusters = [l["cluster"] for l in plan["launches"]]
    assert clusters[0] == max(need) and clusters == sorted(clusters, reverse=True)
    assert max(need) > 2
    assert all(need.count(c) > 0 for c in clusters if c > 1)
    for l in plan["launches"]:
        assert l["blocks"] >= l["cluster"] and l["blocks"] % l["cluster"] == 0
    info = fsb.fsb_batch_info(b)
    assert info["cluster"] == max(need) and info["n_big"] == sum(c > 1 for c in need)
    steps = 5
    stats = np.zeros(sizes.size * steps, fsb.STATS_DTYPE)
    fsb.fsb_batch_step(b, steps, stats)
    fsb.fsb_batch_destroy(b)
    check_batch(tmpl, offsets, seeds, read_state(ts), stats, steps, tmpl.precision)


def test_forced_cluster_size_and_back_to_the_default_plan():
    # on 2, 1 (a whole block), 1 (a packed warp) and 3 blocks
    sizes = np.array([2 * BF - 500, BF - 100, 100, 3 * BF - 1000], dtype=np.uint64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    seeds = (40 + np.arange(sizes.size)).astype(np.uint64)
    tmpl = fsb.fsb_config_init(1, 0)
    ts, state = make_state(offsets[-1])
    b = fsb.fsb_batch_create(tmpl, offsets, seeds, state, init=True)
    assert [l["cluster"] for l in fsb.fsb_batch_plan(b)["launches"]] == [3, 2, 1]
    fsb.fsb_batch_set_cluster(b, 8)
    plan = fsb.fsb_batch_plan(b)
    assert plan["launches"][0]["cluster"] == 8 and plan["queue_schools"][8] == 2
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_batch_set_cluster(b, 2)          # 3 BF - 1000 fish do not fit 2 blocks
    assert e.value.status == fsb.FSB_ERR_UNSUPPORTED
    assert fsb.fsb_batch_plan(b)["launches"][0]["cluster"] == 8   # unchanged
    fsb.fsb_batch_set_cluster(b, 0)
    plan = fsb.fsb_batch_plan(b)
    assert plan["queue_schools"] == {8: 0, 7: 0, 6: 0, 5: 0, 4: 0, 3: 1, 2: 1, 1: 1}
    assert plan["packed_schools"] == {8: 0, 4: 0, 2: 0, 1: 1}     # 100 fish on one warp
    stats = np.zeros(sizes.size * 4, fsb.STATS_DTYPE)
    fsb.fsb_batch_step(b, 4, stats)
    fsb.fsb_batch_destroy(b)
    check_batch(tmpl, offsets, seeds, read_state(ts), stats, 4, tmpl.precision)


def test_explicit_plans_give_the_same_trajectories():
    """Explicit launch plans (one cluster of 8 alone, a few blocks per
    launch, the tuned shares, a wide single-block launch) change which block
    runs which school and in what order; every plan must give every school
    its single-school trajectory."""
    sizes = np.array([65536, 40000, 33000, 20000, 16385, 9000, 8193, 8192, 5000, 700, 31, 1, 2,
                      4097], dtype=np.uint64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    seeds = (5000 + np.arange(sizes.size)).astype(np.uint64)
    tmpl = fsb.fsb_config_init(1, 0, step=1.5, init_weight_mode=1)
    steps = 4
    plans = [[(8, 8)], [(8, 16), (1, 3)], [(8, 8), (4, 4), (2, 2), (1, 1)],
             [(8, 80), (4, 32), (2, 20), (1, 20)], [(8, 8), (1, 100)]]
    refs = [oracle_school(tmpl, int(offsets[k + 1] - offsets[k]), seeds[k], k, steps)
            for k in range(sizes.size)]
    for plan in plans:
        ts, state = make_state(offsets[-1])
        b = fsb.fsb_batch_create(tmpl, offsets, seeds, state, init=True)
        fsb.fsb_batch_set_plan(b, plan)
        stats = np.zeros(sizes.size * steps, fsb.STATS_DTYPE)
        fsb.fsb_batch_step(b, steps, stats)
        fsb.fsb_batch_destroy(b)
        got = read_state(ts)
        for k, (ref, ref_stats) in enumerate(refs):
            lo, hi = int(offsets[k]), int(offsets[k + 1])
            sub = {"x": got["x"][lo:hi], "y": got["y"][lo:hi], "w": got["w"][lo:hi],
                   "prev": got["prev"][lo:hi],
                   "cur": np.sqrt(got["x"][lo:hi] * got["x"][lo:hi] +
                                  got["y"][lo:hi] * got["y"][lo:hi])}
            what = "plan %s school %d (N=%d)" % (plan, k, hi - lo)
            assert_state_equal(sub, ref, what)
            assert_stats_match(stats[k * steps:(k + 1) * steps], ref_stats, tmpl.precision, what)


def pack_edges():
    return [1, 2, 3, 31, 32, 33, 255, 256, TF - 1, TF, TF + 1, 2 * TF - 1, 2 * TF, 2 * TF + 1,
            4 * TF - 1, 4 * TF, 4 * TF + 1, 8 * TF - 1, 8 * TF, 8 * TF + 1, BF]


@pytest.mark.parametrize("plan", [None, [(1, 1)], [(1, 3)], [(2, 2), (1, 1)]])
@pytest.mark.parametrize("steps", [1, 2, 7])
def test_packed_teams_every_size_class(plan, steps):
    """Schools at the edges of every team size (1, 2, 4, 8 times TF fish on
    teams of 1, 2, 4, 8 warps), three of each, beside whole-block
    schools.  On one block (plan (1, 1)) every team runs several schools in
    turn and the teams split level by level while others still run; every
    school must keep its single-school trajectory, maxima exact."""
    edges = pack_edges()
    sizes = np.array(edges * 3, dtype=np.uint64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    seeds = (700 + np.arange(sizes.size)).astype(np.uint64)
    tmpl = fsb.fsb_config_init(1, 0, step=1.25, init_weight_mode=1)
    ts, state = make_state(offsets[-1])
    b = fsb.fsb_batch_create(tmpl, offsets, seeds, state, init=True)
    got_plan = fsb.fsb_batch_plan(b)
    assert got_plan["packed_schools"] == {w: 3 * [team_warps(n) for n in edges].count(w)
                                          for w in (8, 4, 2, 1)}
    if plan is not None:
        fsb.fsb_batch_set_plan(b, plan)
    stats = np.zeros(sizes.size * steps, fsb.STATS_DTYPE)
    fsb.fsb_batch_step(b, steps, stats)
    fsb.fsb_batch_destroy(b)
    check_batch(tmpl, offsets, seeds, read_state(ts), stats, steps, tmpl.precision)


@pytest.mark.parametrize("precision", [fsb.FSB_FP32, fsb.FSB_FP32_KAHAN, fsb.FSB_FP64_ACC])
def test_many_small_schools_more_than_the_warps(precision):
    """3000 schools of 1 to 600 fish (more than the GPU's fish warps), two
    calls: the teams of one warp run several schools each, and the second
    call loads the state the first one stored."""
    rng = np.random.default_rng(11)
    sizes = rng.integers(1, 601, 3000).astype(np.uint64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    seeds = (20_000 + np.arange(sizes.size)).astype(np.uint64)
    tmpl = fsb.fsb_config_init(1, 0, precision=precision)
    ts, state = make_state(offsets[-1])
    b = fsb.fsb_batch_create(tmpl, offsets, seeds, state, init=True)
    s1 = np.zeros(sizes.size * 3, fsb.STATS_DTYPE)
    s2 = np.zeros(sizes.size * 2, fsb.STATS_DTYPE)
    fsb.fsb_batch_step(b, 3, s1)
    fsb.fsb_batch_step(b, 2, s2)
    fsb.fsb_batch_destroy(b)
    stats = np.concatenate([np.concatenate([s1[k * 3:(k + 1) * 3], s2[k * 2:(k + 1) * 2]])
                            for k in range(sizes.size)])
    check_batch(tmpl, offsets, seeds, read_state(ts), stats, 5, precision)
