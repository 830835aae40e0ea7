"""The stand-alone eat() reduction (the paper's max over the school of
prevObjective - currentObjective) under each reduction construct: every
construct gives the exact maximum, and it equals the eat() statistic the
step reports."""
import numpy as np
import pytest

import paper_2507_20173_gb300 as fsb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_20173_gb300 import build
    build.build()
    fsb.lib()


@pytest.mark.parametrize("construct", [fsb.FSB_EAT_REDUCTION, fsb.FSB_EAT_PER_WARP,
                                       fsb.FSB_EAT_CRITICAL])
@pytest.mark.parametrize("n", [1, 3, 4, 5, 1023, 4096, 100_003, 1 << 20])
def test_every_construct_gives_the_exact_maximum(construct, n):
    rng = np.random.default_rng(n)
    prev = rng.uniform(0, 140, n).astype(np.float32)
    cur = (prev + rng.normal(0, 0.05, n)).astype(np.float32)
    if n > 10:
        cur[n // 3] = prev[n // 3] - 7.5  # a clear winner somewhere inside
    p, c = torch.from_numpy(prev).cuda(), torch.from_numpy(cur).cuda()
    got, ms = fsb.fsb_eat_max(p.data_ptr(), c.data_ptr(), n, construct)
    assert got == float(np.max(prev - cur))
    assert ms >= 0.0


def test_all_negative_differences():
    prev = np.full(777, 3.0, np.float32)
    cur = np.linspace(3.5, 9.0, 777).astype(np.float32)
    p, c = torch.from_numpy(prev).cuda(), torch.from_numpy(cur).cuda()
    for construct in (0, 1, 2):
        got, _ = fsb.fsb_eat_max(p.data_ptr(), c.data_ptr(), 777, construct)
        assert got == float(np.max(prev - cur))


def test_matches_the_step_statistic():
    cfg = fsb.fsb_config_init(300_001, 9, path=fsb.FSB_PATH_STREAM)
    s = fsb.School.create(cfg)
    st = s.step(4, stats=True)
    got = s.read()
    s.destroy()
    p = torch.from_numpy(got["prev"]).cuda()
    c = torch.from_numpy(got["cur"]).cuda()
    for construct in (0, 1, 2):
        v, _ = fsb.fsb_eat_max(p.data_ptr(), c.data_ptr(), cfg.n_fish, construct)
        assert v == st["eat_max_diff"][-1]


def test_rejects_bad_arguments():
    t = torch.zeros(8, device="cuda")
    with pytest.raises(fsb.FsbError):
        fsb.fsb_eat_max(t.data_ptr(), t.data_ptr(), 8, 7)
    with pytest.raises(fsb.FsbError):
        fsb.fsb_eat_max(t.data_ptr() + 4, t.data_ptr(), 4, 0)
