"""Pins of the CPU oracle against things other than itself.

The oracle (oracle/) is the definition the CUDA path is checked against, so it
is checked first against what the paper and the mathematics fix:

* Philox4x32-10 against Triton's library implementation (run on the CPU by
  Triton's interpreter), including the counter layout the school uses;
* hand-worked schools (tests/golden/*.txt) whose every value was worked out by
  hand on Pythagorean positions: swim, clamp at the bank, objective, delta,
  max, the paper's eat() statistic, feeding with cap and floor, barycentre;
* exact-arithmetic checks: the objective is the correctly rounded square root,
  the barycentre sums are the exact sums (Fractions / math.fsum);
* invariants and special cases: positions stay in the pond, weights stay in
  [w_min, w_max], a lone fish's weight moves by exactly +-1, a still school
  (s = 0) never eats, equal weights give the mean position, split runs equal
  one run, uniform draws.

All of these run on the CPU only.
"""
import json
import math
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


# ---------------------------------------------------------------- helpers --

def triton_philox(rows):
    """rows: [c0, c1, c2, c3, seed64] -> Triton's Philox4x32-10 words."""
    pytest.importorskip("triton")
    env = dict(os.environ, TRITON_INTERPRET="1")
    proc = subprocess.run([sys.executable, os.path.join(HERE, "triton_philox_ref.py")],
                          input=json.dumps(rows), capture_output=True, text=True,
                          env=env, timeout=600)
    if proc.returncode != 0:
        pytest.skip("Triton interpreter unavailable: " + proc.stderr[-300:])
    return json.loads(proc.stdout)


def round_to_binary(q: Fraction, mant_bits: int, emin: int) -> Fraction:
    """Nearest binary floating-point value (ties to even) to the rational q."""
    if q == 0:
        return Fraction(0)
    sign = -1 if q < 0 else 1
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    while Fraction(2) ** e > q:
        e -= 1
    while Fraction(2) ** (e + 1) <= q:
        e += 1
    e = max(e, emin)
    ulp = Fraction(2) ** (e - mant_bits + 1)
    n = q / ulp
    fl = n.numerator // n.denominator
    rem = n - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return sign * fl * ulp


F32 = (24, -126)
F64 = (53, -1022)


def is_correctly_rounded_sqrt(s_val, f_val, real):
    """f is the nearest binary value to sqrt(s) (sqrt never ties)."""
    s = Fraction(float(s_val))
    f = Fraction(float(f_val))
    if s == 0:
        return f == 0
    lo = Fraction(float(np.nextafter(real(f_val), real(-np.inf))))
    hi = Fraction(float(np.nextafter(real(f_val), real(np.inf))))
    mid_lo = (lo + f) / 2
    mid_hi = (f + hi) / 2
    return mid_lo * mid_lo < s < mid_hi * mid_hi


def parse_fixture(path):
    cfg = None
    init = {}
    steps = []
    for raw in open(path):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        tok = line.split()
        kv = {k: v for k, v in (t.split("=", 1) for t in tok[1:] if "=" in t)}
        if tok[0] == "config":
            cfg = oracle.Config(n_fish=int(kv["n_fish"]), pond_half=float(kv["pond_half"]),
                                step=float(kv["step"]), w0=float(kv["w0"]),
                                w_min=float(kv["w_min"]), w_max=float(kv["w_max"]),
                                swim_mode=int(kv.get("swim_mode", 0)),
                                feed_mode=int(kv.get("feed_mode", 0)),
                                collective_mode=int(kv.get("collective_mode", 0)),
                                step_vol=float(kv.get("step_vol", 0.1)))
        elif tok[0] == "init":
            init[int(tok[1])] = kv
        elif tok[0] == "step":
            steps.append({"draws": {}, "fish": {}, "stats": None})
        elif tok[0] == "draw":
            steps[-1]["draws"][int(tok[1])] = (int(tok[2], 16), int(tok[3], 16))
        elif tok[0] == "fish":
            steps[-1]["fish"][int(tok[1])] = kv
        elif tok[0] == "stats":
            steps[-1]["stats"] = kv
    return cfg, init, steps


FIELD = {"x": "x", "y": "y", "w": "weight", "prev": "prevObjective",
         "cur": "currentObjective"}


# ------------------------------------------------------------------ Philox --

def test_philox_matches_triton_library():
    rng = np.random.default_rng(2024)
    rows = []
    edge = [0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF]
    seeds = [0, 1, 2, 3, 1000, 0xFFFFFFFF, 1 << 32, 0xDEADBEEFCAFEF00D, (1 << 64) - 1]
    for seed in seeds:
        for _ in range(12):
            rows.append([int(v) for v in rng.integers(0, 1 << 32, 4)] + [seed])
        for e in edge:
            rows.append([e, e ^ 0x5A5A5A5A, e, 0, seed])
    ref = triton_philox(rows)
    for row, want in zip(rows, ref):
        c, seed = row[:4], row[4]
        got = oracle.philox4x32_10(c, [seed & 0xFFFFFFFF, seed >> 32])
        assert [int(v) for v in got] == want, (row, want, got)


def test_swim_and_init_counter_layout_matches_triton():
    """Reading of the paper's unnamed RNG: key = seed; counter = (index lo32,
    index hi32 ^ school, step, domain) with domain 0 = swim, 1 = init.  The
    init index is the fish; the swim index is the fish pair i // 2, fish 2p
    taking words 0, 1 and fish 2p + 1 words 2, 3."""
    cases = [(0, 0, 0, 1), (1, 7, 12345, 100), (2, 3, (1 << 32) + 5, 1),
             (0xFFFFFFFFFFFF, 0xFFFFFFFF, 3, 0xFFFFFFFF), (1003, 4095, 65535, 500),
             (5, 9, (1 << 33) + 1, 77), (6, 0, 1, 2)]
    rows, expect = [], []
    for seed, school, i, t in cases:
        cfg = oracle.Config(n_fish=1, seed=seed, school_id=school)
        p = i >> 1
        rows.append([p & 0xFFFFFFFF, ((p >> 32) ^ school) & 0xFFFFFFFF, t, 0, seed])
        expect.append(("swim", cfg, i, t))
        rows.append([i & 0xFFFFFFFF, ((i >> 32) ^ school) & 0xFFFFFFFF, 0, 1, seed])
        expect.append(("init", cfg, i, None))
    ref = triton_philox(rows)
    for (kind, cfg, i, t), want in zip(expect, ref):
        if kind == "swim":
            h = 2 * (i & 1)
            assert [int(v) for v in oracle.swim_words(cfg, i, t)] == want[h:h + 2]
        else:
            assert [int(v) for v in oracle.init_words(cfg, i)] == want[:3]


def test_fish_pair_shares_one_swim_block():
    """The two fish of a pair draw disjoint halves of one Philox block, and
    neighbouring pairs draw different blocks."""
    cfg = oracle.Config(n_fish=8, seed=123, school_id=4)
    for t in (1, 2, 1000):
        blocks = []
        for p in range(4):
            lo = oracle.swim_words(cfg, 2 * p, t)
            hi = oracle.swim_words(cfg, 2 * p + 1, t)
            c = [p, 4, t, 0]
            whole = oracle.philox4x32_10(c, [123, 0])
            assert list(lo) + list(hi) == list(whole)
            blocks.append(tuple(whole))
        assert len(set(blocks)) == 4


def test_philox_words_are_uniform():
    scipy_stats = pytest.importorskip("scipy.stats")
    cfg = oracle.Config(n_fish=1, seed=77)
    words = np.array([oracle.swim_words(cfg, i, t) for i in range(64)
                      for t in range(1, 257)], dtype=np.uint64).ravel()
    for shift in (28, 20, 8):
        bins = np.bincount(((words >> shift) & 0xF).astype(np.int64), minlength=16)
        assert scipy_stats.chisquare(bins).pvalue > 1e-6


# ------------------------------------------------------------ hand-worked --

@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("name", ["handworked_n3.txt", "handworked_bank.txt",
                                  "handworked_mapping.txt", "handworked_weighted_swim.txt",
                                  "handworked_paper_feeding.txt", "handworked_collective.txt"])
def test_handworked_fixture(name, precision):
    cfg, init, steps = parse_fixture(os.path.join(GOLDEN, name))
    dtype = oracle.FISH_F32 if precision == "f32" else oracle.FISH_F64
    real = np.float32 if precision == "f32" else np.float64
    school = np.zeros(cfg.n_fish, dtype=dtype)
    for i, kv in init.items():
        for k, v in kv.items():
            school[FIELD[k]][i] = real(Fraction(v))
    for k, st in enumerate(steps):
        draws = np.zeros((1, cfg.n_fish, 2), np.uint32)
        for i, (r0, r1) in st["draws"].items():
            draws[0, i] = (r0, r1)
        stats = oracle.run(cfg, school, k, 1, draws=draws)[0]
        for i, kv in st["fish"].items():
            for f, v in kv.items():
                got = Fraction(float(school[FIELD[f]][i]))
                assert got == Fraction(v), (name, k + 1, i, f, float(got), v)
        exp = st["stats"]
        names = {"M": "max_abs_delta", "E": "eat_max_diff", "S_w": "sum_w",
                 "S_x": "sum_wx", "S_y": "sum_wy", "A_x": "sum_abs_wx",
                 "A_y": "sum_abs_wy", "I_x": "inst_x", "I_y": "inst_y",
                 "B_x": "vol_bx", "B_y": "vol_by"}
        for key, field in names.items():
            if key in exp:
                assert Fraction(float(stats[field])) == Fraction(exp[key]), (name, k + 1, key)


# --------------------------------------------------------- exact checks --

@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_objective_is_correctly_rounded_distance(precision):
    """Sec. 2.1.1: objective = Euclidean distance to the pond centre, each
    operation rounded once (square, square, sum, square root)."""
    real = np.float32 if precision == "f32" else np.float64
    mant, emin = F32 if precision == "f32" else F64
    cfg = oracle.Config(n_fish=300, seed=11)
    school = oracle.init(cfg, precision)
    oracle.run(cfg, school, 0, 5)
    for f in school[:300]:
        x, y = Fraction(float(f["x"])), Fraction(float(f["y"]))
        s = round_to_binary(round_to_binary(x * x, mant, emin) +
                            round_to_binary(y * y, mant, emin), mant, emin)
        assert is_correctly_rounded_sqrt(float(s), f["currentObjective"], real)
        # three roundings before the square root leave a relative error
        # below 2u in the sum, halved by the root, plus the root's own u:
        # at most (2u + O(u^2)) of the true distance (u = half the epsilon)
        exact = math.hypot(float(x), float(y))
        u = float(np.finfo(real).eps) / 2
        assert abs(float(f["currentObjective"]) - exact) <= 2.001 * u * exact


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_swim_is_rounded_uniform_move_clamped_to_pond(precision):
    """Sec. 2.1.2: each step moves a fish by ((2u0-1)s, (2u1-1)s) with the
    step's draws, rounded once per operation, clamped to the bank."""
    real = np.float32 if precision == "f32" else np.float64
    mant, emin = F32 if precision == "f32" else F64
    cfg = oracle.Config(n_fish=64, seed=5, step=3.0, pond_half=10.0)
    school = oracle.init(cfg, precision)
    for t in range(1, 21):
        before = school.copy()
        oracle.run(cfg, school, t - 1, 1)
        for i in range(cfg.n_fish):
            r = oracle.swim_words(cfg, i, t)
            for coord, word in (("x", r[0]), ("y", r[1])):
                d = Fraction(int(word) >> 8, 1 << 23) - 1          # 2u - 1, exact
                mv = round_to_binary(d * Fraction(float(real(cfg.step))), mant, emin)
                v = round_to_binary(Fraction(float(before[coord][i])) + mv, mant, emin)
                P = Fraction(float(real(cfg.pond_half)))
                v = min(max(v, -P), P)
                assert Fraction(float(school[coord][i])) == v
                assert abs(float(school[coord][i])) <= cfg.pond_half


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_init_inverts_to_the_draw_words(precision):
    """With P = 128 the initial position is exactly (2u - 1) * 128, so the
    draw word's top 24 bits can be read back from it."""
    cfg = oracle.Config(n_fish=500, seed=9, pond_half=128.0, init_weight_mode=1, w0=1.0)
    school = oracle.init(cfg, precision)
    for i in range(cfg.n_fish):
        r = oracle.init_words(cfg, i)
        for coord, word in (("x", r[0]), ("y", r[1])):
            v = Fraction(float(school[coord][i])) / 128
            assert (v + 1) * (1 << 23) == int(word) >> 8
        u2 = Fraction(int(r[2]) >> 8, 1 << 24)
        w = Fraction(float(school["weight"][i]))
        assert Fraction(1, 2) <= w < Fraction(3, 2)
        assert abs(w - (Fraction(1, 2) + u2)) <= Fraction(1, 1 << 24)
        assert school["prevObjective"][i] == school["currentObjective"][i]


def test_init_is_uniform_over_the_pond():
    scipy_stats = pytest.importorskip("scipy.stats")
    cfg = oracle.Config(n_fish=40000, seed=0)
    school = oracle.init(cfg)
    for coord in ("x", "y"):
        v = school[coord].astype(np.float64)
        assert v.min() >= -100.0 and v.max() < 100.0
        bins = np.histogram(v, bins=20, range=(-100, 100))[0]
        assert scipy_stats.chisquare(bins).pvalue > 1e-6
    assert np.all(school["weight"] == 1.0)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_max_and_eat_statistic_equal_brute_force(precision):
    """Sec. 2.3.2: eat() reduces max over the school; M_t = max|cur - prev|
    and the paper's max(prev - cur), recomputed by numpy from the state."""
    cfg = oracle.Config(n_fish=2000, seed=3)
    school = oracle.init(cfg, precision)
    for t in range(1, 16):
        st = oracle.run(cfg, school, t - 1, 1)[0]
        delta = school["currentObjective"] - school["prevObjective"]
        assert st["max_abs_delta"] == np.max(np.abs(delta))
        assert st["eat_max_diff"] == np.max(school["prevObjective"] - school["currentObjective"])
        # normalisation: some fish has |delta / M| exactly 1, none above
        q = np.abs(delta) / delta.dtype.type(st["max_abs_delta"])
        assert q.max() == 1.0


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_barycentre_sums_are_exact_sums(precision):
    mant, emin = F32 if precision == "f32" else F64
    cfg = oracle.Config(n_fish=700, seed=21, init_weight_mode=1)
    school = oracle.init(cfg, precision)
    for t in range(1, 6):
        st = oracle.run(cfg, school, t - 1, 1)[0]
        w = [Fraction(float(v)) for v in school["weight"]]
        x = [Fraction(float(v)) for v in school["x"]]
        y = [Fraction(float(v)) for v in school["y"]]
        exact = {"sum_w": sum(w), "sum_wx": sum(a * b for a, b in zip(w, x)),
                 "sum_wy": sum(a * b for a, b in zip(w, y)),
                 "sum_abs_wx": sum(a * abs(b) for a, b in zip(w, x)),
                 "sum_abs_wy": sum(a * abs(b) for a, b in zip(w, y))}
        scale = {"sum_w": exact["sum_w"], "sum_wx": exact["sum_abs_wx"],
                 "sum_wy": exact["sum_abs_wy"], "sum_abs_wx": exact["sum_abs_wx"],
                 "sum_abs_wy": exact["sum_abs_wy"]}
        for k, v in exact.items():
            err = abs(Fraction(float(st[k])) - v)
            assert err <= Fraction(1, 1 << 50) * scale[k], (k, float(err))
        # math.fsum of the binary64 products is the correctly rounded exact
        # sum when the products are exact (binary32 state)
        if precision == "f32":
            ws = school["weight"].astype(np.float64)
            assert st["sum_wx"] == math.fsum(ws * school["x"].astype(np.float64))


# -------------------------------------------------- invariants / specials --

@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_state_stays_in_pond_and_weights_in_cap(precision):
    cfg = oracle.Config(n_fish=3000, seed=4, step=5.0, init_weight_mode=1)
    school = oracle.init(cfg, precision)
    oracle.run(cfg, school, 0, 60)
    assert np.all(np.abs(school["x"]) <= 100.0)
    assert np.all(np.abs(school["y"]) <= 100.0)
    assert np.all(school["weight"] >= 0.0) and np.all(school["weight"] <= 2.0)
    assert np.sum(np.abs(school["x"]) == 100.0) > 0      # some fish met the bank


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_single_fish_weight_moves_by_exactly_one(precision):
    """N = 1: delta / M = sign(delta), so the weight walks 0, 1, 2 in unit
    steps (w0 = 1, cap 2, floor 0), and the barycentre is the fish."""
    cfg = oracle.Config(n_fish=1, seed=123, step=2.0)
    school = oracle.init(cfg, precision)
    w = 1.0
    for t in range(1, 201):
        st = oracle.run(cfg, school, t - 1, 1)[0]
        d = float(school["currentObjective"][0] - school["prevObjective"][0])
        if d != 0.0:
            w = min(max(w + math.copysign(1.0, d), 0.0), 2.0)
        assert float(school["weight"][0]) == w
        if w > 0:
            assert st["sum_wx"] / st["sum_w"] == float(school["x"][0])
            assert st["sum_wy"] / st["sum_w"] == float(school["y"][0])


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_still_school_never_eats(precision):
    cfg = oracle.Config(n_fish=50, seed=8, step=0.0, init_weight_mode=1)
    school = oracle.init(cfg, precision)
    start = school.copy()
    stats = oracle.run(cfg, school, 0, 10)
    assert np.all(stats["max_abs_delta"] == 0.0)
    for f in ("x", "y", "weight", "currentObjective"):
        assert np.array_equal(school[f], start[f])


def test_equal_weights_give_mean_position():
    cfg = oracle.Config(n_fish=999, seed=10, w_min=1.0, w_max=1.0)
    school = oracle.init(cfg)
    stats = oracle.run(cfg, school, 0, 3)
    xs = school["x"].astype(np.float64)
    assert stats[-1]["sum_w"] == cfg.n_fish
    assert abs(stats[-1]["sum_wx"] / stats[-1]["sum_w"] - math.fsum(xs) / cfg.n_fish) < 1e-12


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_split_run_equals_one_run(precision):
    cfg = oracle.Config(n_fish=257, seed=31, school_id=5)
    a = oracle.init(cfg, precision)
    b = a.copy()
    sa = oracle.run(cfg, a, 0, 30)
    sb1 = oracle.run(cfg, b, 0, 13)
    sb2 = oracle.run(cfg, b, 13, 17)
    assert np.array_equal(a, b)
    assert np.array_equal(sa, np.concatenate([sb1, sb2]))


def test_track_and_eat_fish_follow_the_school():
    """The single-fish helpers used for sampled parity at large sizes agree
    with the whole-school run."""
    cfg = oracle.Config(n_fish=100, seed=42)
    school = oracle.init(cfg)
    start = school.copy()
    stats = oracle.run(cfg, school, 0, 25)
    for i in (0, 17, 99):
        xs, ys, ds, fish = oracle.track_fish(cfg, i, 0, 25, start[i:i + 1].copy())
        assert xs[-1] == school["x"][i] and ys[-1] == school["y"][i]
        assert fish["prevObjective"][0] == school["prevObjective"][i]
        ws = oracle.eat_fish(cfg, float(start["weight"][i]), ds, stats["max_abs_delta"])
        assert ws[-1] == school["weight"][i]


def test_binary32_and_binary64_trajectories_stay_close():
    """Trajectory precision is measured, not pinned ("parity unpinned"):
    the binary32 and binary64 schools draw the same numbers, so they only
    drift apart by rounding."""
    cfg = oracle.Config(n_fish=500, seed=1)
    s32 = oracle.init(cfg, "f32")
    s64 = oracle.init(cfg, "f64")
    oracle.run(cfg, s32, 0, 100)
    oracle.run(cfg, s64, 0, 100)
    assert np.max(np.abs(s32["x"] - s64["x"])) < 1e-3
    assert np.max(np.abs(s32["weight"] - s64["weight"])) < 0.25


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_weighted_swim_bounds_each_move_by_its_weight(precision):
    """Swim mode 1: each coordinate's move is at most s * w / w0 (plus one
    rounding), a fish of weight 0 never moves, and positions stay in the
    pond."""
    cfg = oracle.Config(n_fish=2000, seed=13, step=2.0, swim_mode=1, init_weight_mode=1,
                        w0=4.0, w_max=8.0)
    school = oracle.init(cfg, precision)
    for t in range(1, 31):
        before = school.copy()
        oracle.run(cfg, school, t - 1, 1)
        lim = cfg.step * before["weight"].astype(np.float64) / cfg.w0
        for c in ("x", "y"):
            mv = np.abs(school[c].astype(np.float64) - before[c].astype(np.float64))
            assert np.all(mv <= lim * (1 + 1e-6) + 1e-5)
            assert np.all(np.abs(school[c]) <= cfg.pond_half)
        # the largest moves use most of the allowed width (uniform draws)
        assert np.max(np.abs(school["x"].astype(np.float64) - before["x"]) / lim) > 0.9
        frozen = before["weight"] == 0
        assert np.array_equal(school["x"][frozen], before["x"][frozen])


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_paper_feeding_normaliser_is_the_eat_statistic(precision):
    """Feed mode 1: the normaliser is the reported eat() value; when it is
    positive the best improver's weight rises by exactly 1 (or hits the cap),
    otherwise no weight changes."""
    cfg = oracle.Config(n_fish=500, seed=17, step=1.0, feed_mode=1, w_max=1e9)
    school = oracle.init(cfg, precision)
    for t in range(1, 21):
        before = school["weight"].copy()
        st = oracle.run(cfg, school, t - 1, 1)[0]
        g = school["prevObjective"] - school["currentObjective"]
        assert st["eat_max_diff"] == np.max(g)
        if st["eat_max_diff"] > 0:
            best = np.argmax(g)
            assert school["weight"][best] == before[best] + 1
        else:
            assert np.array_equal(school["weight"], before)


def test_bad_configuration_is_rejected():
    with pytest.raises(ValueError):
        oracle.init(oracle.Config(n_fish=0))
    with pytest.raises(ValueError):
        oracle.init(oracle.Config(n_fish=4, w_min=2.0, w_max=1.0))
    with pytest.raises(ValueError):
        oracle.init(oracle.Config(n_fish=4, swim_mode=2))
    with pytest.raises(ValueError):
        oracle.init(oracle.Config(n_fish=4, feed_mode=3))


# ------------------------------------------------- collective movements --
# (fish-school search variant, collective_mode 1; not in the paper)

def test_grid_exponent_is_the_largest_safe_power_of_two():
    """The grid exponent of an exact school sum is the largest k (capped at
    +-100) with n * bound * 2^k <= 2^62 (the sum of n terms stays below
    2^62), checked in exact arithmetic on the binary64 value of n * bound the
    oracle starts from."""
    lim = Fraction(2) ** 62
    cases = [(1, 1.0), (2, 512.0061), (1000, 0.0141), (1 << 28, 0.02), (1 << 32, 3.5),
             (7, 1e-30), (3, 1e30), (1 << 40, 1e10), (5, 0.0)]
    for n, b in cases:
        k = oracle.grid_exponent(n, b)
        t = Fraction(float(n) * b)
        assert -100 <= k <= 100
        if t == 0:
            assert k == 100
            continue
        if k < 100:
            assert t * Fraction(2) ** (k + 1) > lim, (n, b, k)
        if k > -100:
            assert t * Fraction(2) ** k <= lim, (n, b, k)


def test_volitive_draw_counter_layout_matches_triton():
    """Domain 2 holds the volitive draws, indexed by the fish pair: fish 2p
    takes word 0 and fish 2p + 1 word 1 of the pair's block."""
    cases = [(9, 0, 0, 1), (9, 0, 1, 1), (123, 5, 77, 40), (123, 5, 76, 40),
             ((1 << 40) + 7, 11, (1 << 33) + 3, 9)]
    rows = []
    for seed, school, i, t in cases:
        p = i >> 1
        rows.append([p & 0xFFFFFFFF, ((p >> 32) ^ school) & 0xFFFFFFFF, t, 2, seed])
    ref = triton_philox(rows)
    for (seed, school, i, t), want in zip(cases, ref):
        cfg = oracle.Config(n_fish=1, seed=seed, school_id=school)
        assert oracle.volitive_word(cfg, i, t) == want[i & 1]


def _grids(cfg):
    """Grid exponents of the collective sums, from the bounds of the
    configuration (products dx * g, improvements g, weights)."""
    a = max(abs(cfg.w_min), abs(cfg.w_max), 1.5 * abs(cfg.w0))
    sm = 2.0 * cfg.step * max(1.0, a / cfg.w0) if cfg.swim_mode == 1 else 2.0 * cfg.step
    bd = sm + math.ldexp(1.0, -20) * max(cfg.pond_half, 1.0)
    return (oracle.grid_exponent(cfg.n_fish, 2.0 * bd * bd),
            oracle.grid_exponent(cfg.n_fish, 2.0 * bd),
            oracle.grid_exponent(cfg.n_fish, 2.0 * a * max(cfg.pond_half, 1.0)))


def _coll_cfg(n, **kw):
    base = dict(n_fish=n, seed=21, collective_mode=1, step=2.0, init_weight_mode=1)
    base.update(kw)
    return oracle.Config(**base)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_collective_sums_do_not_depend_on_fish_order(precision):
    """The instinctive vector and the barycentre come from exact grid sums,
    so reordering the school (with each fish keeping its draws) changes
    nothing: same vector, same barycentre, same per-fish states."""
    n, steps = 97, 4
    cfg = _coll_cfg(n, step_vol=0.0)
    rng = np.random.default_rng(5)
    draws = rng.integers(0, 1 << 32, (steps, n, 2), dtype=np.uint64).astype(np.uint32)
    a = oracle.init(cfg, precision)
    perm = rng.permutation(n)
    b = a[perm].copy()
    sa = oracle.run(cfg, a, 0, steps, draws=draws)
    sb = oracle.run(cfg, b, 0, steps, draws=draws[:, perm, :])
    for f in ("inst_x", "inst_y", "vol_bx", "vol_by", "vol_dw", "max_abs_delta"):
        assert np.array_equal(sa[f], sb[f]), f
    assert np.array_equal(a[perm], b)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_volitive_move_is_radial_by_s_vol_u(precision):
    """Against the same step with a volitive step of 0, each fish moves along
    the line through the barycentre B the step reports, by s_vol * u with
    its own draw u, toward B when the school's weight sum grew and away from
    it otherwise (fish clamped at the bank excluded)."""
    n, s_vol = 400, 0.7
    cfg0 = _coll_cfg(n, step_vol=0.0, pond_half=100.0)
    cfg1 = _coll_cfg(n, step_vol=s_vol, pond_half=100.0)
    a = oracle.init(cfg0, precision)
    b = a.copy()
    st = oracle.run(cfg0, a, 0, 1)[0]
    st1 = oracle.run(cfg1, b, 0, 1)[0]
    assert st["vol_bx"] == st1["vol_bx"] and st["vol_by"] == st1["vol_by"]
    bx, by = float(st["vol_bx"]), float(st["vol_by"])
    toward = st["vol_dw"] > 0
    tol = 8 * float(np.spacing(np.float32(100.0) if precision == "f32" else np.float64(100.0)))
    checked = 0
    for i in range(n):
        if max(abs(b["x"][i]), abs(b["y"][i])) >= 100.0:
            continue
        vx, vy = float(a["x"][i]) - bx, float(a["y"][i]) - by
        dx, dy = float(b["x"][i]) - float(a["x"][i]), float(b["y"][i]) - float(a["y"][i])
        dist = math.hypot(vx, vy)
        u = (oracle.volitive_word(cfg1, i, 1) >> 8) * 2.0 ** -24
        assert abs(math.hypot(dx, dy) - s_vol * u) <= tol, i
        assert abs(vx * dy - vy * dx) <= tol * dist, i
        assert (vx * dx + vy * dy < 0) == toward or math.hypot(dx, dy) <= tol, i
        checked += 1
    assert checked > n // 2


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_lone_fish_follows_its_own_improvement(precision):
    """N = 1: when the fish improves, the instinctive vector is its own swim
    displacement (up to the rounding of dx * g on the grid), and the fish is
    its own barycentre (or weighs 0), so it makes no volitive move."""
    real = np.float32 if precision == "f32" else np.float64
    cfg = _coll_cfg(1, step_vol=0.9, step=3.0)
    plain = oracle.Config(**{**cfg.__dict__, "collective_mode": 0})
    seen = 0
    for t in range(60):
        a = oracle.init(cfg, precision)
        oracle.run(cfg, a, 0, t)                  # advance to step t
        ref = a.copy()
        oracle.run(plain, ref, t, 1)              # the swim alone
        st = oracle.run(cfg, a, t, 1)[0]
        g = float(ref["prevObjective"][0]) - float(ref["currentObjective"][0])
        if g <= 0:
            assert st["inst_x"] == 0 and st["inst_y"] == 0
            continue
        seen += 1
        before = oracle.init(cfg, precision)
        oracle.run(cfg, before, 0, t)
        dx = float(ref["x"][0]) - float(before["x"][0])
        # grid quantisation: each grid term is within half a grid unit
        kp, kg = _grids(cfg)[:2]
        quant = (2.0 ** -(kp + 1) + abs(dx) * 2.0 ** -(kg + 1)) / g
        assert abs(st["inst_x"] - dx) <= 1.01 * quant + 4 * float(np.spacing(real(abs(dx) + 1e-30)))
        # no volitive move: the fish is its own barycentre, or weighs 0
        # (then the weight sum is 0 and no barycentre is defined)
        moved = np.clip(real(ref["x"][0]) + real(st["inst_x"]), -cfg.pond_half, cfg.pond_half)
        assert a["x"][0] == moved
        if a["weight"][0] != 0:
            assert st["vol_bx"] == float(a["x"][0]) and st["vol_by"] == float(a["y"][0])
        else:
            assert st["vol_bx"] == 0 and st["vol_by"] == 0
    assert seen > 5


def test_no_improving_fish_means_no_instinctive_move():
    """If every fish's objective worsens, the instinctive vector is 0 and,
    with a volitive step of 0, the school ends where the swim left it."""
    n = 16
    cfg = _coll_cfg(n, step_vol=0.0, step=1.0, pond_half=100.0)
    school = oracle.init(cfg)
    # move every fish outward: dx with the sign of x, dy with the sign of y
    draws = np.zeros((1, n, 2), np.uint32)
    for i in range(n):
        draws[0, i, 0] = 0xFFFFFF00 if school["x"][i] >= 0 else 0
        draws[0, i, 1] = 0xFFFFFF00 if school["y"][i] >= 0 else 0
    plain = oracle.Config(**{**cfg.__dict__, "collective_mode": 0})
    ref = school.copy()
    oracle.run(plain, ref, 0, 1, draws=draws)
    st = oracle.run(cfg, school, 0, 1, draws=draws)[0]
    assert np.all(ref["currentObjective"] > ref["prevObjective"])
    assert st["inst_x"] == 0 and st["inst_y"] == 0
    assert np.array_equal(school["x"], ref["x"]) and np.array_equal(school["y"], ref["y"])
