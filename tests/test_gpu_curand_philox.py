"""The oracle's Philox4x32-10 and its counter layout against cuRAND's device
Philox4_32_10, a library implementation it shares no code with (Salmon et
al., SC'11; the generator the method's random moves are drawn from, reading
R10).  A small CUDA helper (tests/curand_philox.cu) calls curand_init and
curand4 for each key and counter."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

_HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_words():
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib_path = os.path.join(out_dir, "libcurand_philox.so")
    src = os.path.join(_HERE, "curand_philox.cu")
    if not os.path.exists(lib_path) or os.path.getmtime(lib_path) < os.path.getmtime(src):
        tmp = lib_path + ".tmp%d" % os.getpid()
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                        "-Xcompiler", "-fPIC", src, "-o", tmp], check=True)
        os.replace(tmp, lib_path)
    L = ctypes.CDLL(lib_path)
    P = ctypes.c_void_p
    L.curand_philox_words.argtypes = [P, P, P, P, ctypes.c_int]
    L.curand_philox_words.restype = ctypes.c_int

    def words(seeds, ctr_lo, ctr_hi):
        seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        ctr_lo = np.ascontiguousarray(ctr_lo, dtype=np.uint64)
        ctr_hi = np.ascontiguousarray(ctr_hi, dtype=np.uint64)
        assert np.all(ctr_lo < np.uint64(1 << 62))
        out = np.zeros((seeds.size, 4), dtype=np.uint32)
        rc = L.curand_philox_words(seeds.ctypes.data, ctr_lo.ctypes.data, ctr_hi.ctypes.data,
                                   out.ctypes.data, seeds.size)
        assert rc == 0, "CUDA error %d" % rc
        return out
    return words


def _split(v):
    v = int(v)
    return v & 0xFFFFFFFF, v >> 32


def test_philox_block_matches_curand(curand_words):
    rng = np.random.default_rng(2507)
    seeds = [0, 1, 2, 0xFFFFFFFF, 1 << 32, (1 << 64) - 1, 0x0123456789ABCDEF]
    seeds += [int(s) for s in rng.integers(0, 1 << 63, 9, dtype=np.uint64)]
    lows = [0, 1, 2, 0xFFFFFFFF, 1 << 32, (1 << 62) - 1]
    lows += [int(c) for c in rng.integers(0, 1 << 62, 10, dtype=np.uint64)]
    highs = [0, 1, 0xFFFFFFFF, 1 << 32, (1 << 64) - 1]
    highs += [int(c) for c in rng.integers(0, 1 << 63, 5, dtype=np.uint64)]
    cases = [(s, lo, hi) for s in seeds for lo in lows for hi in highs]
    got = curand_words([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases])
    for (s, lo, hi), g in zip(cases, got):
        ctr = [*_split(lo), *_split(hi)]
        key = list(_split(s))
        assert np.array_equal(oracle.philox4x32_10(ctr, key), g), (s, lo, hi)


def test_school_counter_layout_matches_curand(curand_words):
    """Swim draws of fish i at step t: half i % 2 of the block at counter
    (pair lo32, pair hi32 xor school, t, 0); init draws: words 0-2 of the
    block at (i lo32, i hi32 xor school, 0, 1); volitive draw: word i % 2
    of the block at (pair lo32, pair hi32 xor school, t, 2)."""
    rng = np.random.default_rng(3)
    fish = [0, 1, 2, 3, 1001, (1 << 32) - 1, 1 << 32, (1 << 32) + 1, (1 << 40) + 7]
    fish += [int(v) for v in rng.integers(0, 1 << 45, 12, dtype=np.uint64)]
    for seed, school in ((0, 0), (2, 0), (1000 + 17, 17), ((1 << 64) - 1, 4095)):
        cfg = oracle.Config(n_fish=1, seed=seed, school_id=school)
        for t in (1, 2, 100, 0xFFFFFFFF):
            pairs = [i >> 1 for i in fish]
            lo = [(p & 0xFFFFFFFF) | (((p >> 32) ^ school) << 32) for p in pairs]
            swim = curand_words([seed] * len(fish), lo, [t] * len(fish))
            vol = curand_words([seed] * len(fish), lo, [t | (2 << 32)] * len(fish))
            for k, i in enumerate(fish):
                h = i & 1
                assert np.array_equal(oracle.swim_words(cfg, i, t), swim[k, 2 * h:2 * h + 2])
                assert oracle.volitive_word(cfg, i, t) == int(vol[k, h])
        lo = [(i & 0xFFFFFFFF) | (((i >> 32) ^ school) << 32) for i in fish]
        init = curand_words([seed] * len(fish), lo, [1 << 32] * len(fish))
        for k, i in enumerate(fish):
            assert np.array_equal(oracle.init_words(cfg, i), init[k, :3])
