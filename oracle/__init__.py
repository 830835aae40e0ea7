"""CPU oracle of the Fish School Behaviour per-step update.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library in ``paper_2507_20173_gb300``; the two
meet only through the seeded workload generators, which hold none of the
method's arithmetic.

The arithmetic lives in plain C (``fsb_oracle.c``, ``philox.c``), built with
``-O2 -ffp-contract=off -fno-fast-math`` so that every binary32 / binary64
operation rounds once, to nearest-even.  This module only marshals numpy
arrays into it.  ``run_omp`` is the same step with its per-fish loops on
OpenMP threads (the paper's own parallelisation), a multi-core CPU baseline
for ``bench.py``; ``run`` stays the reference every test compares against.

Paper passages followed: Sec. 2.1.1 (Fish structure, initialisation,
objective = distance to the pond centre), Sec. 2.1.2 (200x200 pond, random
movement), Sec. 2.1.3 (Config), Sec. 2.3.2 (the eat() max reduction).  The
readings taken where the paper is silent are written out in ``fsb_oracle.c``.

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py``
(library Philox, exact rounding checks, hand-worked cases, invariants).  The
one measured-only quantity, the drift between the binary32 and binary64
trajectories, is "parity unpinned": it is reported, not asserted.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfsb_oracle.so")
_SOURCES = ("philox.c", "collective.c", "fsb_oracle.c", "fsb_oracle.h")

CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
          "-fPIC", "-Wall", "-Wextra"]

FISH_F32 = np.dtype([("x", "<f4"), ("y", "<f4"), ("weight", "<f4"),
                     ("prevObjective", "<f4"), ("currentObjective", "<f4")])
FISH_F64 = np.dtype([("x", "<f8"), ("y", "<f8"), ("weight", "<f8"),
                     ("prevObjective", "<f8"), ("currentObjective", "<f8")])
STATS = np.dtype([("max_abs_delta", "<f8"), ("eat_max_diff", "<f8"),
                  ("sum_w", "<f8"), ("sum_wx", "<f8"), ("sum_wy", "<f8"),
                  ("sum_abs_wx", "<f8"), ("sum_abs_wy", "<f8"),
                  ("inst_x", "<f8"), ("inst_y", "<f8"), ("vol_bx", "<f8"),
                  ("vol_by", "<f8"), ("vol_dw", "<f8")])


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libfsb_oracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    newest_src = max(os.path.getmtime(os.path.join(_HERE, s)) for s in _SOURCES)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= newest_src):
        return _LIB_PATH
    objs = []
    # -fopenmp only enables fsbo_run_omp_*, the multi-core baseline; the
    # serial functions carry no OpenMP construct
    units = [("philox.c", [], "philox.o"), ("collective.c", [], "collective.o"),
             ("fsb_oracle.c", ["-DFSBO_REAL=float", "-DFSBO_SFX=f32", "-fopenmp"],
              "oracle_f32.o"),
             ("fsb_oracle.c", ["-DFSBO_REAL=double", "-DFSBO_SFX=f64", "-fopenmp"],
              "oracle_f64.o")]
    for src, defs, obj in units:
        out = os.path.join(_BUILD, obj)
        subprocess.run(["gcc", *CFLAGS, *defs, "-c", os.path.join(_HERE, src),
                        "-o", out], check=True)
        objs.append(out)
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.run(["gcc", "-shared", "-fopenmp", *objs, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CConfig(ctypes.Structure):
    _fields_ = [("n_fish", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("school_id", ctypes.c_uint32), ("init_weight_mode", ctypes.c_int32),
                ("pond_half", ctypes.c_double), ("step", ctypes.c_double),
                ("w0", ctypes.c_double), ("w_min", ctypes.c_double),
                ("w_max", ctypes.c_double), ("swim_mode", ctypes.c_int32),
                ("feed_mode", ctypes.c_int32), ("collective_mode", ctypes.c_int32),
                ("step_vol", ctypes.c_double)]


@dataclass
class Config:
    """Sec. 2.1.3 Config (physics fields) plus the generator key."""
    n_fish: int
    seed: int = 0
    school_id: int = 0
    init_weight_mode: int = 0
    pond_half: float = 100.0
    step: float = 0.1
    w0: float = 1.0
    w_min: float = 0.0
    w_max: float = 2.0
    swim_mode: int = 0     # 1: half-width s * (w / w0) (weight-scaled swim)
    feed_mode: int = 0     # 1: normalise feeding by the paper's max(prev - cur)
    collective_mode: int = 0   # 1: instinctive and volitive movements
    step_vol: float = 0.1      # volitive step

    def c(self) -> _CConfig:
        return _CConfig(self.n_fish, self.seed, self.school_id,
                        self.init_weight_mode, self.pond_half, self.step,
                        self.w0, self.w_min, self.w_max, self.swim_mode,
                        self.feed_mode, self.collective_mode, self.step_vol)


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        cfgp = ctypes.POINTER(_CConfig)
        L.fsbo_philox4x32_10.argtypes = [P, P, P]
        L.fsbo_swim_words.argtypes = [cfgp, ctypes.c_uint64, ctypes.c_uint32, P]
        L.fsbo_init_words.argtypes = [cfgp, ctypes.c_uint64, P]
        L.fsbo_volitive_word.argtypes = [cfgp, ctypes.c_uint64, ctypes.c_uint32]
        L.fsbo_volitive_word.restype = ctypes.c_uint32
        L.fsbo_grid_exponent.argtypes = [ctypes.c_uint64, ctypes.c_double]
        L.fsbo_grid_exponent.restype = ctypes.c_int
        for sfx in ("f32", "f64"):
            getattr(L, "fsbo_init_" + sfx).argtypes = [cfgp, P]
            getattr(L, "fsbo_init_" + sfx).restype = ctypes.c_int
            getattr(L, "fsbo_run_" + sfx).argtypes = [cfgp, ctypes.c_uint64,
                                                      ctypes.c_uint32, P, P, P]
            getattr(L, "fsbo_run_" + sfx).restype = ctypes.c_int
            getattr(L, "fsbo_run_omp_" + sfx).argtypes = [cfgp, ctypes.c_uint64,
                                                          ctypes.c_uint32, P, P, ctypes.c_int]
            getattr(L, "fsbo_run_omp_" + sfx).restype = ctypes.c_int
            getattr(L, "fsbo_track_fish_" + sfx).argtypes = [
                cfgp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, P, P, P, P]
        L.fsbo_eat_fish_f32.argtypes = [cfgp, ctypes.c_float, ctypes.c_uint32, P, P, P]
        L.fsbo_eat_fish_f32.restype = ctypes.c_float
        L.fsbo_eat_fish_f64.argtypes = [cfgp, ctypes.c_double, ctypes.c_uint32, P, P, P]
        L.fsbo_eat_fish_f64.restype = ctypes.c_double
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _fish_dtype(precision: str):
    if precision not in ("f32", "f64"):
        raise ValueError("precision must be 'f32' or 'f64'")
    return FISH_F32 if precision == "f32" else FISH_F64


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().fsbo_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def swim_words(cfg: Config, i: int, t: int) -> np.ndarray:
    out = np.zeros(2, dtype=np.uint32)
    c = cfg.c()
    lib().fsbo_swim_words(ctypes.byref(c), i, t, _ptr(out))
    return out


def init_words(cfg: Config, i: int) -> np.ndarray:
    out = np.zeros(3, dtype=np.uint32)
    c = cfg.c()
    lib().fsbo_init_words(ctypes.byref(c), i, _ptr(out))
    return out


def volitive_word(cfg: Config, i: int, t: int) -> int:
    c = cfg.c()
    return int(lib().fsbo_volitive_word(ctypes.byref(c), i, t))


def grid_exponent(n: int, bound: float) -> int:
    return int(lib().fsbo_grid_exponent(n, bound))


def init(cfg: Config, precision: str = "f32") -> np.ndarray:
    """The school at t = 0 (Sec. 2.1.1), as an array of Fish records."""
    school = np.zeros(cfg.n_fish, dtype=_fish_dtype(precision))
    c = cfg.c()
    rc = getattr(lib(), "fsbo_init_" + precision)(ctypes.byref(c), _ptr(school))
    if rc != 0:
        raise ValueError("oracle rejected the configuration")
    return school


def run(cfg: Config, school: np.ndarray, t0: int, n_steps: int,
        draws: np.ndarray | None = None) -> np.ndarray:
    """Advance `school` in place from step t0 by n_steps; returns the
    per-step statistics.  `draws` (n_steps, n_fish, 2) uint32 replaces the
    generator (test hook)."""
    precision = "f32" if school.dtype == FISH_F32 else "f64"
    assert school.dtype == _fish_dtype(precision) and school.size == cfg.n_fish
    stats = np.zeros(n_steps, dtype=STATS)
    dptr = None
    if draws is not None:
        draws = np.ascontiguousarray(draws, dtype=np.uint32)
        assert draws.shape == (n_steps, cfg.n_fish, 2)
        dptr = _ptr(draws)
    c = cfg.c()
    rc = getattr(lib(), "fsbo_run_" + precision)(
        ctypes.byref(c), t0, n_steps, _ptr(school), _ptr(stats), dptr)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return stats


def run_omp(cfg: Config, school: np.ndarray, t0: int, n_steps: int,
            threads: int = 0) -> np.ndarray:
    """``run`` with the per-fish loops on ``threads`` OpenMP threads (0: the
    OpenMP default), the paper's own parallelisation (Sec. 2.3) as a
    multi-core CPU baseline.  Same per-fish state and maxima as ``run``;
    barycentre sums equal to rounding."""
    precision = "f32" if school.dtype == FISH_F32 else "f64"
    assert school.dtype == _fish_dtype(precision) and school.size == cfg.n_fish
    stats = np.zeros(n_steps, dtype=STATS)
    c = cfg.c()
    rc = getattr(lib(), "fsbo_run_omp_" + precision)(
        ctypes.byref(c), t0, n_steps, _ptr(school), _ptr(stats), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return stats


def track_fish(cfg: Config, i: int, t0: int, n_steps: int, fish: np.ndarray):
    """Positions and deltas of fish i for steps t0+1 .. t0+n_steps, starting
    from the one-element Fish record `fish` (advanced in place)."""
    precision = "f32" if fish.dtype == FISH_F32 else "f64"
    real = np.float32 if precision == "f32" else np.float64
    fish = np.ascontiguousarray(fish)
    xs = np.zeros(n_steps, real)
    ys = np.zeros(n_steps, real)
    ds = np.zeros(n_steps, real)
    c = cfg.c()
    getattr(lib(), "fsbo_track_fish_" + precision)(
        ctypes.byref(c), i, t0, n_steps, _ptr(fish), _ptr(xs), _ptr(ys), _ptr(ds))
    return xs, ys, ds, fish


def eat_fish(cfg: Config, w: float, delta: np.ndarray, max_abs_delta: np.ndarray,
             precision: str = "f32") -> np.ndarray:
    """The eat rule on one fish's weight, given its deltas and the school's
    per-step maxima; returns the weight after each step."""
    real = np.float32 if precision == "f32" else np.float64
    delta = np.ascontiguousarray(delta, dtype=real)
    M = np.ascontiguousarray(max_abs_delta, dtype=np.float64)
    assert delta.shape == M.shape
    out = np.zeros(delta.size, real)
    c = cfg.c()
    getattr(lib(), "fsbo_eat_fish_" + precision)(
        ctypes.byref(c), w, delta.size, _ptr(delta), _ptr(M), _ptr(out))
    return out
