"""Shared helpers of the GPU parity tests (marshalling and comparisons)."""
import numpy as np

import oracle
import paper_2507_20173_gb300 as fsb

FIELDS = (("x", "x"), ("y", "y"), ("w", "weight"), ("prev", "prevObjective"),
          ("cur", "currentObjective"))

# Barycentre tolerance per arithmetic mode: error against the oracle's exact
# sums, normalised by sum |w x| (sum w for S_w).  Plain binary32 sums are the
# precision baseline and only get a loose bound.
BARY_TOL = {fsb.FSB_FP32: 1e-3, fsb.FSB_FP32_KAHAN: 1e-5, fsb.FSB_FP64_ACC: 1e-12,
            fsb.FSB_FP64_STATE: 1e-12}


def oracle_config(cfg) -> oracle.Config:
    return oracle.Config(n_fish=cfg.n_fish, seed=cfg.seed, school_id=cfg.school_id,
                         init_weight_mode=cfg.init_weight_mode, pond_half=cfg.pond_half,
                         step=cfg.step, w0=cfg.w0, w_min=cfg.w_min, w_max=cfg.w_max,
                         swim_mode=cfg.swim_mode, feed_mode=cfg.feed_mode,
                         collective_mode=cfg.collective_mode, step_vol=cfg.step_vol)


def oracle_precision(cfg) -> str:
    return "f64" if cfg.precision == fsb.FSB_FP64_STATE else "f32"


def assert_state_equal(got: dict, ref: np.ndarray, where: str = "") -> None:
    for a, b in FIELDS:
        g, r = got[a], ref[b]
        if not np.array_equal(g, r):
            bad = np.nonzero(g != r)[0]
            i = int(bad[0])
            raise AssertionError("%s field %s differs at %d fish (first %d: gpu %r oracle %r)"
                                 % (where, a, bad.size, i, g[i], r[i]))


def bary_errors(stats: np.ndarray, ref: np.ndarray) -> dict:
    return {
        "sum_w": np.abs(stats["sum_w"] - ref["sum_w"]) / np.maximum(np.abs(ref["sum_w"]), 1e-300),
        "sum_wx": np.abs(stats["sum_wx"] - ref["sum_wx"]) / np.maximum(ref["sum_abs_wx"], 1e-300),
        "sum_wy": np.abs(stats["sum_wy"] - ref["sum_wy"]) / np.maximum(ref["sum_abs_wy"], 1e-300),
    }


def assert_stats_match(stats: np.ndarray, ref: np.ndarray, precision: int, where: str = ""):
    assert np.array_equal(stats["max_abs_delta"], ref["max_abs_delta"]), where + " max|delta|"
    assert np.array_equal(stats["eat_max_diff"], ref["eat_max_diff"]), where + " eat_max_diff"
    tol = BARY_TOL[precision]
    for k, e in bary_errors(stats, ref).items():
        assert e.max() <= tol, "%s %s error %.3e > %.1e" % (where, k, e.max(), tol)
