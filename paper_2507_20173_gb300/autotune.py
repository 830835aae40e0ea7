"""Tuning table of the library's launch shapes.

The measuring is native (``fsb_autotune`` / ``fsb_autotune_batch`` in
libfsb.so).  This module only runs it over a range of school sizes, keeps the
winners in a JSON table keyed by GPU name and arithmetic mode, and applies
an entry when a school is created.  The winner's path at each size gives the
cutoff between the resident (on-chip) and the streaming kernels.

    python -m paper_2507_20173_gb300.autotune            # tune, print, save
"""
from __future__ import annotations

import json
import os
import sys

import paper_2507_20173_gb300 as fsb

TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_table.json")
DEFAULT_SIZES = sorted(set([1 << k for k in range(10, 29, 2)] + [10_000, 1 << 21, 1 << 23]))
PRECISIONS = {"FP32": fsb.FSB_FP32, "FP32_KAHAN": fsb.FSB_FP32_KAHAN,
              "FP64_ACC": fsb.FSB_FP64_ACC, "FP64_STATE": fsb.FSB_FP64_STATE}


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(0)


def tune(sizes=None, precision: str = "FP32_KAHAN", steps: int = 20) -> list[dict]:
    """Run the native autotuner for each school size."""
    out = []
    for n in sorted(sizes or DEFAULT_SIZES):
        cfg = fsb.fsb_config_init(int(n), 12345, precision=PRECISIONS[precision])
        r = fsb.fsb_autotune(cfg, steps)
        r["n_fish"] = int(n)
        out.append(r)
    return out


def load(path: str = TABLE_PATH) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def save(table: dict, path: str = TABLE_PATH) -> None:
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def entry_for(table: dict, n_fish: int, precision: str, gpu: str | None = None) -> dict | None:
    """The tuned entry for the largest tuned size not above n_fish (or the
    smallest tuned size), for this GPU and mode; None if nothing is tuned."""
    rows = table.get(gpu or gpu_name(), {}).get(precision, [])
    if not rows:
        return None
    rows = sorted(rows, key=lambda r: r["n_fish"])
    best = rows[0]
    for r in rows:
        if r["n_fish"] <= n_fish:
            best = r
    return best


def create_tuned(cfg: fsb.FsbConfig, table: dict | None = None, **kw) -> fsb.School:
    """fsb.School.create with the path and launch shape the table holds for
    this size (the library's defaults if the table has no entry)."""
    name = {v: k for k, v in PRECISIONS.items()}[cfg.precision]
    e = entry_for(table if table is not None else load(), cfg.n_fish, name)
    if e is not None and cfg.path == fsb.FSB_PATH_AUTO:
        cfg.path = e["path"]
    try:
        school = fsb.School.create(cfg, **kw)
    except fsb.FsbError:
        if e is None:
            raise
        cfg.path = fsb.FSB_PATH_AUTO
        school = fsb.School.create(cfg, **kw)
        return school
    if e is not None:
        try:
            fsb.fsb_set_tuning(school.handle, **e["tuning"])
        except fsb.FsbError:
            pass  # shape not valid for this exact size: keep the defaults
    return school


def main(argv=None) -> int:
    argv = argv if argv is not None else sys.argv[1:]
    precision = argv[0] if argv else "FP32_KAHAN"
    fsb.lib()
    rows = tune(precision=precision)
    table = load()
    table.setdefault(gpu_name(), {})[precision] = rows
    save(table)
    for r in rows:
        print("N=%-10d path=%s rate=%.3e %s" % (r["n_fish"], {1: "stream", 2: "resident"}[r["path"]],
                                              r["fish_steps_per_s"], r["tuning"]))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
