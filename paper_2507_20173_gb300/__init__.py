"""Python binding of libfsb.so, the GB300 Fish School Behaviour library.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The functions keep the C names of include/fsb.h
(``fsb_create``, ``fsb_step``, ``fsb_run_batch``, ``fsb_read_state``,
``fsb_destroy``, ``fsb_strerror`` ...) and raise :class:`FsbError` on a
non-zero status.  PyTorch is used only for device memory and streams.

There is no CPU fallback: if ``libfsb.so`` has not been built, or no CUDA
device is present, the calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfsb.so")

FSB_OK = 0
FSB_ERR_INVALID_ARG = -1
FSB_ERR_CUDA = -2
FSB_ERR_OOM = -3
FSB_ERR_UNSUPPORTED = -4
FSB_ERR_TIMEOUT = -5
FSB_ERR_STATE = -6

FSB_FP32 = 0
FSB_FP32_KAHAN = 1
FSB_FP64_ACC = 2
FSB_FP64_STATE = 3

FSB_EAT_REDUCTION = 0
FSB_EAT_PER_WARP = 1
FSB_EAT_CRITICAL = 2

FSB_PATH_AUTO = 0
FSB_PATH_STREAM = 1
FSB_PATH_RESIDENT = 2

EXPORTED = ("fsb_config_init", "fsb_create", "fsb_step", "fsb_read_state",
            "fsb_last_stats", "fsb_destroy", "fsb_run_batch",
            "fsb_set_kernel_timing", "fsb_kernel_time", "fsb_handle_path",
            "fsb_strerror", "fsb_last_error", "fsb_step_static", "fsb_set_fault_injection",
            "fsb_set_tuning", "fsb_get_tuning", "fsb_batch_create", "fsb_batch_step",
            "fsb_batch_set_cluster", "fsb_batch_info", "fsb_batch_set_timing",
            "fsb_batch_kernel_time", "fsb_batch_destroy", "fsb_autotune",
            "fsb_autotune_batch", "fsb_eat_max", "fsb_batch_plan", "fsb_batch_set_plan",
            "fsb_batch_limits")


class FsbError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__("%s: %s (%s)" % (where, _name(status), detail))
        self.status = status


class FsbConfig(ctypes.Structure):
    _fields_ = [("n_fish", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("school_id", ctypes.c_uint32), ("init_weight_mode", ctypes.c_int32),
                ("pond_half", ctypes.c_double), ("step", ctypes.c_double),
                ("w0", ctypes.c_double), ("w_min", ctypes.c_double),
                ("w_max", ctypes.c_double), ("precision", ctypes.c_int32),
                ("path", ctypes.c_int32), ("swim_mode", ctypes.c_int32),
                ("feed_mode", ctypes.c_int32), ("collective_mode", ctypes.c_int32),
                ("step_vol", ctypes.c_double)]


class FsbStateDev(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("prev_objective", ctypes.c_void_p)]


class FsbStateHost(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("prev_objective", ctypes.c_void_p)]


class FsbStepStats(ctypes.Structure):
    _fields_ = [("max_abs_delta", ctypes.c_double), ("eat_max_diff", ctypes.c_double),
                ("sum_w", ctypes.c_double), ("sum_wx", ctypes.c_double),
                ("sum_wy", ctypes.c_double)]


class FsbTuning(ctypes.Structure):
    _fields_ = [("stream_kernel", ctypes.c_int32), ("stream_block", ctypes.c_int32),
                ("stream_blocks_per_sm", ctypes.c_int32), ("resident_fpt", ctypes.c_int32),
                ("resident_block", ctypes.c_int32), ("stream_stages", ctypes.c_int32),
                ("stream_block_steps", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


STATS_DTYPE = np.dtype([("max_abs_delta", "<f8"), ("eat_max_diff", "<f8"),
                        ("sum_w", "<f8"), ("sum_wx", "<f8"), ("sum_wy", "<f8")])

_lib = None


def lib() -> ctypes.CDLL:
    """Load libfsb.so (built in-tree by ``paper_2507_20173_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libfsb.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    cfgp = ctypes.POINTER(FsbConfig)
    sigs = {
        "fsb_config_init": [cfgp, u64, u64],
        "fsb_create": [cfgp, ctypes.POINTER(FsbStateDev), ctypes.POINTER(FsbStateHost),
                       u64, P, ctypes.POINTER(P)],
        "fsb_step": [P, u32, P],
        "fsb_read_state": [P, P, P, P, P, P, ctypes.POINTER(u64)],
        "fsb_last_stats": [P, P, u32],
        "fsb_destroy": [P],
        "fsb_run_batch": [cfgp, u32, P, P, ctypes.POINTER(FsbStateDev), i32, u64, u32, P, P],
        "fsb_set_kernel_timing": [P, i32],
        "fsb_kernel_time": [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u64)],
        "fsb_handle_path": [P, ctypes.POINTER(i32)],
        "fsb_set_fault_injection": [P, i32, u32, u64],
        "fsb_set_tuning": [P, ctypes.POINTER(FsbTuning)],
        "fsb_batch_create": [cfgp, u32, P, P, ctypes.POINTER(FsbStateDev), i32, u64, P,
                             ctypes.POINTER(P)],
        "fsb_batch_step": [P, u32, P],
        "fsb_batch_set_cluster": [P, i32],
        "fsb_batch_info": [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                           ctypes.POINTER(u32), ctypes.POINTER(u64)],
        "fsb_batch_plan": [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                           ctypes.POINTER(u32)],
        "fsb_batch_set_plan": [P, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "fsb_batch_limits": [ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(i32)],
        "fsb_batch_set_timing": [P, i32],
        "fsb_batch_kernel_time": [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u64)],
        "fsb_batch_destroy": [P],
        "fsb_eat_max": [P, P, u64, i32, ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_float), P],
        "fsb_autotune": [cfgp, u32, ctypes.POINTER(i32), ctypes.POINTER(FsbTuning),
                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u32)],
        "fsb_autotune_batch": [cfgp, u32, P, P, ctypes.POINTER(FsbStateDev), u32,
                               ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)],
        "fsb_get_tuning": [P, ctypes.POINTER(FsbTuning)],
        "fsb_strerror": [i32],
        "fsb_step_static": [cfgp, ctypes.POINTER(FsbStateDev), u64, u32, P, P],
        "fsb_last_error": [],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.fsb_strerror.restype = ctypes.c_char_p
    L.fsb_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _name(status: int) -> str:
    try:
        return lib().fsb_strerror(status).decode()
    except ImportError:
        return str(status)


def _check(status: int, where: str) -> None:
    if status != FSB_OK:
        raise FsbError(status, where, lib().fsb_last_error().decode())


# ------------------------------------------------- C-named entry points --

def fsb_config_init(n_fish: int, seed: int = 0, **fields) -> FsbConfig:
    cfg = FsbConfig()
    _check(lib().fsb_config_init(ctypes.byref(cfg), n_fish, seed), "fsb_config_init")
    for k, v in fields.items():
        setattr(cfg, k, v)
    return cfg


def fsb_create(cfg: FsbConfig, buffers: FsbStateDev | None = None,
               init: FsbStateHost | None = None, start_step: int = 0,
               stream: int | None = None) -> int:
    h = ctypes.c_void_p()
    _check(lib().fsb_create(ctypes.byref(cfg), ctypes.byref(buffers) if buffers else None,
                            ctypes.byref(init) if init else None, start_step,
                            ctypes.c_void_p(stream or 0), ctypes.byref(h)), "fsb_create")
    return h.value


def fsb_step(handle: int, n_steps: int, host_stats: np.ndarray | None = None) -> None:
    ptr = None
    if host_stats is not None:
        assert host_stats.dtype == STATS_DTYPE and host_stats.size >= n_steps
        assert host_stats.flags["C_CONTIGUOUS"]
        ptr = host_stats.ctypes.data_as(ctypes.c_void_p)
    _check(lib().fsb_step(ctypes.c_void_p(handle), n_steps, ptr), "fsb_step")


def fsb_last_stats(handle: int, host_stats: np.ndarray, n_steps: int) -> None:
    assert host_stats.dtype == STATS_DTYPE and host_stats.size >= n_steps
    _check(lib().fsb_last_stats(ctypes.c_void_p(handle),
                                host_stats.ctypes.data_as(ctypes.c_void_p), n_steps),
           "fsb_last_stats")


def fsb_read_state(handle: int, x=None, y=None, w=None, prev_objective=None,
                   current_objective=None) -> int:
    """Copy the state into the given host numpy arrays; returns step t."""
    def p(a):
        if a is None:
            return None
        assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]
        return a.ctypes.data_as(ctypes.c_void_p)
    step = ctypes.c_uint64()
    _check(lib().fsb_read_state(ctypes.c_void_p(handle), p(x), p(y), p(w), p(prev_objective),
                                p(current_objective), ctypes.byref(step)), "fsb_read_state")
    return step.value


def fsb_destroy(handle: int) -> None:
    _check(lib().fsb_destroy(ctypes.c_void_p(handle)), "fsb_destroy")


def fsb_run_batch(tmpl: FsbConfig, offsets: np.ndarray, seeds: np.ndarray,
                  state: FsbStateDev, n_steps: int, init: bool = False,
                  start_step: int = 0, stats: np.ndarray | None = None,
                  stream: int | None = None) -> None:
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    n = seeds.size
    assert offsets.size == n + 1
    sptr = None
    if stats is not None:
        assert stats.dtype == STATS_DTYPE and stats.size >= n * n_steps
        sptr = stats.ctypes.data_as(ctypes.c_void_p)
    _check(lib().fsb_run_batch(ctypes.byref(tmpl), n, offsets.ctypes.data_as(ctypes.c_void_p),
                               seeds.ctypes.data_as(ctypes.c_void_p), ctypes.byref(state),
                               1 if init else 0, start_step, n_steps, sptr,
                               ctypes.c_void_p(stream or 0)), "fsb_run_batch")


def fsb_step_static(cfg: FsbConfig, state: FsbStateDev, start_step: int, n_steps: int,
                    stats_out=None, stream: int | None = None) -> None:
    """Allocation-free step of caller-owned device arrays (see include/fsb.h).
    `stats_out`: None, a host numpy array of STATS_DTYPE, or a device address
    (int) of n_steps records."""
    ptr = None
    if isinstance(stats_out, np.ndarray):
        assert stats_out.dtype == STATS_DTYPE and stats_out.size >= n_steps
        ptr = stats_out.ctypes.data_as(ctypes.c_void_p)
    elif stats_out is not None:
        ptr = ctypes.c_void_p(int(stats_out))
    _check(lib().fsb_step_static(ctypes.byref(cfg), ctypes.byref(state), start_step, n_steps,
                                 ptr, ctypes.c_void_p(stream or 0)), "fsb_step_static")


def fsb_batch_create(tmpl: FsbConfig, offsets: np.ndarray, seeds: np.ndarray,
                     state: FsbStateDev, init: bool = False, start_step: int = 0,
                     stream: int | None = None) -> int:
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    assert offsets.size == seeds.size + 1
    h = ctypes.c_void_p()
    _check(lib().fsb_batch_create(ctypes.byref(tmpl), seeds.size,
                                  offsets.ctypes.data_as(ctypes.c_void_p),
                                  seeds.ctypes.data_as(ctypes.c_void_p), ctypes.byref(state),
                                  1 if init else 0, start_step, ctypes.c_void_p(stream or 0),
                                  ctypes.byref(h)), "fsb_batch_create")
    return h.value


def fsb_batch_step(handle: int, n_steps: int, stats: np.ndarray | None = None) -> None:
    ptr = None
    if stats is not None:
        assert stats.dtype == STATS_DTYPE and stats.flags["C_CONTIGUOUS"]
        ptr = stats.ctypes.data_as(ctypes.c_void_p)
    _check(lib().fsb_batch_step(ctypes.c_void_p(handle), n_steps, ptr), "fsb_batch_step")


def fsb_batch_set_cluster(handle: int, cluster: int) -> None:
    _check(lib().fsb_batch_set_cluster(ctypes.c_void_p(handle), cluster), "fsb_batch_set_cluster")


def fsb_batch_info(handle: int) -> dict:
    c, nc, fb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nb, st = ctypes.c_uint32(), ctypes.c_uint64()
    _check(lib().fsb_batch_info(ctypes.c_void_p(handle), ctypes.byref(c), ctypes.byref(nc),
                                ctypes.byref(fb), ctypes.byref(nb), ctypes.byref(st)),
           "fsb_batch_info")
    return {"cluster": c.value, "n_clusters": nc.value, "filler_blocks": fb.value,
            "n_big": nb.value, "step": st.value}


def fsb_batch_limits() -> dict:
    """Fish one block of the batched kernel holds, fish one warp of a packed
    team holds (0: no packing), and the widest cluster."""
    bf, tf, mc = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int()
    _check(lib().fsb_batch_limits(ctypes.byref(bf), ctypes.byref(tf), ctypes.byref(mc)),
           "fsb_batch_limits")
    return {"block_fish": bf.value, "team_fish": tf.value, "max_cluster": mc.value}


def fsb_batch_plan(handle: int) -> dict:
    """The batch's concurrent launches (cluster size, grid), the schools in
    each work queue keyed by the queue's cluster size (8 down to 1), and the
    schools packed several to a block, keyed by the team's warps (8 down to
    1)."""
    n = ctypes.c_int()
    c, b = (ctypes.c_int * 8)(), (ctypes.c_int * 8)()
    q = (ctypes.c_uint32 * 12)()
    _check(lib().fsb_batch_plan(ctypes.c_void_p(handle), ctypes.byref(n), c, b, q),
           "fsb_batch_plan")
    return {"launches": [{"cluster": c[i], "blocks": b[i]} for i in range(n.value)],
            "queue_schools": {8 - t: q[t] for t in range(7)} | {1: q[7]},
            "packed_schools": {8 >> t: q[8 + t] for t in range(4)}}


def fsb_batch_set_plan(handle: int, launches) -> None:
    """Replace the batch's launches: a sequence of (cluster, blocks)."""
    n = len(launches)
    c = (ctypes.c_int * max(n, 1))(*[int(l[0]) for l in launches])
    b = (ctypes.c_int * max(n, 1))(*[int(l[1]) for l in launches])
    _check(lib().fsb_batch_set_plan(ctypes.c_void_p(handle), n, c, b), "fsb_batch_set_plan")


def fsb_batch_set_timing(handle: int, enable: bool) -> None:
    _check(lib().fsb_batch_set_timing(ctypes.c_void_p(handle), 1 if enable else 0),
           "fsb_batch_set_timing")


def fsb_batch_kernel_time(handle: int) -> tuple[float, int]:
    ms, n = ctypes.c_double(), ctypes.c_uint64()
    _check(lib().fsb_batch_kernel_time(ctypes.c_void_p(handle), ctypes.byref(ms),
                                       ctypes.byref(n)), "fsb_batch_kernel_time")
    return ms.value, n.value


def fsb_batch_destroy(handle: int) -> None:
    _check(lib().fsb_batch_destroy(ctypes.c_void_p(handle)), "fsb_batch_destroy")


def fsb_eat_max(prev_ptr: int, cur_ptr: int, n: int, construct: int = FSB_EAT_REDUCTION,
                stream: int | None = None) -> tuple[float, float]:
    """max(prev - cur) over device arrays; returns (value, device ms)."""
    out, ms = ctypes.c_double(), ctypes.c_float()
    _check(lib().fsb_eat_max(ctypes.c_void_p(prev_ptr), ctypes.c_void_p(cur_ptr), n, construct,
                             ctypes.byref(out), ctypes.byref(ms), ctypes.c_void_p(stream or 0)),
           "fsb_eat_max")
    return out.value, ms.value


def fsb_autotune(cfg: FsbConfig, n_steps: int) -> dict:
    path, t = ctypes.c_int(), FsbTuning()
    rate, tried = ctypes.c_double(), ctypes.c_uint32()
    _check(lib().fsb_autotune(ctypes.byref(cfg), n_steps, ctypes.byref(path), ctypes.byref(t),
                              ctypes.byref(rate), ctypes.byref(tried)), "fsb_autotune")
    return {"path": path.value, "tuning": t.as_dict(), "fish_steps_per_s": rate.value,
            "candidates": tried.value}


def fsb_autotune_batch(tmpl: FsbConfig, offsets: np.ndarray, seeds: np.ndarray,
                       state: FsbStateDev, n_steps: int) -> dict:
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    c, rate = ctypes.c_int(), ctypes.c_double()
    _check(lib().fsb_autotune_batch(ctypes.byref(tmpl), seeds.size,
                                    offsets.ctypes.data_as(ctypes.c_void_p),
                                    seeds.ctypes.data_as(ctypes.c_void_p), ctypes.byref(state),
                                    n_steps, ctypes.byref(c), ctypes.byref(rate)),
           "fsb_autotune_batch")
    return {"cluster": c.value, "fish_steps_per_s": rate.value}


def fsb_set_kernel_timing(handle: int, enable: bool) -> None:
    _check(lib().fsb_set_kernel_timing(ctypes.c_void_p(handle), 1 if enable else 0),
           "fsb_set_kernel_timing")


def fsb_kernel_time(handle: int) -> tuple[float, int]:
    ms = ctypes.c_double()
    n = ctypes.c_uint64()
    _check(lib().fsb_kernel_time(ctypes.c_void_p(handle), ctypes.byref(ms), ctypes.byref(n)),
           "fsb_kernel_time")
    return ms.value, n.value


def fsb_set_fault_injection(handle: int, block: int, step: int, timeout_ns: int = 0) -> None:
    _check(lib().fsb_set_fault_injection(ctypes.c_void_p(handle), block, step, timeout_ns),
           "fsb_set_fault_injection")


def fsb_set_tuning(handle: int, **fields) -> None:
    t = FsbTuning(**fields)
    _check(lib().fsb_set_tuning(ctypes.c_void_p(handle), ctypes.byref(t)), "fsb_set_tuning")


def fsb_get_tuning(handle: int) -> dict:
    t = FsbTuning()
    _check(lib().fsb_get_tuning(ctypes.c_void_p(handle), ctypes.byref(t)), "fsb_get_tuning")
    return t.as_dict()


def fsb_handle_path(handle: int) -> int:
    p = ctypes.c_int()
    _check(lib().fsb_handle_path(ctypes.c_void_p(handle), ctypes.byref(p)), "fsb_handle_path")
    return p.value


def fsb_strerror(status: int) -> str:
    return lib().fsb_strerror(status).decode()


def fsb_last_error() -> str:
    return lib().fsb_last_error().decode()


# ------------------------------------------------ torch-buffer helper --

@dataclass
class School:
    """A school whose four state arrays are torch CUDA tensors (marshalling
    helper around fsb_create / fsb_step / fsb_read_state)."""
    cfg: FsbConfig
    handle: int
    tensors: tuple

    @staticmethod
    def create(cfg: FsbConfig, init: dict | None = None, start_step: int = 0,
               stream=None, device: str = "cuda") -> "School":
        import torch
        dtype = torch.float64 if cfg.precision == FSB_FP64_STATE else torch.float32
        ts = tuple(torch.empty(cfg.n_fish, dtype=dtype, device=device) for _ in range(4))
        bufs = FsbStateDev(*(t.data_ptr() for t in ts))
        host = None
        keep = None
        if init is not None:
            npdt = np.float64 if dtype == torch.float64 else np.float32
            keep = [np.ascontiguousarray(init[k], dtype=npdt)
                    for k in ("x", "y", "w", "prev_objective")]
            host = FsbStateHost(*(a.ctypes.data for a in keep))
        s = stream if stream is not None else torch.cuda.current_stream()
        h = fsb_create(cfg, bufs, host, start_step, s.cuda_stream)
        del keep
        return School(cfg, h, ts)

    def step(self, n_steps: int, stats: bool = False):
        out = np.zeros(n_steps, STATS_DTYPE) if stats else None
        fsb_step(self.handle, n_steps, out)
        return out

    def read(self) -> dict:
        npdt = np.float64 if self.cfg.precision == FSB_FP64_STATE else np.float32
        n = self.cfg.n_fish
        st = {k: np.empty(n, npdt) for k in ("x", "y", "w", "prev", "cur")}
        st["step"] = fsb_read_state(self.handle, st["x"], st["y"], st["w"], st["prev"], st["cur"])
        return st

    def destroy(self) -> None:
        if self.handle:
            fsb_destroy(self.handle)
            self.handle = 0
