"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (CPU only: no compute calls)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

import paper_2507_20173_gb300 as fsb
from paper_2507_20173_gb300 import build as fsb_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*"
                             r"(fsb_[A-Za-z0-9_]+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return fsb_build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fsb_create", "fsb_step", "fsb_run_batch", "fsb_read_state",
                     "fsb_destroy", "fsb_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_names_statuses(libpath):
    L = fsb.lib()
    for n in declared_functions():
        assert hasattr(L, n)
    assert fsb.fsb_strerror(fsb.FSB_ERR_TIMEOUT) == "FSB_ERR_TIMEOUT"
    assert fsb.fsb_strerror(0) == "FSB_OK"


def test_batch_limits_need_no_gpu(libpath):
    # 11 pairs per fish thread of a 512-thread block; 16 warps share a block
    assert fsb.fsb_batch_limits() == {"block_fish": 11264, "team_fish": 704, "max_cluster": 8}


def test_config_defaults_and_host_validation(libpath):
    cfg = fsb.fsb_config_init(10, 3)
    assert (cfg.pond_half, cfg.step, cfg.w0, cfg.w_min, cfg.w_max) == (100.0, 0.1, 1.0, 0.0, 2.0)
    assert cfg.precision == fsb.FSB_FP32_KAHAN and cfg.path == fsb.FSB_PATH_AUTO
    # validation happens before any CUDA call, so it runs without a GPU
    bad = fsb.fsb_config_init(0, 3)
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_create(bad)
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    bad = fsb.fsb_config_init(10, 3, w_min=3.0)
    with pytest.raises(fsb.FsbError) as e:
        fsb.fsb_create(bad)
    assert e.value.status == fsb.FSB_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert L_create_null_out(libpath) == fsb.FSB_ERR_INVALID_ARG
    del h


def L_create_null_out(libpath):
    L = fsb.lib()
    cfg = fsb.fsb_config_init(10, 3)
    return L.fsb_create(ctypes.byref(cfg), None, None, 0, None, None)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(fsb, "_lib", None)
    monkeypatch.setattr(fsb, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        fsb.lib()


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes structures of the binding have the size and field offsets
    of the C structures in include/fsb.h (a small C program prints them)."""
    structs = {"fsb_config": fsb.FsbConfig, "fsb_state_dev": fsb.FsbStateDev,
               "fsb_state_host": fsb.FsbStateHost, "fsb_step_stats": fsb.FsbStepStats,
               "fsb_tuning": fsb.FsbTuning}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "fsb.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));'
                         % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True,
                               check=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
