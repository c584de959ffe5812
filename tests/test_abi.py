"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
entry point include/lob.h declares.  No call here touches the device."""
import ctypes
import os
import re

from paper_2511_02136_gb300 import lob

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(lob_[a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_header_declares_the_binding_surface():
    assert sorted(lob.EXPORTS) == _declared("lob.h")


def test_library_exports_every_declared_symbol():
    path = lob.build()
    so = ctypes.CDLL(path)
    for name in _declared("lob.h"):
        assert hasattr(so, name), name


def test_host_only_entry_points():
    lob.build()
    cfg = lob.lob_config(8, 2, 100, 10, 1000, 1, 500, -1, 1, 0, 10000, 0)
    assert lob.lob_obs_dim(cfg) == 45
    cfg.top_levels = 20
    assert lob.lob_obs_dim(cfg) == 85
    cfg.n_agents = 0
    assert lob.lob_obs_dim(cfg) == 0
    assert lob.lob_strerror(lob.LOB_EBADMSG).startswith("malformed")
    assert lob.lob_strerror(0) == "ok"


def test_built_for_sm103a_only():
    for cmd in [lob.nvcc_cmd("x.so")] + [lob.nvcc_cmd("x.o", src=s) for s in lob._SOURCES]:
        assert "arch=compute_103a,code=sm_103a" in cmd
        assert sum(1 for c in cmd if c == "-gencode") == 1


def test_one_library_per_process():
    """Pointing the binding at another library after the first load raises
    instead of silently calling the library already loaded."""
    lob.build()
    lob._load()
    old = lob.LIB_PATH
    try:
        lob.LIB_PATH = old + ".other.so"
        try:
            lob._load()
        except RuntimeError as e:
            assert "one process per library" in str(e)
        else:
            raise AssertionError("a second library path was accepted")
    finally:
        lob.LIB_PATH = old
    assert lob._load() is not None
