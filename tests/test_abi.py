"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/lbehd.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(lbehd_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2608_12868_b300 import build
    build.build()
    from paper_2608_12868_b300 import lbehd
    return lbehd.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert "lbehd_init" in names and "lbehd_step" in names and "lbehd_observe" in names
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2608_12868_b300",
                                                                     "liblbehd.so")],
                         capture_output=True, text=True, check=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n


def test_binding_layout_matches_library(lib):
    from paper_2608_12868_b300 import lbehd
    assert lib.lbehd_abi_version() == 4
    assert lib.lbehd_config_size() == ctypes.sizeof(lbehd.Config)
    assert set(lbehd.EXPORTS) <= set(_declared())


def test_library_is_built_for_sm_103a(lib):
    from paper_2608_12868_b300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_init_rejects_bad_configs_before_touching_the_gpu(lib):
    from paper_2608_12868_b300 import lbehd
    c = lbehd.Config()
    h = ctypes.c_void_p()
    c.dim = 4
    assert lib.lbehd_init(ctypes.byref(c), ctypes.byref(h)) == -1
    assert b"dim" in lib.lbehd_last_error(None)
    c.dim, c.nx, c.ny, c.nz = 3, 15, 8, 8
    assert lib.lbehd_init(ctypes.byref(c), ctypes.byref(h)) == -1
    assert b"even" in lib.lbehd_last_error(None)


def test_batch_init_rejects_bad_arguments_before_touching_the_gpu(lib):
    from paper_2608_12868_b300 import lbehd
    cfgs = (lbehd.Config * 2)()
    cfgs[0].dim, cfgs[1].dim = 3, 2
    b = ctypes.c_void_p()
    assert lib.lbehd_batch_init(cfgs, 0, ctypes.byref(b)) == -1
    assert lib.lbehd_batch_init(cfgs, 2, ctypes.byref(b)) == -1
    assert b"share dim" in lib.lbehd_last_error(None)
    assert lib.lbehd_batch_size(None) == 0
    assert lib.lbehd_batch_instance(None, 0) is None


def test_entry_points_reject_a_null_handle_without_a_gpu(lib):
    """Every handle-taking call returns LBEHD_ERR_INVALID_ARG for a null handle and leaves a
    message, before any CUDA call (so this runs without a device)."""
    from paper_2608_12868_b300 import lbehd
    P = ctypes.c_void_p
    v = ctypes.c_longlong()
    obs = lbehd.Obs()
    calls = {
        "lbehd_step": lambda: lib.lbehd_step(None, 1),
        "lbehd_observe": lambda: lib.lbehd_observe(None, ctypes.byref(obs)),
        "lbehd_set_option": lambda: lib.lbehd_set_option(None, 1, 0),
        "lbehd_get_option": lambda: lib.lbehd_get_option(None, 1, ctypes.byref(v)),
        "lbehd_save_state": lambda: lib.lbehd_save_state(None, P(16)),
        "lbehd_load_state": lambda: lib.lbehd_load_state(None, P(16)),
    }
    for name, call in calls.items():
        assert call() == -1, name
        assert lib.lbehd_last_error(None), name
    assert lib.lbehd_state_bytes(None) == 0
