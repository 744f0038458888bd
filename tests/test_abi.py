"""The C-ABI library loads on a machine without a GPU and exports every entry point that
include/qis.h declares; without a device, the first call fails loudly (no CPU fallback)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2010_00180_gb300 import build, qis

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return qis.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "qis.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qis_[a-z_]+)\s*\(", text)))


def test_header_matches_binding():
    assert header_functions() == sorted(qis.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", qis.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (qis_\w+)", out))
    for name in header_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_config_struct_layout(lib):
    assert C.sizeof(qis.Config) == 48
    assert qis.Config.seed.offset == 32
    assert qis.Config.flips.offset == 40


def test_create_rejects_bad_config(lib):
    cfg = qis.Config(0, 4, 1, 16, 1, 0, 0, 0)            # K = 0
    h = C.c_void_p()
    assert lib.qis_create(C.byref(cfg), C.byref(h)) == -1
    assert b"K" in lib.qis_last_error(None)
    cfg = qis.Config(8, 4, 7, 16, 1, 0, 0, 0)            # unknown precision
    assert lib.qis_create(C.byref(cfg), C.byref(h)) == -1
    cfg = qis.Config(8, 4, 1, 16, 1, 0, 0, 0, 3)         # unknown flip set
    assert lib.qis_create(C.byref(cfg), C.byref(h)) == -1
    assert b"flip" in lib.qis_last_error(None)


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="a GPU is present")
def test_no_gpu_fails_loudly(lib):
    with pytest.raises(qis.QISError) as e:
        qis.Context(K=8, R=4, precision="split_bf16", max_n=16)
    assert e.value.name == "CUDA"
