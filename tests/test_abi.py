"""The C ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1911_09135_gb300 import _build, alb

HEADER = os.path.join(_build.INCLUDE_DIR, "alb.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(alb_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    _build.build_alb()
    return alb.load()


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 19
    out = subprocess.run(["nm", "-D", "--defined-only", alb.lib_path()], stdout=subprocess.PIPE,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (alb_\w+)", out))
    missing = [s for s in syms if s not in exported]
    assert not missing, missing
    for s in syms:
        assert hasattr(lib, s)
    assert sorted(alb.EXPORTS) == syms


def test_build_targets_sm103a_only():
    assert _build.GENCODE == "-gencode=arch=compute_103a,code=sm_103a"


def test_host_only_entry_points(lib):
    # The paper's default threshold rule: number of threads launched (Sec. 4.1, Sec. 5):
    assert alb.alb_threshold_rule(80, 2048) == 163840   # V100, as printed in Sec. 5
    assert alb.alb_threshold_rule(56, 2048) == 114688   # P100, as printed in Sec. 5
    assert alb.alb_version() == 10000
    assert alb.alb_status_str(0) == "ALB_OK"
    assert alb.alb_status_str(6) == "ALB_ERR_NOT_SYMMETRIC"
    p = alb.alb_default_params()
    assert p.hub_threshold == -1 and p.twc_warp_min == 32 and p.twc_cta_min == 256
    assert p.distribution == 0 and p.exec_mode == 0


def test_argument_errors_need_no_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.alb_graph_create(0, 0, None, None, None, 0, None, ctypes.byref(h)) == 1
    assert lib.alb_graph_create(4, 1 << 32, None, None, None, 0, None, ctypes.byref(h)) == 1
    assert lib.alb_bfs(None, 0, None, None) == 1
    assert lib.alb_default_params(None) == 1
