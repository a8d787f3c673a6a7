"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function that include/spr.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "spr.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(spr_[a-z0-9_]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def lib():
    from paper_2309_10212_gb300 import build
    build.build()
    return ctypes.CDLL(build.SO)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["spr_create_volume", "spr_set_camera", "spr_set_isovalue",
                 "spr_set_cache_budget", "spr_set_speculation", "spr_render_pass",
                 "spr_render_to_convergence", "spr_get_framebuffer"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2309_10212_gb300 import _lib
    assert set(declared_functions()) == set(_lib.PROTOTYPES)


def test_host_only_calls(lib):
    from paper_2309_10212_gb300 import _lib
    L = _lib.load()
    assert L.spr_version() == 10000
    assert L.spr_status_string(_lib.SPR_ERR_DEVICE_TIMEOUT) == b"bounded device wait timed out"
    # a mismatched allocator pair is rejected before any device call
    assert L.spr_set_allocator(_lib.ALLOC_FN(lambda n, s, c: None), _lib.FREE_FN(), None) \
        == _lib.SPR_ERR_INVALID_ARG
    assert b"both" in L.spr_last_error()


def test_sources_target_sm103a_only():
    from paper_2309_10212_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
