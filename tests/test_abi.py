"""The C ABI library: it builds for sm_103a, loads, exports every symbol that
include/rp.h declares, and refuses to compute without a GPU (no CPU
fallback).  CPU only: no compute call runs here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_16302_gb300 import build, rp
    build.build()
    return rp.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "rp.h")).read()
    return sorted(set(re.findall(r"^(?:rp_status|void|const char \*)\s*(rp_\w+)\(", src, re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("rp_scene_create", "rp_edit", "rp_render_residual", "rp_render_primal",
                 "rp_dump_samples", "rp_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2406_16302_gb300 import rp
    syms = declared_symbols()
    assert sorted(rp.EXPORTS) == syms
    for name in syms:
        assert hasattr(lib, name), name


def test_no_cpu_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2406_16302_gb300 import rp, scenes
    scene, _ = scenes.cfg1_box_sphere(width=8, height=8)
    with pytest.raises(rp.RPError) as e:
        rp.Scene(scene)
    assert e.value.status == 3          # RP_ERR_CUDA
    assert "no CPU fallback" in str(e.value)


def test_record_layout_matches_header():
    from paper_2406_16302_gb300 import rp
    assert rp.RECORD_DTYPE.itemsize == 68


def test_null_arguments_are_refused_synchronously(lib):
    """Argument errors come back at once, without touching a device."""
    from paper_2406_16302_gb300 import rp
    assert lib.rp_sync_status(None) == 1            # RP_ERR_INVALID_ARG
    assert b"null" in lib.rp_last_error()
    assert lib.rp_get_stats(None, None) == 1
