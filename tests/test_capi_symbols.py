"""The C-ABI library builds for sm_103a and exports every entry point of include/ar.h."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ar.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ar_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_boundary():
    names = _declared()
    for must in ["ar_scene_create", "ar_scene_destroy", "ar_render_abstract", "ar_serve_submit",
                 "ar_serve_poll", "ar_last_error"]:
        assert must in names


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_exports_every_symbol():
    from paper_2503_00308_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)   # loads without a GPU: no CUDA call happens at load time
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_last_error_without_gpu_calls():
    from paper_2503_00308_gb300 import _build, ar
    _build.build()
    # argument validation happens before any CUDA call, and sets the thread's message
    with pytest.raises(ar.ArError) as e:
        ar.ar_scene_create(None, None, None, None, None, -1, 0)
    assert e.value.code == ar.AR_EINVAL
    assert ar.ar_last_error() != ""
    with pytest.raises(ar.ArError) as e:
        ar.ar_scene_set_blend(None, ar.AR_BLEND_RELATIONAL)
    assert e.value.code == ar.AR_EINVAL
