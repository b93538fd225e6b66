"""The C ABI without a GPU: the library builds, loads and exports every
entry point declared in include/hivision.h; host-side argument checks."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hivision.h")


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z0-9_]+\s*\*?\s*(hv_[a-z0-9_]+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2005_12489_gb300 import build
    build.build()
    from paper_2005_12489_gb300 import hv
    return hv


def test_header_declares_the_boundary():
    names = declared()
    for n in ("hv_create", "hv_destroy", "hv_last_error", "hv_layer_load_points",
              "hv_layer_load_linestrings", "hv_layer_load_polygons", "hv_layer_build_index",
              "hv_render_tiles", "hv_layer_save", "hv_layer_load_file", "hv_layer_free",
              "hv_server_start", "hv_server_submit", "hv_server_poll", "hv_server_stop"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.lib()
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    assert sorted(lib.SIGNATURES) == declared()


def test_host_only_calls(lib):
    assert lib.hv_tile_bytes(lib.HV_MODE_MASK) == 8192
    assert lib.hv_tile_bytes(lib.HV_MODE_COVERAGE) == 65536
    assert lib.hv_tile_bytes(lib.HV_MODE_RGBA) == 262144
    assert lib.hv_tile_bytes(9) == 0
    assert lib.REQ_DTYPE.itemsize == 16
    L = lib.lib()
    assert L.hv_render_tiles(None, None, 0, 0, 1, None, None, 0, None) == lib.HV_EINVAL
    assert "NULL layer" in lib.hv_last_error()
    assert L.hv_layer_build_index(None, 1, None) == lib.HV_EINVAL
    assert L.hv_layer_free(None) == lib.HV_EINVAL
    assert L.hv_destroy(None) == lib.HV_EINVAL


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="a GPU is present")
def test_create_without_gpu_reports_error(lib):
    with pytest.raises(lib.HVError) as e:
        lib.hv_create(0)
    assert e.value.status in (lib.HV_ECUDA, lib.HV_EINVAL)


def test_missing_library_fails_loudly():
    """Without the CUDA library every call raises: there is no CPU fallback."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2005_12489_gb300 import hv\n"
            "hv.LIB_PATH = '/nonexistent/libhivision.so'\n"
            "try:\n"
            "    hv.hv_create(0)\n"
            "except ImportError as e:\n"
            "    print('raised', e)\n"
            "    sys.exit(0)\n"
            "sys.exit(3)\n" % root)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and "not built" in out.stdout, out.stdout + out.stderr
