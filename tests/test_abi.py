"""CPU-side checks of the boundary: the C header is valid C, libhav.so builds
for sm_103a, loads without a GPU, and exports every function include/hav.h
declares.  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hav.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hav_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libhav():
    from paper_2305_14306_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_is_plain_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "hav.h"\nint main(void) { hav_params p; (void)p; return 0; }\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I",
                    os.path.join(ROOT, "include"), str(src)], check=True)


def test_every_declared_symbol_is_exported(libhav):
    names = declared_functions()
    assert "hav_sample" in names and "hav_sample_batched" in names
    missing = [n for n in names if not hasattr(libhav, n)]
    assert not missing, missing


def test_binding_declares_the_same_names():
    from paper_2305_14306_gb300 import hav
    assert set(hav.EXPORTS) == set(declared_functions())


def test_struct_layouts_match_header(libhav, tmp_path):
    # sizes/offsets of the public structs as the C compiler sees them
    src = tmp_path / "s.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "hav.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(hav_params), sizeof(hav_layer_trace),'
        ' offsetof(hav_layer_trace, s), offsetof(hav_layer_trace, K), sizeof(hav_tuning),'
        ' offsetof(hav_tuning, chunk_min), offsetof(hav_tuning, small_points),'
        ' offsetof(hav_params, search), offsetof(hav_tuning, cluster_ctas)); return 0;}\n')
    exe = tmp_path / "s"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    from paper_2305_14306_gb300 import hav
    assert int(out[0]) == ctypes.sizeof(hav.hav_params)
    assert int(out[1]) == ctypes.sizeof(hav.hav_layer_trace)
    assert int(out[2]) == hav.hav_layer_trace.s.offset
    assert int(out[3]) == hav.hav_layer_trace.K.offset
    assert int(out[4]) == ctypes.sizeof(hav.hav_tuning)
    assert int(out[5]) == hav.hav_tuning.chunk_min.offset
    assert int(out[6]) == hav.hav_tuning.small_points.offset
    assert hav.hav_tuning.solo_points.offset == hav.hav_tuning.small_points.offset + 4
    assert int(out[7]) == hav.hav_params.search.offset
    assert int(out[8]) == hav.hav_tuning.cluster_ctas.offset


def test_params_default_and_status_strings(libhav):
    from paper_2305_14306_gb300 import hav
    hav.load()
    p = hav.params()
    assert (p.sigma_num, p.sigma_den, p.t_max, p.layers, p.layer_ratio) == (5, 100, 20, 2, 4)
    assert list(p.aspect) == [1.0, 1.0, 1.0]
    assert (p.select, p.fixed_s, p.search) == (0, 0.0, 0)
    for code in range(8):
        assert hav.load().hav_status_string(code)


def test_argument_errors_need_no_device(libhav):
    # invalid arguments are rejected before any CUDA call
    from paper_2305_14306_gb300 import hav
    L = hav.load()
    assert L.hav_context_create(None, 10, 1) == hav.HAV_ERR_INVALID
    h = ctypes.c_void_p()
    assert L.hav_context_create(ctypes.byref(h), 0, 1) == hav.HAV_ERR_INVALID
    assert L.hav_context_create(ctypes.byref(h), 10, 0) == hav.HAV_ERR_INVALID
    assert L.hav_context_create(ctypes.byref(h), 10, 257) == hav.HAV_ERR_INVALID
    assert L.hav_sample(None, None, 10, 5, None, None, None) == hav.HAV_ERR_INVALID
    assert L.hav_workspace_bytes(1 << 20, 1) > 0
    assert L.hav_context_get_tuning(None, None) == hav.HAV_ERR_INVALID
    assert L.hav_context_set_tuning(None, None) == hav.HAV_ERR_INVALID
    n = ctypes.c_uint64(7)
    assert L.hav_context_launches(None, ctypes.byref(n)) == hav.HAV_ERR_INVALID and n.value == 7
