"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry point
declared in include/blacklight.h. No compute calls here."""
import ctypes
import os
import re

from paper_2203_15963_gb300 import native

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "blacklight.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(blacklight_\w+)\s*\(", text)))


def test_library_builds_loads_and_exports_header_symbols():
    native.build()
    lib = ctypes.CDLL(native.library_path())
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_sizes_match_header_layout():
    # the binding's ctypes structs follow the C layout; the library checks .size at run time
    assert ctypes.sizeof(native.Camera) == 4 + 4 + 8 * 3 + 8 * 3 + 8 * 3 + 8 + 4 + 4 + 8 + 4 + 4
    assert ctypes.sizeof(native.Out) == 64


def test_ctypes_struct_sizes_equal_the_c_compilers(tmp_path):
    """Compile the header with the host C compiler and compare every struct's size and the
    parameter count with the binding's ctypes mirrors."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no host C compiler")
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "blacklight.h"\nint main(void) {\n'
                   ' printf("%zu %zu %zu %zu %zu %zu %d\\n", sizeof(bl_camera_t), sizeof(bl_metric_t),'
                   ' sizeof(bl_grid_t), sizeof(bl_out_t), sizeof(bl_adapt_t), sizeof(bl_mlp_train_t),'
                   ' BL_MLP_PARAMS);\n printf("%zu %zu\\n", sizeof(bl_launch_config_t), sizeof(bl_peaks_t));\n'
                   ' return 0;\n}\n')
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    want = [ctypes.sizeof(native.Camera), ctypes.sizeof(native.Metric),
            ctypes.sizeof(native.Grid), ctypes.sizeof(native.Out), ctypes.sizeof(native.Adapt),
            ctypes.sizeof(native.MlpTrain), native.MLP_PARAMS, ctypes.sizeof(native.LaunchConfig),
            ctypes.sizeof(native.Peaks)]
    assert got == want


def test_strerror_without_gpu():
    L = native.load()
    assert L.blacklight_strerror(-1) == b"invalid argument"
    assert L.blacklight_strerror(0) == b"success"
