"""The C-ABI library builds for sm_103a, loads, and exports every function the
public header declares.  CPU only: no call here touches a GPU."""
import ctypes
import importlib.util
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _buildlib():
    path = os.path.join(ROOT, "paper_1609_01839_gb300", "buildlib.py")
    spec = importlib.util.spec_from_file_location("gfd_buildlib_t", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def libpath():
    try:
        return _buildlib().build()
    except RuntimeError as e:  # nvcc missing
        pytest.skip(str(e))


def header_decls():
    text = open(os.path.join(ROOT, "include", "gfdeconv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gfdeconv_\w+)\s*\(", text)))


def test_header_declares_expected_entry_points():
    names = header_decls()
    for required in ("gfdeconv_create", "gfdeconv_destroy", "gfdeconv_solve",
                     "gfdeconv_solve_batched", "gfdeconv_guidfilter", "gfdeconv_status",
                     "gfdeconv_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in header_decls() if not hasattr(lib, n)]
    assert not missing, missing
    # dynamic symbol table says the same (C linkage, no mangling)
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(gfdeconv_\w+)", out))
    assert set(header_decls()) <= exported


def test_build_targets_sm_103a_only():
    """The build compiles every unit for sm_103a and nothing else (the loaded
    kernels' binaryVersion is checked at run time by the GPU tests)."""
    b = _buildlib()
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_arch_query_fails_cleanly_without_a_gpu(libpath):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: covered by the GPU tests")
    lib = ctypes.CDLL(libpath)
    lib.gfdeconv_device_arch.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    b = ctypes.c_int(-7)
    assert lib.gfdeconv_device_arch(0, ctypes.byref(b), None) == -5  # GFD_ERR_CUDA
    assert b.value == -7  # nothing written


def test_host_only_calls(libpath):
    lib = ctypes.CDLL(libpath)
    lib.gfdeconv_strerror.restype = ctypes.c_char_p
    lib.gfdeconv_strerror.argtypes = [ctypes.c_int]
    assert lib.gfdeconv_strerror(0) == b"ok"
    assert b"power" in lib.gfdeconv_strerror(-2)
    # null context / arguments are rejected on the host before any CUDA call
    lib.gfdeconv_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.gfdeconv_create(None, 0, None) == -1
    lib.gfdeconv_solve_batched.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_int, ctypes.c_void_p]
    assert lib.gfdeconv_solve_batched(None, 1, None, 1, None) == -1
    lib.gfdeconv_last_launch_count.restype = ctypes.c_longlong
    lib.gfdeconv_last_launch_count.argtypes = [ctypes.c_void_p]
    assert lib.gfdeconv_last_launch_count(None) == -1


def test_binding_struct_matches_header_layout(libpath):
    """The ctypes mirror of gfdeconv_image has the C layout (sizes/offsets)."""
    import paper_1609_01839_gb300 as gfd
    names = [f[0] for f in gfd.Image._fields_]
    text = open(os.path.join(ROOT, "include", "gfdeconv.h")).read()
    body = text[text.index("typedef struct {\n  const float* y;"):text.index("} gfdeconv_image;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"[\w\*\s]+?\b(\w+)\s*[,;]", body)
    assert names == fields, (names, fields)
    assert ctypes.sizeof(gfd.Image) == 8 + 4 + 4 + 8 + 4 + 4 + 8 + 8 + 8 + 9 * 8


def test_binding_constants_match_the_header(libpath):
    """Every status bit, arithmetic, boundary and error code the header
    defines has the same value in the binding."""
    import paper_1609_01839_gb300 as gfd
    text = open(os.path.join(ROOT, "include", "gfdeconv.h")).read()
    defs = dict(re.findall(r"#define GFD_((?:STATUS|VAR|BOUNDARY)_\w+)\s+(-?\d+)", text))
    defs.update(re.findall(r"GFD_(ERR_\w+)\s*=\s*(-?\d+)", text))
    assert {"STATUS_PASSES_EXHAUSTED", "STATUS_COPY_TIMEOUT", "VAR_COMPENSATED",
            "BOUNDARY_TRUNCATED", "ERR_INVALID_ARG"} <= set(defs)
    for name, value in defs.items():
        if hasattr(gfd, name):
            assert getattr(gfd, name) == int(value), name
    for name in ("STATUS_NONCONVERGED", "STATUS_NONFINITE", "STATUS_BAD_PSF", "STATUS_BAD_RHO",
                 "STATUS_PASSES_EXHAUSTED", "STATUS_COPY_TIMEOUT", "VAR_COMPENSATED", "VAR_FP64",
                 "VAR_FP32", "VAR_FP32_RAW", "VAR_DOUBLE_FLOAT", "BOUNDARY_PERIODIC",
                 "BOUNDARY_TRUNCATED", "ERR_INVALID_ARG", "ERR_SCRATCH_LIMIT"):
        assert getattr(gfd, name) == int(defs[name]), name
