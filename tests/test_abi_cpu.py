"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every function include/*.h declares (no compute calls without a GPU)."""
import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header="cagra_gb.h"):
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", header)):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w \*]*?\b([A-Za-z_]\w*)\s*\(", txt,
                            flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1608_01362_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    from paper_1608_01362_gb300 import cagra
    declared = _declared()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert sorted(cagra.EXPORTS) == declared


def test_probe_library_is_separate(lib):
    """The benchmark's measurement probes live in libcagra_probes.so, declared
    in include/cagra_probes.h; the product library does not export them."""
    from paper_1608_01362_gb300 import build, probes
    plib = ctypes.CDLL(build.PROBES_LIB)
    declared = _declared("cagra_probes.h")
    assert declared == sorted(probes.EXPORTS)
    for name in declared:
        assert hasattr(plib, name)
        assert not hasattr(lib, name), f"{name} exported by the product library"
    assert sorted(set(glob.glob(os.path.join(ROOT, "include", "*.h")))) == sorted(
        os.path.join(ROOT, "include", h) for h in ("cagra_gb.h", "cagra_probes.h"))


def test_status_strings_without_gpu(lib):
    lib.cg_status_string.restype = ctypes.c_char_p
    lib.cg_last_error_message.restype = ctypes.c_char_p
    assert lib.cg_status_string(0) == b"CG_OK"
    assert lib.cg_status_string(-1) == b"CG_ERR_INVALID_ARG"
    assert lib.cg_version() >= 100
    # argument checks run on the host before any CUDA call
    lib.pr_build_segments.restype = ctypes.c_int
    out = ctypes.c_void_p()
    st = lib.pr_build_segments(None, None, ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int32(1),
                               None, ctypes.c_int32(16), ctypes.byref(out), None)
    assert st == -1 and b"V must be" in lib.cg_last_error_message()
    q = ctypes.c_double(-1.0)
    assert lib.cg_segmented_stats(None, None, ctypes.byref(q), None) == -1
    assert b"null handle" in lib.cg_last_error_message() and q.value == -1.0


def test_binding_refuses_without_library(tmp_path):
    from paper_1608_01362_gb300 import cagra
    with pytest.raises(cagra.CagraError):
        saved = cagra._lib
        cagra._lib = None
        try:
            cagra.load(str(tmp_path / "missing.so"))
        finally:
            cagra._lib = saved
