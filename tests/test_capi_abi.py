"""CPU checks of the C ABI: the sm_103a library builds, loads, and exports every
entry point that include/csem.h declares, with the binding's signatures.  No
compute call is made here (there is no GPU on this side)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "csem.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(csem_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_16665_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_four_paper_calls():
    names = declared_functions()
    for n in ("csem_fwd_model", "csem_adjoint_model", "csem_gradient", "csem_estimate_adjoint_basis"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2211_16665_gb300 import _capi
    assert set(declared_functions()) == set(_capi.SIGNATURES)


def test_binding_loads_library(lib):
    from paper_2211_16665_gb300 import _capi
    L = _capi.lib()
    assert L.csem_last_error() == b""


def test_struct_layouts_match_header_sizes():
    from paper_2211_16665_gb300 import _capi
    # pointer-sized fields on LP64: grid = 3 ints (+pad) + 3 ptrs + int (+pad)
    assert ctypes.sizeof(_capi.Grid) == 48
    assert ctypes.sizeof(_capi.PointsC) == 40
    assert ctypes.sizeof(_capi.Info) == 88
    assert ctypes.sizeof(_capi.Opts) == 88


def test_header_is_plain_c(tmp_path):
    """The boundary is a C ABI: the header compiles as C99 with warnings as errors."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    src = tmp_path / "use.c"
    src.write_text('#include "csem.h"\nint main(void) { csem_opts o = {0}; o.order = 4; return o.order - 4; }\n')
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), "-c",
                    str(src), "-o", str(tmp_path / "use.o")], check=True)
