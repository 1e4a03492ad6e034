"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/rbffd.h declares (no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rbffd.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbffd_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2206_06495_gb300 import build
    return build.build()


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ("rbffd_build_weights", "rbffd_apply_op", "rbffd_step", "rbffd_create",
              "rbffd_destroy", "rbffd_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_prototypes_cover_header(libpath):
    from paper_2206_06495_gb300 import rbffd
    assert set(rbffd.PROTOTYPES) == set(_declared())
    lib = rbffd.lib()
    assert lib.rbffd_version() >= 100


def test_struct_layouts_match_header(libpath):
    """ctypes mirrors of the ABI structs have the sizes the compiler gives them."""
    from paper_2206_06495_gb300 import rbffd
    import subprocess
    import tempfile
    code = r'''
#include <stdio.h>
#include "rbffd.h"
int main(){printf("%zu %zu %zu %zu %zu %zu\n", sizeof(rbffd_params), sizeof(rbffd_ell),
 sizeof(rbffd_flow), sizeof(rbffd_state), sizeof(rbffd_stats), (size_t)0);return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "s")
        inc = "/usr/local/cuda/include"
        r = subprocess.run(["gcc", c, "-I", os.path.join(ROOT, "include"), "-I", inc, "-o", exe],
                           capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("no C compiler / CUDA headers: " + r.stderr[:200])
        sizes = [int(v) for v in subprocess.run([exe], capture_output=True,
                                                text=True).stdout.split()]
    assert sizes[:5] == [ctypes.sizeof(rbffd.Params), ctypes.sizeof(rbffd.Ell),
                         ctypes.sizeof(rbffd.FlowC), ctypes.sizeof(rbffd.StateC),
                         ctypes.sizeof(rbffd.Stats)]


def test_product_path_has_no_cpu_fallback():
    """The binding refuses to run without a GPU instead of computing on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2206_06495_gb300 import rbffd
    with pytest.raises(RuntimeError):
        rbffd.Context()
