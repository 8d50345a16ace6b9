"""Host-side checks of the C-ABI that need no GPU: the library builds for sm_103a,
loads, exports every function include/soliton.h declares, and rejects bad
arguments before touching the device."""
import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+(?:\s+\w+)?\s*\*?\s*(ss_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2603_24370_gb300 import build
    from paper_2603_24370_gb300 import soliton as S
    build.build()
    return S.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ss_create_grid", "ss_set_theory", "ss_init_ansatz", "ss_step", "ss_minimise",
                     "ss_observables", "ss_destroy", "ss_last_error", "ss_batch_create", "ss_batch_minimise",
                     "ss_net_create", "ss_net_train_step", "ss_net_predict", "ss_net_save", "ss_net_load"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_empty_error(lib):
    assert lib.ss_version() >= 1
    assert isinstance(lib.ss_last_error(), bytes)


@pytest.mark.parametrize("nx,ny,dx,dy,prec", [
    (4, 10, 0.1, 0.1, 1),      # below the 5-site minimum (halo 2 on each side)
    (10, 3, 0.1, 0.1, 1),
    (10, 10, 0.0, 0.1, 1),     # non-positive spacing
    (10, 10, 0.1, -1.0, 2),
    (10, 10, float("nan"), 0.1, 2),
    (10, 10, 0.1, 0.1, 4),     # unknown precision
])
def test_create_grid_rejects_bad_arguments_on_the_host(lib, nx, ny, dx, dy, prec):
    from paper_2603_24370_gb300 import soliton as S
    ctx = ctypes.c_void_p(1234)
    rc = lib.ss_create_grid(ctypes.byref(ctx), nx, ny, dx, dy, prec, None)
    assert rc == S.SS_ERR_ARG
    assert ctx.value is None
    assert len(S.last_error()) > 0


def test_null_context_is_rejected(lib):
    from paper_2603_24370_gb300 import soliton as S
    assert lib.ss_step(None, 1, None) == S.SS_ERR_ARG
    assert lib.ss_observables(None, None) == S.SS_ERR_ARG
    assert lib.ss_destroy(None) == S.SS_OK


def test_built_for_sm_103a_only():
    from paper_2603_24370_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_product_path_does_not_reach_the_oracle():
    """The package never imports, links or opens anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_2603_24370_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "soliton_oracle" not in text and "liboracle" not in text, fn
