"""The C ABI library builds for sm_103a, loads without a GPU and exports
every function that include/wln.h declares (no compute calls here)."""
import ctypes
import os

import numpy as np
import pytest

from paper_1407_7486_gb300 import build, wln


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    assert os.path.exists(path)
    return wln.load(path)


def test_header_and_binding_agree():
    assert wln.header_symbols() == sorted(wln.SIGNATURES)


def test_library_exports_every_declared_symbol(lib):
    for name in wln.header_symbols():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm103a():
    log = open(os.path.join(os.path.dirname(build.LIB), "ptxas.log")).read()
    assert "sm_103a" in log
    assert "wilson_kernel" in log


def test_create_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.wln_create(ctypes.byref(h), 0, None)
    assert st == 3 and not h.value           # WLN_ECUDA, no context


def test_null_arguments_are_rejected_without_a_device(lib):
    assert lib.wln_destroy(None) == 1
    assert lib.wln_synchronize(None) == 1
    assert lib.wln_last_error(None) == b"no context"
    assert lib.wln_ensemble_info(None, None, None, None) == 1


def test_mapped_grid_helper_matches_oracle_nodes():
    # host-only helper of the C ABI (no GPU work): nodes of x = 1/(1 + v/scale)
    from oracle import stats as ost
    for n, scale, start in ((64, 1.0, 0.01), (33, 2.5, 0.0), (1, 1.0, 0.3), (7, 0.2, 5.0)):
        np.testing.assert_allclose(wln.mapped_grid(n, scale, start),
                                   ost.mapped_nodes(n, scale, start), rtol=1e-15, atol=0)
    with pytest.raises(wln.WlnError):
        wln.mapped_grid(4, -1.0, 0.0)


def _build_c_example(tmp_path):
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    lib = build.build()
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    exe = str(tmp_path / "c_api_example")
    subprocess.check_call([gcc, "-O2", "-I", os.path.join(root, "include"),
                           os.path.join(here, "c_api_example.c"), "-L", os.path.dirname(lib),
                           "-lwln", f"-Wl,-rpath,{os.path.dirname(lib)}", "-o", exe])
    return exe


def test_c_example_compiles_and_links_against_the_library(tmp_path):
    # the header is plain C and every symbol the example uses resolves in libwln.so
    assert os.path.exists(_build_c_example(tmp_path))
