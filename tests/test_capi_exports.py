"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/nls.h (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nls.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(nls_[a-z_0-9]+)\s*\(",
                                 text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_16341_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_api():
    fns = declared_functions()
    for name in ("nls_batch_create", "nls_solve", "nls_status", "nls_batch_destroy"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_2403_16341_gb300 as nls
    assert set(nls.EXPORTED) == set(declared_functions())
    for f in declared_functions():
        assert callable(getattr(nls, f))


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2403_16341_gb300 as nls
    with pytest.raises(nls.NlsError):
        nls.nls_batch_create(0)


def test_header_enum_values_match_binding():
    import paper_2403_16341_gb300 as nls
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    found = 0
    for name, expr in re.findall(r"\b(NLS_[A-Z0-9_]+)\s*=\s*(-?\d+(?:\s*<<\s*\d+)?)", text):
        a, _, b = expr.partition("<<")
        value = int(a) << int(b) if b else int(a)
        assert getattr(nls, name) == value, name
        found += 1
    assert found >= 30
