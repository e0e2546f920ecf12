"""Host-side checks of the C ABI: the library builds, loads, and exports every
symbol that include/ndf.h declares; host-only helpers behave.  No kernel runs."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ndf_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2307_02203_gb300 import build

    return ctypes.CDLL(build.build())


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 14
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_2307_02203_gb300 import ndf

    assert _declared() <= set(ndf.exported_symbols())


def test_host_helpers(lib):
    from paper_2307_02203_gb300 import ndf

    assert ndf.ndf_index(3, 2, 1, 10, 5, 4) == (1 * 5 + 2) * 10 + 3
    assert ndf.ndf_index(10, 0, 0, 10, 5, 4) == -1
    assert ndf.ndf_status_str(ndf.NDF_ERR_ARG) == "invalid argument"
    assert ndf.ndf_status_str(ndf.NDF_ERR_TIMEOUT) == "device wait timed out"


def test_create_without_gpu_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2307_02203_gb300 import ndf

    with pytest.raises(ndf.NdfError) as ei:
        ndf.ndf_create(0)
    assert ei.value.status == ndf.NDF_ERR_CUDA


def test_null_context_is_rejected(lib):
    from paper_2307_02203_gb300 import ndf

    assert lib.ndf_synchronize(None) == ndf.NDF_ERR_ARG
    assert lib.ndf_launch_count(None) == 0


def _handle_calls():
    """(name, first parameter) of every ndf_status call on a context or model."""
    src = open(os.path.join(ROOT, "include", "ndf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = []
    for name, params in re.findall(r"\bndf_status\s+(ndf_\w+)\s*\(([^)]*)\)", src):
        first = params.split(",")[0]
        if re.search(r"\b(ndf_ctx|ndf_model|ndf_hash_model)\s*\*", first):
            out.append(name)
    return out


def test_null_handles_are_rejected(lib):
    """Every call on a context or model returns NDF_ERR_ARG for a NULL handle
    (checked on the host before anything else), whatever the other arguments."""
    from paper_2307_02203_gb300 import ndf

    names = _handle_calls()
    assert len(names) >= 40
    for name in names:
        f = getattr(ndf._lib, name)
        args = []
        for t in f.argtypes:
            if isinstance(t, type) and issubclass(t, ctypes.Structure):
                args.append(t())
            elif t in (ctypes.c_float, ctypes.c_double):
                args.append(0.0)
            elif isinstance(t, type) and issubclass(t, ctypes._SimpleCData) and t not in (
                    ctypes.c_void_p, ctypes.c_char_p):
                args.append(0)
            else:
                args.append(None)
        assert f(*args) == ndf.NDF_ERR_ARG, name
    assert ndf._lib.ndf_pearson_noalloc(None, None, 2, 1, 0, None, None) == ndf.NDF_ERR_ARG


def test_noalloc_pointer_rule(lib):
    """ndf_pearson_noalloc accepts device memory of the current device and managed
    memory, and rejects host memory and memory of another GPU (the rule itself is
    a host function, so a second GPU is not needed to check it)."""
    from paper_2307_02203_gb300 import ndf

    assert ndf.ndf_noalloc_pointer_usable(True, False, 0, 0)
    assert ndf.ndf_noalloc_pointer_usable(True, False, 3, 3)
    assert not ndf.ndf_noalloc_pointer_usable(True, False, 1, 0)   # another GPU's memory
    assert not ndf.ndf_noalloc_pointer_usable(True, False, 0, 1)
    assert ndf.ndf_noalloc_pointer_usable(False, True, 1, 0)       # managed: every device
    assert not ndf.ndf_noalloc_pointer_usable(False, False, 0, 0)  # host memory
