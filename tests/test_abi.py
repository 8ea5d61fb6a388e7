"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/lrp.h (no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(lrp_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("lrp_build_coarse", "lrp_parareal_solve", "lrp_propagate", "lrp_create"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2508_08873_gb300 import _native
    lib = _native.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers every declared entry point
    bound = {s[0] for s in _native.SIGNATURES}
    assert set(declared_functions()) <= bound, set(declared_functions()) - bound


def test_status_strings_without_gpu():
    from paper_2508_08873_gb300 import _native
    lib = _native.load()
    assert lib.lrp_status_string(0) == b"ok"
    assert lib.lrp_status_string(3).startswith(b"not converged")


def test_create_fails_cleanly_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    from paper_2508_08873_gb300 import _native, api
    with pytest.raises(_native.LrpError):
        api.Context(0)


def test_every_parameter_is_documented_and_readable():
    """Every name lrp_set_param accepts is documented in include/lrp.h and
    readable back through lrp_get_param."""
    api = open(os.path.join(ROOT, "paper_2508_08873_gb300", "csrc", "api.cu")).read()
    i = api.index("lrp_status lrp_set_param")
    j = api.index("lrp_status lrp_get_param")
    k = api.index("\n}\n", j)
    set_names = set(re.findall(r'k == "([a-z0-9_]+)"', api[i:j]))
    get_names = set(re.findall(r'k == "([a-z0-9_]+)"', api[j:k]))
    header = open(os.path.join(ROOT, "include", "lrp.h")).read()
    assert {"tri_refine", "tri_refine_rounds", "tri_refine_cluster", "krylov_refine"} <= set_names
    assert not [n for n in set_names | get_names if '"%s"' % n not in header]
    assert set_names <= get_names, set_names - get_names
