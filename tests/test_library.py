"""CPU checks of the C ABI library: it builds for sm_103a, loads without a GPU
and exports every function that include/ghostmg.h declares, and the Python
binding declares the same set (no compute calls: this container has no GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ghostmg.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mg(?:1d)?_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2505_05105_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    fns = declared_functions()
    for name in ("mg_setup", "mg_solve", "mg_adjoint", "mg_destroy", "mg_strerror",
                 "mg1d_cycles"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mg(?:1d)?_[a-z_0-9]+)$", out, flags=re.M))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_binding_matches_header(lib_path):
    from paper_2505_05105_gb300 import ghostmg
    assert sorted(ghostmg.SIGNATURES) == declared_functions()
    lib = ghostmg.load()
    for name in declared_functions():
        assert hasattr(lib, name)
    # pure host calls (no device work)
    s = ghostmg.mg_default_stab()
    assert (s.gamma, s.alpha, s.eta, s.nu1, s.nu2) == (2.0, 1.75, 4, 2, 1)
    assert ghostmg.mg_strerror(ghostmg.MG_ERR_NOT_SPD).startswith("coarsest")


def test_build_targets_sm103a_only():
    from paper_2505_05105_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_checks_packed_sizes_before_any_call(lib_path):
    """mg1d_cycles refuses packed arrays shorter than the problems need on
    the host, before the library is called."""
    import numpy as np
    import pytest
    from paper_2505_05105_gb300 import ghostmg
    with pytest.raises(ValueError):
        ghostmg.mg1d_cycles([(64, 0.5, 0.5, 10.0), (32, 0.3, 0.2, 5.0)], np.zeros(97))
    # the stab structure carries the global-penalty fields
    s = ghostmg.mg_default_stab()
    assert s.lambda_mode == ghostmg.MG_LAMBDA_LOCAL and s.c_global == 0.0
