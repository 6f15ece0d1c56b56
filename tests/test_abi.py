"""The C-ABI library builds, loads and exports every symbol include/*.h
declares (no GPU needed: nothing here calls into CUDA)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1206_6409_gb300 import build
    return build.build()


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gencd_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("gencd_create", "gencd_set_lambda", "gencd_set_params", "gencd_solve", "gencd_get_w",
                     "gencd_objective", "gencd_propose_at", "gencd_destroy", "gencd_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)", out))
    assert exported == set(_declared()), exported ^ set(_declared())


def test_binding_covers_the_header(libpath):
    from paper_1206_6409_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()
    for name in binding.EXPORTS:
        assert callable(getattr(binding, name))
    binding.lib()


def test_build_targets_sm_103a_only():
    from paper_1206_6409_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_errors_cross_the_abi_as_codes(libpath):
    from paper_1206_6409_gb300 import binding as gb
    with pytest.raises(gb.GencdError) as e:
        gb._check(gb.lib().gencd_set_lambda(None, 1.0))
    assert e.value.code == gb.GENCD_EINVAL
    assert "NULL" in gb.gencd_last_error()
    p = gb.gencd_params()
    assert gb.lib().gencd_default_params(ctypes.byref(p)) == 0
    assert p.variant == gb.GENCD_THREAD_GREEDY and p.tol_kkt == 1e-8 and p.check_every == 10
