"""The C ABI library builds, loads without a GPU and exports every symbol that
include/chebrbm.h declares; the Python binding fails loudly without CUDA."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "chebrbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[a-z_ ]*?\b(?:cr_status|int|long long|size_t|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return set(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2103_08804_gb300 import build
    return build.build()


def test_header_declares_the_hot_path_calls():
    d = _declared()
    for name in ("rbm_logpsi", "mc_sweep", "cheb_local_target", "logderiv", "logpsi_backward",
                 "sr_step", "cheb_moment", "cheb_gram", "cheb_krylov"):
        assert name in d


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _declared() - exported
    assert not missing, missing
    from paper_2103_08804_gb300 import api
    assert set(api.SYMBOLS) == _declared()
    lib = api.load(lib_path)
    for name in _declared():
        assert hasattr(lib, name)


def test_binding_refuses_to_run_without_cuda(monkeypatch):
    import torch
    from paper_2103_08804_gb300 import api
    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    with pytest.raises(RuntimeError):
        api.Context(4, 1, 4, 8)


def test_null_context_and_bad_arguments_are_rejected(lib_path):
    import ctypes
    from paper_2103_08804_gb300 import api
    lib = api.load(lib_path)
    assert lib.cr_destroy(None) == 1
    assert lib.cr_sync_status(None) == 1
    h = ctypes.c_void_p()
    bad = api.Lattice(2, 1, 1.0)  # Lx < 3
    assert lib.cr_create(ctypes.byref(h), ctypes.byref(bad), 4, 8, 0, 0, None) == 1
    odd = api.Lattice(5, 1, 1.0)  # no S^z = 0 sector
    assert lib.cr_create(ctypes.byref(h), ctypes.byref(odd), 4, 8, 0, 0, None) == 1
    ok = api.Lattice(4, 1, 1.0)
    assert lib.cr_create(ctypes.byref(h), ctypes.byref(ok), 600, 8, 0, 0, None) == 1  # M > 512
    # the symmetry projection: no context, no workspace size, no call
    assert lib.sym_workspace_bytes(None, 8) == 0
    assert lib.sym_h_workspace_bytes(None, 8) == 0
    assert lib.sym_btilde(None, None, 1, None, None, 8, None, 0, None) == 1
    hp = (ctypes.c_double * 3)(0.0, 1.0, 0.0)
    assert lib.sym_hbtilde(None, None, 1, None, None, 8, hp, None, 0, None, None) == 1
