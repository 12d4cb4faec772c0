"""The C-ABI library builds, loads and exports every function include/*.h declares.

No compute call is made here, so these run without a GPU.
"""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                             src, flags=re.M):
            name = m.group(1)
            if name not in ("sizeof", "defined"):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1302_7203_gb300 import build
    try:
        return build.build()
    except RuntimeError as e:   # no toolkit on this machine
        pytest.skip(str(e))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for fn in ("arrow_eig", "arrow_eig_host", "ae_default_opts", "ae_status_string",
               "ae_last_cuda_error", "ae_debug_rcp"):
        assert fn in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [f for f in sorted(declared_functions()) if not hasattr(L, f)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_1302_7203_gb300 import arrowhead
    assert set(arrowhead.EXPORTED) == declared_functions()


def test_host_side_helpers_without_gpu(libpath):
    from paper_1302_7203_gb300 import arrowhead
    o = arrowhead.default_opts()
    assert o.precision == arrowhead.AE_FP64 and o.max_iter == 2200 and o.fixup == 1
    assert abs(o.knu_max - 10.0) == 0.0
    L = arrowhead.lib()
    assert L.ae_status_string(0) == b"ok"
    assert L.ae_status_string(-3) == b"invalid argument"
    # argument checks happen before any CUDA call
    assert L.arrow_eig(0, None, None, 0.0, None, None, 0, None, None, None, None, None,
                       None) == -1
    assert L.arrow_eig(3, None, None, 0.0, None, None, 0, None, None, None, None, None,
                       None) == -2


def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    from paper_1302_7203_gb300 import arrowhead
    monkeypatch.setattr(arrowhead, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(arrowhead, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        arrowhead.lib()
