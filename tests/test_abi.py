"""Host-side checks of the C ABI (no GPU needed): the library builds and
exports every entry point include/bez.h declares, and argument errors are
reported before any CUDA work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(bez_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libbez():
    from paper_2603_15447_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["bez_create", "bez_destroy", "bez_last_error", "bez_eval"]:
        assert required in names


def test_every_declared_symbol_is_exported(libbez):
    missing = [n for n in declared_functions() if not hasattr(libbez, n)]
    assert not missing, f"declared in include/*.h but not exported: {missing}"


def test_argument_errors_without_gpu(libbez):
    from paper_2603_15447_gb300 import bez
    L = bez.lib()
    o = bez.Opts(0, 0, 0, 0, 0, 0, 0, None)
    # null context is rejected on the host
    st = L.bez_eval(None, None, 1, 3, 3, None, 4, None, ctypes.byref(o), None)
    assert st == bez.Status.INVALID_ARG
    assert b"context" in L.bez_last_error()
    assert L.bez_version().startswith(b"bez")


def test_create_reports_missing_device_cleanly(libbez):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2603_15447_gb300 import bez
    h = ctypes.c_void_p()
    st = bez.lib().bez_create(ctypes.byref(h), 0)
    assert st in (bez.Status.CUDA, bez.Status.INVALID_ARG)
    assert not h.value


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no fallback: without libbez.so every call raises instead of computing
    # anything elsewhere
    from paper_2603_15447_gb300 import bez
    monkeypatch.setattr(bez, "_lib", None)
    monkeypatch.setattr(bez, "LIB_PATH", str(tmp_path / "libbez.so"))
    with pytest.raises(RuntimeError, match="libbez.so not found"):
        bez.lib()
    import numpy as np
    with pytest.raises(RuntimeError, match="libbez.so not found"):
        bez.bez_eval(np.zeros((2, 4, 3), np.float32), np.zeros(3, np.float32))


def test_noalloc_binding_refuses_arrays_on_different_gpus():
    # bez_eval_spline_noalloc runs on the current device and never switches
    # devices; the binding makes the arrays' device current and refuses a
    # call whose arrays sit on two GPUs before reaching the library
    from paper_2603_15447_gb300 import bez

    class FakeDevice:
        def __init__(self, index):
            self.index = index

    class FakeCudaTensor:
        is_cuda = True

        def __init__(self, index):
            self.device = FakeDevice(index)

    a, b = FakeCudaTensor(0), FakeCudaTensor(1)
    assert bez._common_device(a, None, FakeCudaTensor(0)) == 0
    assert bez._common_device(None, None) is None
    with pytest.raises(bez.BezError) as e:
        bez._common_device(a, None, b)
    assert e.value.status == bez.Status.INVALID_ARG and "different GPUs" in str(e.value)
