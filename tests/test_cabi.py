"""CPU checks of the C ABI: the library loads, exports every declared symbol, and the
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pid.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pid_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_15187_gb300 import build, binding
    build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pid_soft_masks", "pid_from_fields", "pid_mean", "pid_batch", "pid_full"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert missing == []


def test_binding_mirrors_every_export(lib):
    from paper_2512_15187_gb300 import binding
    for n in _declared():
        assert n in binding.EXPORTS, n


def test_null_handle_is_rejected_on_the_host(lib):
    from paper_2512_15187_gb300 import binding as B
    assert lib.pid_mean(None, None, 4, 10, 10, None, None, None, None, None, None) == \
        B.PID_ERR_INVALID_ARG
    assert lib.pid_full(None, None, 4, 10, 10, None, None, None, None, None, None, None, None,
                        None) == B.PID_ERR_INVALID_ARG
    assert lib.pid_status_string(B.PID_ERR_DOMAIN).startswith(b"input outside")
    assert lib.pid_destroy(None) == B.PID_OK


def test_struct_layout_matches_header():
    from paper_2512_15187_gb300 import binding as B
    assert ctypes.sizeof(B.pid_iso) == 24
    assert ctypes.sizeof(B.pid_options) == 16
    # data, N, M, ld, w, is_field+reserved, iso, opt, 8 output pointers
    assert ctypes.sizeof(B.pid_ensemble) == 8 * 5 + 8 + 24 + 16 + 8 * 8


def test_serving_structs_and_host_checks(lib):
    import ctypes
    from paper_2512_15187_gb300 import binding as B
    assert ctypes.sizeof(B.pid_serve_cfg) == 40
    assert ctypes.sizeof(B.pid_serve_stats) == 88
    out = ctypes.c_void_p()
    assert lib.pid_serve_start(ctypes.byref(out), None) == B.PID_ERR_INVALID_ARG
    bad = B.pid_serve_cfg(0, 0, 1, 1, 0, 0, 0)           # max_inflight < 1
    assert lib.pid_serve_start(ctypes.byref(out), ctypes.byref(bad)) == B.PID_ERR_INVALID_ARG
    assert lib.pid_serve_stop(None) == B.PID_OK


def test_bands_host_checks(lib):
    from paper_2512_15187_gb300 import binding as B
    assert lib.pid_contour_bands(None, None, 4, 10, 10, None, None, 0.5, 0.5, None, None) == \
        B.PID_ERR_INVALID_ARG


def test_binding_rejects_tensors_a_kernel_cannot_read():
    # host tensors, wrong dtypes and wrong lengths fail in the binding, before any call
    import torch

    from paper_2512_15187_gb300 import binding as B
    with pytest.raises(ValueError):
        B._check_matrix(torch.zeros(2, 3), "data")                      # host memory
    with pytest.raises(ValueError):
        B._check_matrix(torch.zeros(2, 3, dtype=torch.float64), "data")
    dev = torch.device("cuda", 0)
    assert B._weights(None, 3, dev) is None
    with pytest.raises(ValueError):
        B._weights(torch.ones(3), 3, dev)                                # host memory
    iso = B.make_iso((0.5, 0.1, 1, "uniform"))
    assert (iso.kind, iso.superlevel, iso.mu, iso.sigma) == (B.PID_ISO_UNIFORM, 1, 0.5, 0.1)
    assert B.make_iso((0.5, 0.05)).kind == B.PID_ISO_NORMAL
    with pytest.raises(KeyError):
        B.make_iso((0.5, 0.1, 0, "triangle"))
