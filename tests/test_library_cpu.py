"""CPU-only checks of the C-ABI library: it builds, loads, exports every
function declared in include/rpq.h, and rejects malformed input on the host
before any device work (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np

import paper_2001_06770_b300 as rpq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rpq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rpq_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["rpq_load_kg", "rpq_free_kg", "rpq_search", "rpq_search_batch", "rpq_trace", "rpq_strerror"]:
        assert f in names


def test_library_exports_every_declared_symbol():
    L = rpq.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) <= set(rpq.SYMBOLS) | {"rpq_last_error"}


def test_checked_library_exports_every_declared_symbol():
    """The bounds-checked build (device-side index checks compiled in) is the
    same boundary: it loads on the host and exports every declared call."""
    from paper_2001_06770_b300 import build as _build
    L = ctypes.CDLL(_build.build(checked=True))
    for name in declared_functions():
        assert hasattr(L, name), name


def test_strerror_names_codes():
    L = rpq.lib()
    assert L.rpq_strerror(0) == b"RPQ_OK"
    assert L.rpq_strerror(-1) == b"RPQ_EINVAL"
    assert L.rpq_strerror(-5) == b"RPQ_ELIMIT"


def _desc(n, row_ptr, col, label, kw_ptr, kw_nodes, n_labels=4, alpha=0.5, abar=3.0):
    keep = [np.ascontiguousarray(x) for x in (row_ptr, col, label, kw_ptr, kw_nodes)]
    p = [x.ctypes.data_as(ctypes.c_void_p) for x in keep]
    d = rpq.KGDesc(n, int(keep[0][-1]), p[0], p[1], p[2], n_labels, len(keep[3]) - 1, p[3], p[4], alpha, abar)
    return d, keep


def test_host_validation_rejects_before_device_work():
    L = rpq.lib()
    h = ctypes.c_void_p()
    rp = np.array([0, 1, 2], np.int64)
    col = np.array([1, 0], np.int32)
    lab = np.zeros(2, np.uint16)
    kp = np.array([0, 1], np.int64)
    kn = np.array([0], np.int32)
    bad = [
        dict(n=0),                                              # empty graph
        dict(row_ptr=np.array([0, 2, 1], np.int64)),            # decreasing row_ptr
        dict(alpha=1.5),                                        # alpha outside (0, 1)
        dict(abar=0.0),                                         # abar not positive
        dict(n_labels=0),                                       # no labels
        dict(n_labels=rpq.MAX_LABELS + 1),                      # above the limit
        dict(kw_nodes=np.array([7], np.int32)),                 # keyword node out of range
        dict(kw_ptr=np.array([1, 1], np.int64)),                # kw_ptr[0] != 0
    ]
    for case in bad:
        args = dict(n=2, row_ptr=rp, col=col, label=lab, kw_ptr=kp, kw_nodes=kn)
        args.update(case)
        d, keep = _desc(**args)
        rc = L.rpq_load_kg(ctypes.byref(d), ctypes.byref(h))
        assert rc in (rpq.RPQ_EINVAL, rpq.RPQ_ELIMIT), (case, rc)
        assert not h.value
        assert L.rpq_last_error()


def test_null_arguments_rejected():
    L = rpq.lib()
    assert L.rpq_load_kg(None, None) == rpq.RPQ_EINVAL
    assert L.rpq_search(None, None, None, None, None) == rpq.RPQ_EINVAL
    assert L.rpq_free_kg(None) == rpq.RPQ_OK
