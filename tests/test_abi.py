"""The C ABI without a GPU: the library builds and loads, exports every entry
point include/qegb.h declares, and its host-only logic (the plane-wave sphere of
Sec. 3.2.2 item (vi), argument checking) matches the oracle bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import qeinputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def q():
    from paper_2104_10502_gb300.build import build
    build()
    import paper_2104_10502_gb300 as q
    return q


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s+(qe_\w+)\s*\(", src, re.M))
    return names


def test_every_declared_symbol_is_exported(q):
    names = _declared()
    assert {"qe_hpsi", "qe_davidson", "qe_gsphere", "qe_ctx_create"} <= names
    lib = ctypes.CDLL(q.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert names == set(q.SYMBOLS)


@pytest.mark.parametrize("name", ["C0", "C1", "SMALL", "C3T"])
def test_gsphere_bit_exact_against_oracle(q, name):
    c = qeinputs.config(name)
    m, kin = q.gsphere(c["lat"], c["k"], c["ecut"], c["grid"])
    mo, ko, _ = oracle.gsphere(c["lat"], c["k"], c["ecut"])
    assert np.array_equal(m, mo)
    assert np.array_equal(kin, ko)


def test_gsphere_skewed_cell_and_k_points(q):
    lat = np.array([[7.0, 0.3, 0.0], [0.2, 8.0, 0.1], [0.0, -0.4, 9.0]])
    b = oracle.reciprocal(lat)
    for kf in ([0, 0, 0], [0.25, 0, 0], [0.5, 0.5, 0], [0.25, 0.75, 0.5]):
        k = np.array(kf) @ b
        m, kin = q.gsphere(lat, k, 15.0)
        mo, ko, _ = oracle.gsphere(lat, k, 15.0)
        assert np.array_equal(m, mo) and np.array_equal(kin, ko)


def test_gsphere_errors(q):
    lat = qeinputs.cubic(10.0)
    with pytest.raises(q.QEError) as e:
        q.gsphere(lat, [0, 0, 0], -1.0)
    assert e.value.code == q.QE_EINVAL
    with pytest.raises(q.QEError) as e:
        q.gsphere(lat, [0, 0, 0], 20.0, (14, 15, 15))
    assert e.value.code == q.QE_EINVAL
    with pytest.raises(q.QEError):
        q.gsphere(np.zeros((3, 3)), [0, 0, 0], 20.0)
    # capacity too small
    lib = q.lib()
    npw = ctypes.c_int(10)
    mil = (ctypes.c_int * 30)()
    latc = np.ascontiguousarray(lat, dtype=np.float64)
    k = np.zeros(3)
    rc = lib.qe_gsphere(latc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 20.0, None,
                        ctypes.byref(npw), mil, None)
    assert rc == q.QE_EINVAL


def test_null_arguments_are_rejected(q):
    lib = q.lib()
    assert lib.qe_hpsi(None, None, 0, None, None, None) == q.QE_EINVAL
    assert lib.qe_davidson(None, None, 0, 1e-8, 10, 0, None, None, None, None, None) == q.QE_EINVAL
    assert lib.qe_profile(None, 1) == q.QE_EINVAL
    assert len(lib.qe_last_error()) > 0


def test_context_without_gpu_fails_cleanly(q):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    with pytest.raises(q.QEError) as e:
        q.Context(0)
    assert e.value.code == q.QE_ECUDA


def test_problem_keeps_its_arrays_alive(q):
    """A problem descriptor holds raw pointers; the binding must keep the arrays
    it was built from alive for as long as the descriptor lives (temporaries
    passed straight into problem() included)."""
    import gc
    import weakref
    c = qeinputs.config("SMALL")
    v = np.zeros((c["grid"][2], c["grid"][1], c["grid"][0]))
    beta = np.zeros((2, 10, 2))
    d = np.eye(2)
    refs = [weakref.ref(a) for a in (v, beta, d)]
    pr = q.problem(c["lat"], c["k"], c["ecut"], c["grid"], v, beta, d, 1)
    del v, beta, d
    gc.collect()
    assert all(r() is not None for r in refs)
    assert pr.vloc_r == refs[0]().ctypes.data
    del pr
    gc.collect()
    assert all(r() is None for r in refs)
