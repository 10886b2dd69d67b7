"""Python binding of libqegb (plane-wave H|psi> and block Davidson on GB300).

Argument marshalling only: every step of the computation runs in the CUDA
library behind the C ABI declared in include/qegb.h.  Host arrays are NumPy
(complex128 or float64); device arrays are CUDA torch tensors (their
``data_ptr()`` is passed through, with the tensor's current stream unless one
is given).  There is no fallback: if the library is missing or fails to load,
importing the binding raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqegb.so")

QE_OK, QE_EINVAL, QE_ENOMEM, QE_ENOCONV, QE_EAGAIN, QE_PENDING, QE_ETIMEOUT, QE_ECUDA, \
    QE_ECANCELED = range(9)
QE_FP64, QE_MIXED = 0, 1
# flags or-ed into precision (k = 0): QE_GAMMA for hpsi (bands real in r, two per FFT),
# QE_NO_GAMMA for davidson (keep complex bands)
QE_GAMMA, QE_NO_GAMMA = 0x100, 0x200
# or-ed into QE_FP64 for hpsi: the FFT in float64 on the FP64 pipe (default: float-float pairs)
QE_FFT_FP64PIPE = 0x400
# or-ed into QE_MIXED for davidson: reduced eigenproblems of the mixed iterations in FP32
# (default: FP64 Rayleigh-Ritz)
QE_RR_FP32 = 0x800
# or-ed into precision for hpsi (device arrays): the operator is unchanged since the
# previous hpsi call on the context; its prepared forms are reused
QE_SAME_OPERATOR = 0x1000
QE_HOST, QE_DEVICE = 0, 1

SYMBOLS = ["qe_last_error", "qe_ctx_create", "qe_ctx_destroy", "qe_gsphere",
           "qe_vloc_gaussian", "qe_beta_gaussian", "qe_hpsi", "qe_davidson", "qe_profile",
           "qe_profile_read", "qe_hpsi_noalloc", "qe_serve_create", "qe_serve_submit",
           "qe_serve_poll", "qe_serve_cancel", "qe_serve_stats", "qe_serve_destroy",
           "qe_hpsi_batch", "qe_batch_create", "qe_batch_run", "qe_batch_destroy", "qe_autotune",
           "qe_davidson_batch", "qe_test_grid_wait", "qe_cg", "qe_density", "qe_hpsi_gen", "qe_scf_step"]
QE_SERVE_FAKE_SOLVER = 1


class QEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"QE error {code}: {msg}")
        self.code = code


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libqegb.so not built ({LIB_PATH}); run "
                          "`python -m paper_2104_10502_gb300.build`")
    return ctypes.CDLL(LIB_PATH)


_lib = _load()
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


class Projectors(ctypes.Structure):
    _fields_ = [("natom", ctypes.c_int), ("tau", _P), ("nrad", ctypes.c_int), ("l", _P),
                ("radial", _P)]


class Problem(ctypes.Structure):
    _fields_ = [("lat", ctypes.c_double * 9), ("k", ctypes.c_double * 3),
                ("ecutwfc", ctypes.c_double), ("grid", ctypes.c_int * 3),
                ("vloc_r", _P), ("nproj", ctypes.c_int), ("beta", _P), ("dmat", _P),
                ("nbnd", ctypes.c_int), ("mem", ctypes.c_int)]


_lib.qe_last_error.restype = ctypes.c_char_p
_lib.qe_ctx_create.argtypes = [ctypes.c_int, ctypes.POINTER(_P)]
_lib.qe_ctx_destroy.argtypes = [_P]
_lib.qe_ctx_destroy.restype = None
_lib.qe_gsphere.argtypes = [_D, _D, ctypes.c_double, _I, _I, _I, _D]
_lib.qe_vloc_gaussian.argtypes = [_P, _D, _I, ctypes.c_int, _D, ctypes.c_double, ctypes.c_double,
                                  _P, ctypes.c_int, _P]
_lib.qe_beta_gaussian.argtypes = [_P, _D, _D, ctypes.c_double, ctypes.c_int, _D, ctypes.c_int, _D,
                                  _P, ctypes.c_int, _P]
_lib.qe_profile.argtypes = [_P, ctypes.c_int]
_lib.qe_test_grid_wait.argtypes = [_P, ctypes.c_longlong]
_lib.qe_profile_read.argtypes = [_P, ctypes.c_int, ctypes.c_char_p, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_longlong), _D,
                                 ctypes.POINTER(ctypes.c_longlong)]
_lib.qe_serve_create.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.POINTER(_P)]
_lib.qe_serve_submit.argtypes = [_P, ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_double,
                                 ctypes.c_int, _P, ctypes.POINTER(ctypes.c_uint64)]
_lib.qe_serve_poll.argtypes = [_P, ctypes.c_uint64, ctypes.c_int, _P, _P, _P, _I,
                               ctypes.POINTER(ctypes.c_double)]
_lib.qe_serve_cancel.argtypes = [_P, ctypes.c_uint64]
_lib.qe_serve_stats.argtypes = [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                _I, _I, ctypes.POINTER(ctypes.c_size_t)]
_lib.qe_serve_destroy.argtypes = [_P]
_lib.qe_serve_destroy.restype = None
_lib.qe_hpsi_batch.argtypes = [_P, ctypes.c_int, ctypes.POINTER(Problem), ctypes.c_int,
                               ctypes.POINTER(_P), ctypes.POINTER(_P), _P]
_lib.qe_batch_create.argtypes = [_P, ctypes.c_int, ctypes.POINTER(Problem), ctypes.c_int,
                                 ctypes.POINTER(_P), ctypes.POINTER(_P), _P, ctypes.POINTER(_P)]
_lib.qe_batch_run.argtypes = [_P, _P]
_lib.qe_batch_destroy.argtypes = [_P]
_lib.qe_batch_destroy.restype = None
_lib.qe_autotune.argtypes = [_P, ctypes.POINTER(Problem), ctypes.c_int, _P]
_lib.qe_hpsi_noalloc.argtypes = [ctypes.POINTER(Problem), ctypes.c_int, _P, _P, _P]
_lib.qe_hpsi.argtypes = [_P, ctypes.POINTER(Problem), ctypes.c_int, _P, _P, _P]
_lib.qe_hpsi_gen.argtypes = [_P, ctypes.POINTER(Problem), ctypes.POINTER(Projectors), ctypes.c_int,
                             _P, _P, _P]
_lib.qe_davidson.argtypes = [_P, ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_double,
                             ctypes.c_int, ctypes.c_int, _P, _P, _P, _I, _P]
_lib.qe_density.argtypes = [_P, _D, ctypes.c_double, _I, ctypes.c_int, _D, _I, ctypes.POINTER(_P),
                            ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.c_int, _P]
_lib.qe_scf_step.argtypes = [_P, _D, ctypes.c_double, _I, ctypes.c_int, _D, _I, ctypes.POINTER(_P),
                             ctypes.POINTER(_P), _P, _P, ctypes.c_double, ctypes.c_int, _P, _P,
                             ctypes.c_int, _P]
_lib.qe_cg.argtypes = [_P, ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                       ctypes.c_int, _P, _P, _P, _I, _P]
_lib.qe_davidson_batch.argtypes = [_P, ctypes.c_int, ctypes.POINTER(Problem), ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P),
                                   ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _I, _P]


def lib() -> ctypes.CDLL:
    return _lib


def _check(rc: int, allow=()):
    if rc != QE_OK and rc not in allow:
        raise QEError(rc, _lib.qe_last_error().decode())
    return rc


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, mem flag) of a host NumPy array or a CUDA torch tensor."""
    if x is None:
        return None, QE_HOST
    if _is_torch(x):
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("device arrays must be contiguous CUDA tensors")
        return ctypes.c_void_p(x.data_ptr()), QE_DEVICE
    if not (isinstance(x, np.ndarray) and x.flags.c_contiguous
            and x.dtype in (np.float64, np.complex128)):
        raise ValueError("host arrays must be C-contiguous float64/complex128 NumPy arrays")
    return ctypes.c_void_p(x.ctypes.data), QE_HOST


def _stream(stream, *tensors):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    for t in tensors:
        if t is not None and _is_torch(t):
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    return ctypes.c_void_p(0)


def gsphere(lat, k, ecut: float, grid=None):
    """Plane-wave sphere: (miller int32 (npw, 3), kin float64 (npw,))."""
    lat = _f64(lat, 9)
    k = _f64(k, 3)
    g = None if grid is None else np.ascontiguousarray(grid, dtype=np.int32)
    npw = ctypes.c_int(0)
    gp = None if g is None else g.ctypes.data_as(_I)
    _check(_lib.qe_gsphere(_dptr(lat), _dptr(k), float(ecut), gp, ctypes.byref(npw), None, None))
    miller = np.zeros((npw.value, 3), dtype=np.int32)
    kin = np.zeros(npw.value, dtype=np.float64)
    _check(_lib.qe_gsphere(_dptr(lat), _dptr(k), float(ecut), gp, ctypes.byref(npw),
                           miller.ctypes.data_as(_I), _dptr(kin)))
    return miller, kin


def hpsi_noalloc(prob: "Problem", psi, hpsi, precision=QE_FP64, stream=None):
    """H|psi> through the entry point that allocates no device memory (its
    workspace is a fixed 64 MiB array inside the library).  All arrays must be
    CUDA tensors on the current device."""
    pp, mp = _ptr(psi)
    ph, mh = _ptr(hpsi)
    if prob.nbnd > 0 and (mp != QE_DEVICE or mh != QE_DEVICE):
        raise ValueError("qe_hpsi_noalloc takes device arrays only")
    _check(_lib.qe_hpsi_noalloc(ctypes.byref(prob), int(precision), pp, ph, _stream(stream, psi)))
    return hpsi


class Context:
    """One CUDA device, its plan cache and workspaces (qe_ctx)."""

    def __init__(self, device: int = 0):
        h = _P()
        _check(_lib.qe_ctx_create(int(device), ctypes.byref(h)))
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            _lib.qe_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- per-kernel timing ---------------------------------------------------
    def profile(self, enable: bool = True):
        _check(_lib.qe_profile(self._h, int(bool(enable))))

    def profile_read(self):
        """({kernel: (timed launches, total ms)}, kernels launched since reset)."""
        out = {}
        launches = ctypes.c_longlong(0)
        _check(_lib.qe_profile_read(self._h, -1, None, 0, None, None, ctypes.byref(launches)))
        i = 0
        while True:
            name = ctypes.create_string_buffer(64)
            calls = ctypes.c_longlong(0)
            ms = ctypes.c_double(0.0)
            rc = _lib.qe_profile_read(self._h, i, name, 64, ctypes.byref(calls), ctypes.byref(ms),
                                      None)
            if rc == QE_EINVAL:
                break
            _check(rc)
            out[name.value.decode()] = (calls.value, ms.value)
            i += 1
        return out, launches.value

    def test_grid_wait(self, wait_ns: int):
        """Test hook: make every grid barrier of later Davidson solves run out
        after wait_ns nanoseconds (0 restores normal barriers)."""
        _check(_lib.qe_test_grid_wait(self._h, int(wait_ns)))

    # ---- builders ---------------------------------------------------------
    def vloc_gaussian(self, lat, grid, tau, out, amp=-2.0, sigma=1.0, stream=None):
        lat = _f64(lat, 9)
        g = np.ascontiguousarray(grid, dtype=np.int32)
        tau = _f64(tau)
        p, mem = _ptr(out)
        _check(_lib.qe_vloc_gaussian(self._h, _dptr(lat), g.ctypes.data_as(_I), tau.size // 3,
                                     _dptr(tau), float(amp), float(sigma), p, mem,
                                     _stream(stream, out)))
        return out

    def beta_gaussian(self, lat, k, ecut, tau, widths, out, stream=None):
        lat = _f64(lat, 9)
        k = _f64(k, 3)
        tau = _f64(tau)
        w = _f64(widths)
        p, mem = _ptr(out)
        _check(_lib.qe_beta_gaussian(self._h, _dptr(lat), _dptr(k), float(ecut), tau.size // 3,
                                     _dptr(tau), w.size, _dptr(w), p, mem, _stream(stream, out)))
        return out

    # ---- operator and eigensolver -----------------------------------------
    @staticmethod
    def problem(lat, k, ecut, grid, vloc, beta, dmat, nbnd) -> Problem:
        pr = Problem()
        pr.lat[:] = [float(x) for x in _f64(lat, 9).ravel()]
        pr.k[:] = [float(x) for x in _f64(k, 3).ravel()]
        pr.ecutwfc = float(ecut)
        pr.grid[:] = [int(x) for x in grid]
        pv, mem = _ptr(vloc)
        pr.vloc_r = pv
        nproj = 0 if beta is None else int(beta.shape[0])
        pr.nproj = nproj
        if nproj:
            pb, mb = _ptr(beta)
            pd, md = _ptr(dmat)
            if mb != mem or md != mem:
                raise ValueError("vloc, beta and dmat must live in the same memory")
            pr.beta, pr.dmat = pb, pd
        pr.nbnd = int(nbnd)
        pr.mem = mem
        # the descriptor holds raw pointers: keep the arrays alive with it
        pr._keep = (vloc, beta, dmat)
        return pr

    @staticmethod
    def problem_gen(lat, k, ecut, grid, vloc, dmat, nproj, nbnd) -> Problem:
        """Problem descriptor for hpsi_gen: no stored beta, nproj projectors
        generated from their definition, D over them."""
        pr = Context.problem(lat, k, ecut, grid, vloc, None, None, nbnd)
        pd, md = _ptr(dmat)
        if nproj and md != pr.mem:
            raise ValueError("vloc and dmat must live in the same memory")
        pr.nproj = int(nproj)
        pr.dmat = pd if nproj else None
        pr._keep = (vloc, None, dmat)
        return pr

    def hpsi(self, prob: Problem, psi, hpsi, precision=QE_FP64, stream=None):
        pp, mp = _ptr(psi)
        ph, mh = _ptr(hpsi)
        if prob.nbnd > 0 and (mp != prob.mem or mh != prob.mem):
            raise ValueError("psi/hpsi must live where the problem's arrays live")
        _check(_lib.qe_hpsi(self._h, ctypes.byref(prob), int(precision), pp, ph,
                            _stream(stream, psi)))
        return hpsi

    def hpsi_gen(self, prob: Problem, tau, lrad, radial, psi, hpsi, precision=QE_FP64,
                 stream=None):
        """H|psi> with projectors generated on the fly from atom positions tau
        (natom, 3), angular momenta lrad (nrad,) and the radial table radial
        (nrad, npw) (host float64 or a CUDA tensor, where the problem lives);
        prob.beta is not read."""
        tau = _f64(tau)
        lr = np.ascontiguousarray(lrad, dtype=np.int32)
        pr_, mr = _ptr(radial)
        if lr.size and mr != prob.mem:
            raise ValueError("the radial table must live where the problem's arrays live")
        pj = Projectors(int(tau.size // 3), ctypes.c_void_p(tau.ctypes.data), int(lr.size),
                        ctypes.c_void_p(lr.ctypes.data), pr_)
        pp, mp = _ptr(psi)
        ph, mh = _ptr(hpsi)
        if prob.nbnd > 0 and (mp != prob.mem or mh != prob.mem):
            raise ValueError("psi/hpsi must live where the problem's arrays live")
        _check(_lib.qe_hpsi_gen(self._h, ctypes.byref(prob), ctypes.byref(pj), int(precision), pp, ph,
                                _stream(stream, psi)))
        return hpsi

    # ---- batches ------------------------------------------------------------------
    @staticmethod
    def _batch_args(probs, psis, hpsis):
        n = len(probs)
        arr = (Problem * n)(*probs)
        pp = (_P * n)(*[_ptr(x)[0] for x in psis])
        hp = (_P * n)(*[_ptr(x)[0] for x in hpsis])
        return n, arr, pp, hp

    def hpsi_batch(self, probs, psis, hpsis, precision=QE_FP64, stream=None):
        """H|psi> for a list of device-resident problems in one set of launches."""
        n, arr, pp, hp = self._batch_args(probs, psis, hpsis)
        _check(_lib.qe_hpsi_batch(self._h, n, arr, int(precision), pp, hp,
                                  _stream(stream, *psis)))
        return hpsis

    def batch_create(self, probs, psis, hpsis, precision=QE_FP64, stream=None):
        """Record the batch into a CUDA graph (see Batch)."""
        return Batch(self, probs, psis, hpsis, precision, stream)

    def autotune(self, prob: Problem, precision=QE_FP64, stream=None):
        _check(_lib.qe_autotune(self._h, ctypes.byref(prob), int(precision),
                                _stream(stream) if stream is not None else ctypes.c_void_p(0)))

    def davidson(self, prob: Problem, psi, evals, resid=None, precision=QE_FP64, tol=1e-8,
                 max_iter=100, max_dim=0, stream=None):
        """Returns (status, iters); status QE_OK or QE_ENOCONV."""
        pp, mp = _ptr(psi)
        pe, me = _ptr(evals)
        pr_, mr = _ptr(resid)
        if mp != prob.mem or me != prob.mem or (resid is not None and mr != prob.mem):
            raise ValueError("psi/evals/resid must live where the problem's arrays live")
        it = ctypes.c_int(0)
        rc = _check(_lib.qe_davidson(self._h, ctypes.byref(prob), int(precision), float(tol),
                                     int(max_iter), int(max_dim), pp, pe, pr_, ctypes.byref(it),
                                     _stream(stream, psi)), allow=(QE_ENOCONV,))
        return rc, it.value

    def cg(self, prob: Problem, psi, evals, resid=None, precision=QE_FP64, tol=1e-8,
           max_iter=100, max_sweeps=20, stream=None):
        """Band-by-band CG.  Returns (status, iters); status QE_OK or QE_ENOCONV."""
        pp, mp = _ptr(psi)
        pe, me = _ptr(evals)
        pr_, mr = _ptr(resid)
        if mp != prob.mem or me != prob.mem or (resid is not None and mr != prob.mem):
            raise ValueError("psi/evals/resid must live where the problem's arrays live")
        it = ctypes.c_int(0)
        rc = _check(_lib.qe_cg(self._h, ctypes.byref(prob), int(precision), float(tol), int(max_iter),
                               int(max_sweeps), pp, pe, pr_, ctypes.byref(it), _stream(stream, psi)),
                    allow=(QE_ENOCONV,))
        return rc, it.value

    def density(self, lat, ecut, grid, kpts, psis, weights, rho, precision=QE_FP64, stream=None):
        """rho = (1/Omega) sum_k sum_n w_nk |psi_nk(r)|^2 on the grid.  psis: per k
        point, host complex128 (nb, npw) arrays or CUDA tensors (nb, npw, 2);
        weights: per k point, host float64 (nb,); rho: host float64 or CUDA
        tensor (N3, N2, N1), where the bands live."""
        lat = _f64(lat, 9)
        g = np.ascontiguousarray(grid, dtype=np.int32)
        kp = _f64(kpts).reshape(-1, 3)
        nk = kp.shape[0]
        if len(psis) != nk or len(weights) != nk:
            raise ValueError("one band block and one weight vector per k point")
        nb = np.ascontiguousarray([int(p.shape[0]) for p in psis], dtype=np.int32)
        ws = [_f64(w) for w in weights]
        pr, mr = _ptr(rho)
        ptrs, mems = [], set()
        for p in psis:
            pp, mp = _ptr(p)
            ptrs.append(pp)
            mems.add(mp)
        if mems and mems != {mr}:
            raise ValueError("bands and rho must live in the same memory")
        parr = (_P * max(nk, 1))(*ptrs)
        warr = (_P * max(nk, 1))(*[ctypes.c_void_p(w.ctypes.data) for w in ws])
        _check(_lib.qe_density(self._h, _dptr(lat), float(ecut), g.ctypes.data_as(_I), nk,
                               _dptr(kp), nb.ctypes.data_as(_I), parr, warr, int(precision), pr, mr,
                               _stream(stream, rho)))
        return rho

    def scf_step(self, lat, ecut, grid, kpts, psis, weights, vext, vin, alpha, vnew, rho=None,
                 precision=QE_FP64, stream=None):
        """One self-consistency step: V_new = (1 - alpha) V_in + alpha (V_ext + V_H[rho] +
        v_x[rho]) with rho from the bands (arrays as density(); vext, vin, vnew, rho
        where the bands live)."""
        lat = _f64(lat, 9)
        g = np.ascontiguousarray(grid, dtype=np.int32)
        kp = _f64(kpts).reshape(-1, 3)
        nk = kp.shape[0]
        nb = np.ascontiguousarray([int(p.shape[0]) for p in psis], dtype=np.int32)
        ws = [_f64(w) for w in weights]
        ptrs, mems = [], set()
        for p in psis:
            pp, mp = _ptr(p)
            ptrs.append(pp)
            mems.add(mp)
        pe, me = _ptr(vext)
        pi_, mi = _ptr(vin)
        pn, mn = _ptr(vnew)
        pr_, mr = _ptr(rho)
        if len({me, mi, mn} | mems | ({mr} if rho is not None else set())) != 1:
            raise ValueError("bands, potentials and rho must live in the same memory")
        parr = (_P * max(nk, 1))(*ptrs)
        warr = (_P * max(nk, 1))(*[ctypes.c_void_p(w.ctypes.data) for w in ws])
        _check(_lib.qe_scf_step(self._h, _dptr(lat), float(ecut), g.ctypes.data_as(_I), nk, _dptr(kp),
                                nb.ctypes.data_as(_I), parr, warr, pe, pi_, float(alpha),
                                int(precision), pn, pr_, mn, _stream(stream, vnew)))
        return vnew

    def davidson_batch(self, probs, psis, evals, resids=None, precision=QE_FP64, tol=1e-8,
                       max_iter=100, max_dim=0, stream=None):
        """Lockstep Davidson over device-resident problems.  Returns (rc, status
        list, iters list); rc QE_OK, or QE_ENOCONV if some solve did not converge."""
        n = len(probs)
        arr = (Problem * n)(*probs)
        pp = (_P * n)(*[_ptr(x)[0] for x in psis])
        pe = (_P * n)(*[_ptr(x)[0] for x in evals])
        pr_ = (_P * n)(*[_ptr(x)[0] for x in resids]) if resids is not None else None
        its = (ctypes.c_int * max(n, 1))()
        sts = (ctypes.c_int * max(n, 1))()
        rc = _check(_lib.qe_davidson_batch(self._h, n, arr, int(precision), float(tol),
                                           int(max_iter), int(max_dim), pp, pe, pr_, its, sts,
                                           _stream(stream, *psis)), allow=(QE_ENOCONV,))
        return rc, list(sts)[:n], list(its)[:n]


class Batch:
    """A batched H|psi> captured in a CUDA graph (qe_batch_*).  Keeps references
    to the problems and arrays: replay with run() after updating psi in place."""

    def __init__(self, ctx, probs, psis, hpsis, precision, stream):
        self._keep = (list(probs), list(psis), list(hpsis))
        n, arr, pp, hp = Context._batch_args(probs, psis, hpsis)
        self._keep += (arr, pp, hp)
        h = _P()
        self._stream = _stream(stream, *psis)
        _check(_lib.qe_batch_create(ctx._h, n, arr, int(precision), pp, hp, self._stream,
                                    ctypes.byref(h)))
        self._h = h

    def run(self, stream=None):
        _check(_lib.qe_batch_run(self._h, self._stream if stream is None else _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            _lib.qe_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def problem(lat, k, ecut, grid, vloc, beta, dmat, nbnd) -> Problem:
    """Flat problem descriptor (see Context.problem)."""
    return Context.problem(lat, k, ecut, grid, vloc, beta, dmat, nbnd)


class Server:
    """Continuous-batching Davidson server (qe_serve_*).  Inputs are host
    arrays, copied at submit; results come back from poll()."""

    def __init__(self, device=0, budget_bytes=8 << 30, max_slots=4, max_queue=256, fake=False):
        h = _P()
        _check(_lib.qe_serve_create(int(device), int(budget_bytes), int(max_slots), int(max_queue),
                                    QE_SERVE_FAKE_SOLVER if fake else 0, ctypes.byref(h)))
        self._h = h
        self._shapes = {}

    def submit(self, prob: Problem, psi0: np.ndarray, precision=QE_FP64, tol=1e-8, max_iter=100):
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
        t = ctypes.c_uint64(0)
        rc = _lib.qe_serve_submit(self._h, ctypes.byref(prob), int(precision), float(tol),
                                  int(max_iter), ctypes.c_void_p(psi0.ctypes.data), ctypes.byref(t))
        if rc == QE_EAGAIN:
            return None
        _check(rc)
        self._shapes[t.value] = psi0.shape
        return t.value

    def poll(self, ticket, timeout_ms=-1):
        """None while pending; else a dict with status, psi, evals, resid, iters, latency_s."""
        if ticket not in self._shapes:
            _check(_lib.qe_serve_poll(self._h, ctypes.c_uint64(ticket), 0, None, None, None, None,
                                      None))
        nb, npw = self._shapes[ticket]
        psi = np.zeros((nb, npw), dtype=np.complex128)
        ev = np.zeros(nb)
        rs = np.zeros(nb)
        it = ctypes.c_int(0)
        lat = ctypes.c_double(0.0)
        rc = _lib.qe_serve_poll(self._h, ctypes.c_uint64(ticket), int(timeout_ms),
                                ctypes.c_void_p(psi.ctypes.data), ctypes.c_void_p(ev.ctypes.data),
                                ctypes.c_void_p(rs.ctypes.data), ctypes.byref(it), ctypes.byref(lat))
        if rc == QE_PENDING:
            return None
        if rc not in (QE_OK, QE_ENOCONV, QE_ECANCELED):
            _check(rc)
        del self._shapes[ticket]
        return dict(status=rc, psi=psi, evals=ev, resid=rs, iters=it.value, latency_s=lat.value)

    def cancel(self, ticket):
        _check(_lib.qe_serve_cancel(self._h, ctypes.c_uint64(ticket)))

    def stats(self):
        sub, comp = ctypes.c_longlong(0), ctypes.c_longlong(0)
        run, que = ctypes.c_int(0), ctypes.c_int(0)
        used = ctypes.c_size_t(0)
        _check(_lib.qe_serve_stats(self._h, ctypes.byref(sub), ctypes.byref(comp), ctypes.byref(run),
                                   ctypes.byref(que), ctypes.byref(used)))
        return dict(submitted=sub.value, completed=comp.value, running=run.value, queued=que.value,
                    bytes_in_use=used.value)

    def close(self):
        if getattr(self, "_h", None):
            _lib.qe_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
