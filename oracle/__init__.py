"""FP64 CPU oracle (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C99,
``double complex``, OpenMP over sites) through ctypes and shares no code
with the CUDA library.  All arrays are numpy complex128 in the canonical
layouts of the ``synth`` module:

  spinor  (Lt, Lz, Ly, Lx, 4, 3)       gauge  (Lt, Lz, Ly, Lx, 4, 3, 3)
  clover  (Lt, Lz, Ly, Lx, 12, 12)     index spin*3 + colour

Every function names the definition it implements in ``oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile oracle.c into liboracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=gnu99", "-O2", "-fcx-limited-range", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_L = C.c_long
_PREC = C.CFUNCTYPE(None, _P, _P, _P)

_SIGS = {
    "oracle_num_threads": (_I, []),
    "oracle_set_num_threads": (None, [_I]),
    "oracle_gamma": (None, [_I, _P]),
    "oracle_sigma": (None, [_I, _I, _P]),
    "oracle_hop": (None, [_P, _I, _P, _P, _P]),
    "oracle_hop_sites": (None, [_P, _I, _P, _P, _P, _L, _P]),
    "oracle_field_strength": (None, [_P, _P, _P]),
    "oracle_clover": (None, [_P, _P, _D, _D, _P]),
    "oracle_invert_site_matrices": (_I, [_L, _I, _P, _P]),
    "oracle_apply_site_matrices": (None, [_L, _P, _P, _P]),
    "oracle_gamma5": (None, [_L, _P, _P]),
    "oracle_wilson_clover": (None, [_P, _I, _P, _P, _D, _P, _P]),
    "oracle_wilson_clover_dag": (None, [_P, _I, _P, _P, _D, _P, _P]),
    "oracle_schur": (None, [_P, _I, _P, _P, _P, _D, _P, _P]),
    "oracle_schur_dag": (None, [_P, _I, _P, _P, _P, _D, _P, _P]),
    "oracle_true_residual": (_D, [_P, _I, _P, _P, _D, _P, _P]),
    "oracle_cgnr": (_I, [_P, _I, _P, _P, _D, _P, _P, _D, _I, _P, _P]),
    "oracle_eo_cg": (_I, [_P, _I, _P, _P, _P, _D, _P, _P, _D, _I, _P, _P]),
    "oracle_schur_cg_iters": (None, [_P, _I, _P, _P, _P, _D, _P, _P, _I]),
    "oracle_cgnr_iters": (None, [_P, _I, _P, _P, _D, _P, _P, _I]),
    "oracle_net_layer": (None, [_P, _I, _P, _I, _I, _P, _P, _P]),
    "oracle_net_layer_adj": (None, [_P, _I, _P, _I, _I, _P, _P, _P]),
    "oracle_net_layer_wgrad": (None, [_P, _I, _P, _I, _I, _P, _P, _P]),
    "oracle_fgcr": (_I, [_P, _I, _P, _P, _D, _P, _P, _D, _I, _I, _PREC, _P, _P, _P]),
    "oracle_sap": (None, [_P, _I, _P, _P, _D, _P, _I, _I, _P, _P]),
}


def _load(path):
    handle = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(handle, name)
        f.restype = res
        f.argtypes = args
    return handle


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _load(_LIB)
    return _lib


def use_library(path):
    """Swap in another build of oracle.c (used by the mutation tests, which
    compile deliberately broken copies to show that the pins catch them).
    Returns the previous handle; pass ``None`` to restore the default."""
    global _lib
    prev = _lib
    _lib = None if path is None else _load(path)
    return prev


def num_threads():
    """Threads of the oracle's OpenMP loops (the cores a timed run uses)."""
    return int(lib().oracle_num_threads())


def set_num_threads(n):
    """Run later OpenMP loops of the oracle on n threads (timing only)."""
    lib().oracle_set_num_threads(int(n))


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _dims(dims):
    return (C.c_int * 4)(*[int(v) for v in dims])


def dims_of(field):
    """dims (Lx, Ly, Lz, Lt) of a canonical spinor/gauge array."""
    lt, lz, ly, lx = field.shape[:4]
    return (lx, ly, lz, lt)


def gamma(mu):
    """DeGrand-Rossi gamma_mu (mu = 0..3: x, y, z, t; 4: gamma_5)."""
    g = np.zeros((4, 4), np.complex128)
    lib().oracle_gamma(mu, _p(g))
    return g


def sigma(mu, nu):
    s = np.zeros((4, 4), np.complex128)
    lib().oracle_sigma(mu, nu, _p(s))
    return s


def hop(U, psi, tanti=1):
    """H psi (Wilson hopping term), full lattice."""
    U, psi = _c(U), _c(psi)
    out = np.empty_like(psi)
    lib().oracle_hop(_dims(dims_of(U)), tanti, _p(U), _p(psi), _p(out))
    return out


def hop_sites(U, psi, sites, tanti=1):
    """(H psi)(x) at the canonical site indices ``sites``; shape (n, 4, 3)."""
    U, psi = _c(U), _c(psi)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), np.complex128)
    lib().oracle_hop_sites(_dims(dims_of(U)), tanti, _p(U), _p(psi), _p(sites), len(sites),
                           _p(out))
    return out


def field_strength(U):
    """Fhat_{mu nu}(x), shape (..., 6, 3, 3), planes xy, xz, xt, yz, yt, zt."""
    U = _c(U)
    F = np.empty(U.shape[:4] + (6, 3, 3), np.complex128)
    lib().oracle_field_strength(_dims(dims_of(U)), _p(U), _p(F))
    return F


def clover(U, kappa, csw):
    """Per-site 12x12 clover matrix A(x)."""
    U = _c(U)
    A = np.empty(U.shape[:4] + (12, 12), np.complex128)
    lib().oracle_clover(_dims(dims_of(U)), _p(U), kappa, csw, _p(A))
    return A


def invert_site_matrices(A):
    """Per-site inverse by Gauss-Jordan with partial pivoting; (Ainv, n_singular)."""
    A = _c(A)
    n = A.shape[-1]
    nsites = A.size // (n * n)
    out = np.empty_like(A)
    bad = lib().oracle_invert_site_matrices(nsites, n, _p(A), _p(out))
    return out, bad


def apply_site_matrices(A, psi):
    A, psi = _c(A), _c(psi)
    out = np.empty_like(psi)
    lib().oracle_apply_site_matrices(psi.size // 12, _p(A), _p(psi), _p(out))
    return out


def gamma5(psi):
    psi = _c(psi)
    out = np.empty_like(psi)
    lib().oracle_gamma5(psi.size // 12, _p(psi), _p(out))
    return out


def _Aptr(A):
    return None if A is None else _p(A)


def wilson_clover(U, A, kappa, psi, tanti=1, dag=False):
    """M psi = A psi - kappa H psi (A None: A = 1); dag: M^dag psi."""
    U, psi = _c(U), _c(psi)
    A = None if A is None else _c(A)
    out = np.empty_like(psi)
    f = lib().oracle_wilson_clover_dag if dag else lib().oracle_wilson_clover
    f(_dims(dims_of(U)), tanti, _p(U), _Aptr(A), kappa, _p(psi), _p(out))
    return out


def schur(U, A, Ainv, kappa, psi, tanti=1, dag=False):
    """Odd-site Schur complement Mhat (full-lattice arrays, even sites zero)."""
    U, psi = _c(U), _c(psi)
    A = None if A is None else _c(A)
    Ainv = None if Ainv is None else _c(Ainv)
    out = np.empty_like(psi)
    f = lib().oracle_schur_dag if dag else lib().oracle_schur
    f(_dims(dims_of(U)), tanti, _p(U), _Aptr(A), _Aptr(Ainv), kappa, _p(psi), _p(out))
    return out


def true_residual(U, A, kappa, b, x, tanti=1):
    U, b, x = _c(U), _c(b), _c(x)
    A = None if A is None else _c(A)
    return lib().oracle_true_residual(_dims(dims_of(U)), tanti, _p(U), _Aptr(A), kappa, _p(b),
                                      _p(x))


def cgnr(U, A, kappa, b, tol=1e-10, maxiter=100000, tanti=1):
    """CG on M^dag M over the full lattice; returns (x, iters, true_res, ok)."""
    U, b = _c(U), _c(b)
    A = None if A is None else _c(A)
    x = np.empty_like(b)
    it, res = C.c_int(0), C.c_double(0)
    st = lib().oracle_cgnr(_dims(dims_of(U)), tanti, _p(U), _Aptr(A), kappa, _p(b), _p(x), tol,
                           maxiter, C.byref(it), C.byref(res))
    return x, it.value, res.value, st == 0


def eo_cg(U, A, Ainv, kappa, b, tol=1e-10, maxiter=100000, tanti=1):
    """Even-odd preconditioned CG-NE solve; returns (x, iters, true_res, ok)."""
    U, b = _c(U), _c(b)
    A = None if A is None else _c(A)
    Ainv = None if Ainv is None else _c(Ainv)
    x = np.empty_like(b)
    it, res = C.c_int(0), C.c_double(0)
    st = lib().oracle_eo_cg(_dims(dims_of(U)), tanti, _p(U), _Aptr(A), _Aptr(Ainv), kappa, _p(b),
                            _p(x), tol, maxiter, C.byref(it), C.byref(res))
    return x, it.value, res.value, st == 0


def schur_cg_iters(U, A, Ainv, kappa, bhat, niter, tanti=1):
    U, bhat = _c(U), _c(bhat)
    A = None if A is None else _c(A)
    Ainv = None if Ainv is None else _c(Ainv)
    x = np.empty_like(bhat)
    lib().oracle_schur_cg_iters(_dims(dims_of(U)), tanti, _p(U), _Aptr(A), _Aptr(Ainv), kappa,
                                _p(bhat), _p(x), niter)
    return x


def cgnr_iters(U, A, kappa, b, niter, tanti=1):
    U, b = _c(U), _c(b)
    A = None if A is None else _c(A)
    x = np.empty_like(b)
    lib().oracle_cgnr_iters(_dims(dims_of(U)), tanti, _p(U), _Aptr(A), kappa, _p(b), _p(x), niter)
    return x


def net_layer(U, W, psi, tanti=1):
    """Parallel-transport convolution; psi (..., cin, 4, 3), W (9, 4cout, 4cin)."""
    U, W, psi = _c(U), _c(W), _c(psi)
    cin = W.shape[2] // 4
    cout = W.shape[1] // 4
    assert psi.shape[4] == cin
    out = np.empty(psi.shape[:4] + (cout, 4, 3), np.complex128)
    lib().oracle_net_layer(_dims(dims_of(U)), tanti, _p(U), cin, cout, _p(W), _p(psi), _p(out))
    return out


def net_layer_adj(U, W, g, tanti=1):
    """Adjoint of net_layer applied to g (..., cout, 4, 3)."""
    U, W, g = _c(U), _c(W), _c(g)
    cin = W.shape[2] // 4
    cout = W.shape[1] // 4
    out = np.empty(g.shape[:4] + (cin, 4, 3), np.complex128)
    lib().oracle_net_layer_adj(_dims(dims_of(U)), tanti, _p(U), cin, cout, _p(W), _p(g), _p(out))
    return out


def net_layer_wgrad(U, psi, g, cout, tanti=1):
    """dL/dRe W + i dL/dIm W for the layer input psi and output gradient g."""
    U, psi, g = _c(U), _c(psi), _c(g)
    cin = psi.shape[4]
    gW = np.empty((9, 4 * cout, 4 * cin), np.complex128)
    lib().oracle_net_layer_wgrad(_dims(dims_of(U)), tanti, _p(U), cin, cout, _p(psi), _p(g),
                                 _p(gW))
    return gW


def sap(U, A, kappa, r, block, ncycle=1, nmr=4, tanti=1):
    """Schwarz alternating procedure (block MR with Dirichlet boundaries,
    checkerboard-coloured blocks): z ~ M^{-1} r."""
    U, r = _c(U), _c(r)
    A = None if A is None else _c(A)
    z = np.empty_like(r)
    bs = (C.c_int * 4)(*[int(v) for v in block])
    lib().oracle_sap(_dims(dims_of(U)), tanti, _p(U), _Aptr(A), kappa, bs, ncycle, nmr, _p(r), _p(z))
    return z


def fgcr(U, A, kappa, b, tol=1e-10, nkrylov=20, maxiter=100000, prec=None, tanti=1):
    """Flexible GCR(nkrylov) on M with right preconditioner ``prec(r) -> z``
    (numpy callable, None = identity); returns (x, iters, true_res, ok)."""
    U, b = _c(U), _c(b)
    A = None if A is None else _c(A)
    x = np.empty_like(b)
    it, res = C.c_int(0), C.c_double(0)
    shape = b.shape
    n = b.size

    def _cb(_ctx, rp, zp):
        r = np.ctypeslib.as_array(C.cast(rp, C.POINTER(C.c_double)), shape=(2 * n,))
        z = np.ctypeslib.as_array(C.cast(zp, C.POINTER(C.c_double)), shape=(2 * n,))
        rr = r.view(np.complex128).reshape(shape).copy()
        z.view(np.complex128)[:] = np.ascontiguousarray(prec(rr), np.complex128).reshape(-1)

    cb = _PREC(_cb) if prec is not None else C.cast(None, _PREC)
    st = lib().oracle_fgcr(_dims(dims_of(U)), tanti, _p(U), _Aptr(A), kappa, _p(b), _p(x), tol,
                           nkrylov, maxiter, cb, None, C.byref(it), C.byref(res))
    return x, it.value, res.value, st == 0


def fgmres_dr(U, A, kappa, b, tol=1e-10, m=20, k=0, maxiter=100000, prec=None, tanti=1, history=None,
              on_restart=None):
    """Flexible GMRES(m) with k deflated vectors at restarts on M (Sec. 7;
    oracle/fgmresdr.py).  prec(r) -> z on canonical arrays (None: identity).
    Returns (x, iterations, true relative residual, converged)."""
    from . import fgmresdr
    U = _c(U)
    A = None if A is None else _c(A)
    shape = b.shape

    def matvec(v):
        return wilson_clover(U, A, kappa, v.reshape(shape), tanti=tanti).reshape(-1)

    p = None if prec is None else (lambda v: np.asarray(prec(v.reshape(shape)), dtype=complex).reshape(-1))
    x, it, res, ok = fgmresdr.fgmres_dr(matvec, b, tol, m, k, maxiter, p, history, on_restart)
    return x.reshape(shape), it, res, ok
