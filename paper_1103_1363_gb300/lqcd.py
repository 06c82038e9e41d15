"""Thin Python binding of the C ABI in include/lqcd.h.

Argument marshalling only: every computation runs in liblqcd.so's CUDA
kernels.  PyTorch provides device memory (the workspace and the vectors)
and streams.  The functions keep the C names; ``Lattice`` is a small
convenience owner of one context and its workspace tensor.

If liblqcd.so has not been built this module raises on import: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# LQCD_LIB selects another build of the same library (kernel experiments)
LIB_PATH = os.environ.get("LQCD_LIB") or os.path.join(_HERE, "liblqcd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("liblqcd.so is not built: run __graft_entry__.build() (nvcc, sm_103a)")

_lib = C.CDLL(LIB_PATH)

LQCD_OK = 0
STATUS = {0: "OK", 1: "ERR_INVALID", 2: "ERR_CUDA", 3: "ERR_NOMEM", 4: "ERR_STATE",
          5: "ERR_NOT_CONVERGED", 6: "ERR_BREAKDOWN", 7: "ERR_TIMEOUT", 8: "ERR_CLOVER_SINGULAR"}
F64, F32, F16, BF16, F16_LINKS, BF16_LINKS = range(6)
F16_SPINORS, BF16_SPINORS = 7, 8  # 6 is not used
PREC = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16, "f16links": F16_LINKS,
        "bf16links": BF16_LINKS, "f16spinors": F16_SPINORS, "bf16spinors": BF16_SPINORS}
PREC_NAMES = ("f64", "f32", "f16", "bf16", "f16links", "bf16links", None, "f16spinors", "bf16spinors")  # by value
# storage precision of links / clover for each mode (the bit it needs in prec_mask)
_STORAGE = {F64: F64, F32: F32, F16: F16, BF16: BF16, F16_LINKS: F16, BF16_LINKS: BF16,
            F16_SPINORS: F32, BF16_SPINORS: F32}
OP_HOP, OP_SCHUR, OP_FULL, DAG = 0, 1, 2, 1 << 8
SOLVER_CG_EO, SOLVER_CG_FULL, SOLVER_FGCR, SOLVER_FGMRES_DR = 0, 1, 2, 3


class lqcd_config(C.Structure):
    _fields_ = [("dims", C.c_int * 4), ("t_antiperiodic", C.c_int), ("recon", C.c_int),
                ("prec_mask", C.c_int), ("max_nrhs", C.c_int), ("gcr_nkrylov", C.c_int),
                ("part", C.c_int * 4), ("coord", C.c_int * 4)]


class lqcd_solver_params(C.Structure):
    _fields_ = [("solver", C.c_int), ("inner_prec", C.c_int), ("maxiter", C.c_int),
                ("reliable_interval", C.c_int), ("reliable_delta", C.c_double),
                ("check_interval", C.c_int), ("nkrylov", C.c_int), ("use_graph", C.c_int),
                ("residual_prec", C.c_int), ("ndefl", C.c_int), ("persistent", C.c_int),
                ("persistent_wait_us", C.c_int)]


class lqcd_solver_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("reliable_updates", C.c_int), ("restarts", C.c_int),
                ("dslash_count", C.c_long), ("kernel_launches", C.c_long),
                ("true_residual", C.c_double), ("seconds", C.c_double),
                ("preconditioner_fallback", C.c_int), ("precision_fallback", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lqcd_profile_entry(C.Structure):
    _fields_ = [("launches", C.c_long), ("ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


_P, _I, _D, _S = C.c_void_p, C.c_int, C.c_double, C.c_size_t
_SIGS = {
    "lqcd_create": [C.POINTER(lqcd_config), _P, C.POINTER(_P)],
    "lqcd_destroy": [_P],
    "lqcd_set_stream": [_P, _P],
    "lqcd_workspace_size": [_P, C.POINTER(_S)],
    "lqcd_set_workspace": [_P, _P, _S],
    "lqcd_field_bytes": [_P, _I, C.POINTER(_S)],
    "lqcd_gauge_load": [_P, _P],
    "lqcd_clover_compute": [_P, _D, _D],
    "lqcd_pack": [_P, _P, _P, _I, _I, _I],
    "lqcd_unpack": [_P, _P, _P, _I, _I, _I],
    "lqcd_dslash": [_P, _P, _P, _I, _D, _D, _I, _I, _I],
    "lqcd_clover_apply": [_P, _P, _P, _I, _I, _I, _I],
    "lqcd_solver_params_default": [C.POINTER(lqcd_solver_params)],
    "lqcd_solve": [_P, _P, _P, _D, _I, C.POINTER(lqcd_solver_params), C.POINTER(lqcd_solver_stats)],
    "lqcd_sync": [_P],
    "lqcd_profile_enable": [_P, _I],
    "lqcd_profile_read": [_P, C.POINTER(lqcd_profile_entry)],
    "lqcd_dslash_schur_static": [_P, _P, _P, _D, _D, _I, _I, _I],
    "lqcd_set_preconditioner": [_P, _P],
    "lqcd_training_pair": [_P, _P, _P, _P, _P, _I],
    "lqcd_halo_layout": [_P, _I, C.POINTER(_S), C.POINTER(_S), C.POINTER(_S)],
    "lqcd_halo_pack": [_P, _P, _P, _I, _I, _I, _I],
    "lqcd_halo_dslash": [_P, _P, _P, _P, _I, _I, _I, _P, _D, _I, _I, _I],
    "lqcd_norm2": [_P, _P, _I, _I, _I, C.POINTER(_D)],
    "lqcd_set_preconditioner_sap": [_P, _P, _I, _I],
    "lqcd_harmonic_ritz": [_I, _P, _I, _I, _P, _P],
    "lqcd_sap_apply": [_P, _P, _P, _P, _I, _I],
    "lqcd_tune": [_P, _I, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "lqcd_tune_set": [_P, _I, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "lqcd_fma_peak": [_I, _I, C.POINTER(C.c_double)],
    "lqcd_net_set_wait": [_P, C.c_ulonglong, _I],
    "lqcd_solve_batch": [C.POINTER(_P), _I, C.POINTER(_P), C.POINTER(_P), C.POINTER(_D),
                         C.POINTER(lqcd_solver_params), C.POINTER(lqcd_solver_stats)],
    "lqcd_net_create": [_P, _I, _P, _I, _I, C.POINTER(_P)],
    "lqcd_net_destroy": [_P],
    "lqcd_net_workspace_size": [_P, C.POINTER(_S)],
    "lqcd_net_set_workspace": [_P, _P, _S],
    "lqcd_net_num_weights": [_P, C.POINTER(_S)],
    "lqcd_net_set_max_ctas": [_P, _I],
    "lqcd_net_bind": [_P, _P],
    "lqcd_net_profile_enable": [_P, _I],
    "lqcd_net_profile_read": [_P, C.POINTER(lqcd_profile_entry), _I],
    "lqcd_net_set_weights": [_P, _P],
    "lqcd_net_get_weights": [_P, _P, _P],
    "lqcd_net_layer_apply": [_P, _I, _I, _P, _P, _I],
    "lqcd_net_layer_wgrad": [_P, _I, _P, _P, _I, _I],
    "lqcd_net_forward": [_P, _P, _P, _I],
    "lqcd_net_train_step": [_P, _P, _P, _I, _D, _D, _D, _D, C.POINTER(_D)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.lqcd_last_error.restype = C.c_char_p
_lib.lqcd_last_error.argtypes = []

EXPORTED = list(_SIGS) + ["lqcd_last_error"]


class LqcdError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.lqcd_last_error().decode()
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status), msg))


def _check(st, where):
    if st != LQCD_OK:
        raise LqcdError(st, where)
    return st


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (no copy)."""
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(x.ctypes.data)
    if isinstance(x, int):
        return C.c_void_p(x)
    raise TypeError(type(x))


def _stream_handle(stream):
    if stream is None:
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------ C-name wrappers

def lqcd_last_error():
    return _lib.lqcd_last_error().decode()


def lqcd_create(dims, t_antiperiodic=1, recon=12, precisions=("f64", "f32", "f16", "bf16"),
                max_nrhs=1, gcr_nkrylov=0, stream=None, part=(1, 1, 1, 1), coord=(0, 0, 0, 0)):
    cfg = lqcd_config()
    for i in range(4):
        cfg.part[i] = int(part[i])
        cfg.coord[i] = int(coord[i])
    for i, d in enumerate(dims):
        cfg.dims[i] = int(d)
    cfg.t_antiperiodic = int(t_antiperiodic)
    cfg.recon = int(recon)
    cfg.prec_mask = 0
    for p in precisions:
        cfg.prec_mask |= 1 << _STORAGE[PREC[p]]
    cfg.max_nrhs = int(max_nrhs)
    cfg.gcr_nkrylov = int(gcr_nkrylov)
    ctx = C.c_void_p()
    _check(_lib.lqcd_create(C.byref(cfg), _stream_handle(stream), C.byref(ctx)), "lqcd_create")
    return ctx


def lqcd_destroy(ctx):
    _check(_lib.lqcd_destroy(ctx), "lqcd_destroy")


def lqcd_set_stream(ctx, stream):
    _check(_lib.lqcd_set_stream(ctx, _stream_handle(stream)), "lqcd_set_stream")


def lqcd_workspace_size(ctx):
    n = C.c_size_t()
    _check(_lib.lqcd_workspace_size(ctx, C.byref(n)), "lqcd_workspace_size")
    return n.value


def lqcd_set_workspace(ctx, ws):
    _check(_lib.lqcd_set_workspace(ctx, _ptr(ws), ws.numel() * ws.element_size()),
           "lqcd_set_workspace")


def lqcd_field_bytes(ctx, prec):
    n = C.c_size_t()
    _check(_lib.lqcd_field_bytes(ctx, PREC.get(prec, prec), C.byref(n)), "lqcd_field_bytes")
    return n.value


def lqcd_gauge_load(ctx, links):
    _check(_lib.lqcd_gauge_load(ctx, _ptr(links)), "lqcd_gauge_load")


def lqcd_clover_compute(ctx, kappa, csw):
    _check(_lib.lqcd_clover_compute(ctx, float(kappa), float(csw)), "lqcd_clover_compute")


def lqcd_pack(ctx, internal, canonical, parity, prec, nrhs=1):
    _check(_lib.lqcd_pack(ctx, _ptr(internal), _ptr(canonical), int(parity), PREC.get(prec, prec),
                          int(nrhs)), "lqcd_pack")


def lqcd_unpack(ctx, canonical, internal, parity, prec, nrhs=1):
    _check(_lib.lqcd_unpack(ctx, _ptr(canonical), _ptr(internal), int(parity), PREC.get(prec, prec),
                            int(nrhs)), "lqcd_unpack")


def lqcd_dslash(ctx, out, inp, parity, kappa, csw, op_flags, prec, nrhs=1):
    _check(_lib.lqcd_dslash(ctx, _ptr(out), _ptr(inp), int(parity), float(kappa), float(csw),
                            int(op_flags), PREC.get(prec, prec), int(nrhs)), "lqcd_dslash")


def lqcd_dslash_schur_static(ctx, out, inp, kappa, csw, dag, prec, nrhs=1):
    """Schur operator with its intermediate in the library's fixed device
    array (no workspace scratch); see include/lqcd.h."""
    _check(_lib.lqcd_dslash_schur_static(ctx, _ptr(out), _ptr(inp), float(kappa), float(csw),
                                         int(bool(dag)), PREC.get(prec, prec), int(nrhs)),
           "lqcd_dslash_schur_static")


def lqcd_training_pair(ctx, r, e, xstar, x=None, nrhs=1):
    """e = x* - x, r = M e as canonical FP32 complex spinors (device)."""
    _check(_lib.lqcd_training_pair(ctx, _ptr(r), _ptr(e), _ptr(xstar), _ptr(x) if x is not None else None,
                                   int(nrhs)), "lqcd_training_pair")


def lqcd_halo_layout(ctx, prec):
    """(offsets[8], lengths[8], total) of a face buffer set, segment 2 mu + side."""
    off, ln, tot = (C.c_size_t * 8)(), (C.c_size_t * 8)(), C.c_size_t()
    _check(_lib.lqcd_halo_layout(ctx, PREC.get(prec, prec), off, ln, C.byref(tot)), "lqcd_halo_layout")
    return list(off), list(ln), tot.value


def lqcd_halo_pack(ctx, send, inp, parity, dag, prec, nrhs=1):
    _check(_lib.lqcd_halo_pack(ctx, _ptr(send), _ptr(inp), int(parity), int(bool(dag)), PREC.get(prec, prec),
                               int(nrhs)), "lqcd_halo_pack")


def lqcd_halo_dslash(ctx, out, inp, recv, parity, dag=False, epi=0, y=None, a=1.0, stage=0, prec="f32", nrhs=1):
    _check(_lib.lqcd_halo_dslash(ctx, _ptr(out), _ptr(inp), _ptr(recv) if recv is not None else None, int(parity),
                                 int(bool(dag)), int(epi), _ptr(y) if y is not None else None, float(a), int(stage),
                                 PREC.get(prec, prec), int(nrhs)), "lqcd_halo_dslash")


def lqcd_norm2(ctx, field, parity, prec, nrhs=1):
    out = (C.c_double * nrhs)()
    _check(_lib.lqcd_norm2(ctx, _ptr(field), int(parity), PREC.get(prec, prec), int(nrhs), out), "lqcd_norm2")
    return list(out)


def lqcd_clover_apply(ctx, out, inp, parity, inverse, prec, nrhs=1):
    _check(_lib.lqcd_clover_apply(ctx, _ptr(out), _ptr(inp), int(parity), int(inverse),
                                  PREC.get(prec, prec), int(nrhs)), "lqcd_clover_apply")


def lqcd_solver_params_default():
    p = lqcd_solver_params()
    _check(_lib.lqcd_solver_params_default(C.byref(p)), "lqcd_solver_params_default")
    return p


def lqcd_solve(ctx, x, b, tol, nrhs=1, params=None, raise_on_error=True):
    """Returns (status, stats dict)."""
    if params is None:
        params = lqcd_solver_params_default()
    st = lqcd_solver_stats()
    rc = _lib.lqcd_solve(ctx, _ptr(x), _ptr(b), float(tol), int(nrhs), C.byref(params), C.byref(st))
    if raise_on_error:
        _check(rc, "lqcd_solve")
    return rc, st.as_dict()


def lqcd_sync(ctx):
    _check(_lib.lqcd_sync(ctx), "lqcd_sync")


def lqcd_solve_batch(ctxs, xs, bs, tols, params=None, raise_on_error=True):
    """Solve several lattices together; returns (status, [stats dict])."""
    n = len(ctxs)
    if params is None:
        params = lqcd_solver_params_default()
    carr = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    xarr = (C.c_void_p * n)(*[_ptr(x).value for x in xs])
    barr = (C.c_void_p * n)(*[_ptr(b).value for b in bs])
    tarr = (C.c_double * n)(*[float(t) for t in tols])
    st = (lqcd_solver_stats * n)()
    rc = _lib.lqcd_solve_batch(carr, n, xarr, barr, tarr, C.byref(params), st)
    if raise_on_error:
        _check(rc, "lqcd_solve_batch")
    return rc, [s.as_dict() for s in st]


def lqcd_harmonic_ritz(hbar, nz, k):
    """Harmonic Ritz pairs of FGMRES-DR's deflation step (host, no GPU):
    hbar complex (nz + 1, nz); returns (theta[k], g[nz, k])."""
    # column-major storage = the C-contiguous transpose
    ht = np.ascontiguousarray(np.asarray(hbar, dtype=np.complex128)[:nz + 1, :nz].T)
    theta = np.zeros(k, dtype=np.complex128)
    gt = np.zeros((k, nz), dtype=np.complex128)
    _check(_lib.lqcd_harmonic_ritz(int(nz), _ptr(ht), int(nz + 1), int(k), _ptr(theta), _ptr(gt)),
           "lqcd_harmonic_ritz")
    return theta, gt.T


def _block4(block):
    if block is None:
        return None
    if len(block) != 4:
        raise ValueError("block needs four extents")
    return C.cast((C.c_int * 4)(*[int(b) for b in block]), C.c_void_p)


def lqcd_set_preconditioner_sap(ctx, block, ncycle=1, nmr=4):
    """SAP as the FGCR right preconditioner (block=None switches it off)."""
    _check(_lib.lqcd_set_preconditioner_sap(ctx, _block4(block), int(ncycle), int(nmr)),
           "lqcd_set_preconditioner_sap")


def lqcd_sap_apply(ctx, z, r, block, ncycle=1, nmr=4):
    """z = SAP(r) on internal FP32 full fields (device)."""
    _check(_lib.lqcd_sap_apply(ctx, _ptr(z), _ptr(r), _block4(block), int(ncycle), int(nmr)),
           "lqcd_sap_apply")


def lqcd_tune(ctx, prec):
    """Autotune the hopping kernels; returns {"block": (plain, plain reducing,
    dagger, dagger reducing), "sites_per_thread": (plain reducing, dagger
    reducing)} (0 sites per thread: one wave of resident blocks)."""
    best = (C.c_int * 4)()
    sites = (C.c_int * 2)()
    _check(_lib.lqcd_tune(ctx, PREC.get(prec, prec), best, sites), "lqcd_tune")
    return {"block": tuple(best), "sites_per_thread": tuple(sites)}


def lqcd_fma_peak(device, kind):
    """Measured multiply-add peak of a GPU in TFLOP/s: kind 0 FP32, 1 FP32
    packed pairs, 2 FP64."""
    out = C.c_double(0.0)
    _check(_lib.lqcd_fma_peak(int(device), int(kind), C.byref(out)), "lqcd_fma_peak")
    return out.value


BLOCK_STAGED = 1  # LQCD_BLOCK_STAGED: the shared-memory staged kernel for a plain class


def lqcd_tune_set(ctx, prec, block, sites=None):
    """Set the tuner's choices directly: block = (plain, plain reducing,
    dagger, dagger reducing), each 32, 64, 96 or 128, or BLOCK_STAGED for the
    plain ones; sites = (plain reducing, dagger reducing) or None."""
    b = (C.c_int * 4)(*[int(v) for v in block])
    s = (C.c_int * 2)(*[int(v) for v in sites]) if sites is not None else None
    _check(_lib.lqcd_tune_set(ctx, PREC.get(prec, prec), b, s), "lqcd_tune_set")


def lqcd_profile_enable(ctx, enable=True):
    _check(_lib.lqcd_profile_enable(ctx, int(bool(enable))), "lqcd_profile_enable")


def lqcd_profile_read(ctx):
    """{prec name: {launches, ms, bytes, flops}} since the last read."""
    arr = (lqcd_profile_entry * len(PREC_NAMES))()
    _check(_lib.lqcd_profile_read(ctx, arr), "lqcd_profile_read")
    return {PREC_NAMES[i]: {k: getattr(arr[i], k) for k, _ in lqcd_profile_entry._fields_}
            for i in range(len(PREC_NAMES)) if PREC_NAMES[i]}


def solver_params(**kw):
    p = lqcd_solver_params_default()
    for k, v in kw.items():
        if k in ("inner_prec", "residual_prec"):
            v = PREC.get(v, v)
        setattr(p, k, v)
    return p


class Net:
    """A parallel-transport convolution network bound to a Lattice (thin
    owner of an lqcd_net handle and its workspace tensor)."""

    def __init__(self, lat, channels=(1, 12, 12, 1), bf16=True, max_batch=1):
        self.lat = lat
        self.bound = lat
        self.channels = tuple(int(c) for c in channels)
        arr = (C.c_int * len(self.channels))(*self.channels)
        h = C.c_void_p()
        _check(_lib.lqcd_net_create(lat.ctx, len(self.channels) - 1, arr, int(bool(bf16)),
                                    int(max_batch), C.byref(h)), "lqcd_net_create")
        self.h = h
        n = C.c_size_t()
        _check(_lib.lqcd_net_workspace_size(h, C.byref(n)), "lqcd_net_workspace_size")
        self.workspace = torch.empty(n.value + 256, dtype=torch.uint8, device=lat.device)
        off = (-self.workspace.data_ptr()) % 256
        _check(_lib.lqcd_net_set_workspace(h, C.c_void_p(self.workspace.data_ptr() + off), n.value),
               "lqcd_net_set_workspace")
        _check(_lib.lqcd_net_num_weights(h, C.byref(n)), "lqcd_net_num_weights")
        self.num_weights = n.value

    def close(self):
        if self.h is not None:
            _lib.lqcd_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bind(self, lat):
        """Transport with lat's links from now on (same lattice as the network's)."""
        _check(_lib.lqcd_net_bind(self.h, lat.ctx), "lqcd_net_bind")
        self.bound = lat

    def set_max_ctas(self, max_ctas):
        """Cap the CTAs of the persistent BF16 launches (0: one per SM)."""
        _check(_lib.lqcd_net_set_max_ctas(self.h, int(max_ctas)), "lqcd_net_set_max_ctas")

    def profile_enable(self, enable=True):
        _check(_lib.lqcd_net_profile_enable(self.h, int(bool(enable))), "lqcd_net_profile_enable")

    def profile_read(self):
        """{(layer, kind): {launches, ms, bytes, flops}}, kind 'fwd', 'adj' or 'wgrad'."""
        n = 3 * (len(self.channels) - 1)
        arr = (lqcd_profile_entry * n)()
        _check(_lib.lqcd_net_profile_read(self.h, arr, n), "lqcd_net_profile_read")
        kinds = ("fwd", "adj", "wgrad")
        return {(i // 3, kinds[i % 3]): {"launches": arr[i].launches, "ms": arr[i].ms, "bytes": arr[i].bytes,
                                         "flops": arr[i].flops} for i in range(n)}

    def use_as_preconditioner(self, enable=True):
        """Make this network the FGCR right preconditioner of its lattice."""
        _check(_lib.lqcd_set_preconditioner(self.lat.ctx, self.h if enable else None),
               "lqcd_set_preconditioner")

    def set_weights(self, w):
        """w: complex64 tensor/array of num_weights entries."""
        t = torch.as_tensor(w).to(torch.complex64).contiguous()
        assert t.numel() == self.num_weights
        _check(_lib.lqcd_net_set_weights(self.h, _ptr(t)), "lqcd_net_set_weights")
        torch.cuda.synchronize()

    def get_weights(self, grad=False):
        w = torch.empty(self.num_weights, dtype=torch.complex64)
        g = torch.empty(self.num_weights, dtype=torch.complex64) if grad else None
        _check(_lib.lqcd_net_get_weights(self.h, _ptr(w), _ptr(g) if grad else None),
               "lqcd_net_get_weights")
        return (w, g) if grad else w

    def set_wait(self, limit_ns=0, expire_test=False):
        """Bound of the tensor-core kernels' waits (0: the default 2 s);
        expire_test makes each CTA's last wait run out (test of that path)."""
        _check(_lib.lqcd_net_set_wait(self.h, int(limit_ns), int(bool(expire_test))), "lqcd_net_set_wait")

    def layer_apply(self, layer, out, inp, batch=1, adjoint=False):
        _check(_lib.lqcd_net_layer_apply(self.h, int(layer), int(bool(adjoint)), _ptr(out), _ptr(inp),
                                         int(batch)), "lqcd_net_layer_apply")

    def layer_wgrad(self, layer, inp, gout, batch=1, zero=True):
        _check(_lib.lqcd_net_layer_wgrad(self.h, int(layer), _ptr(inp), _ptr(gout), int(batch),
                                         int(bool(zero))), "lqcd_net_layer_wgrad")

    def forward(self, out, inp, batch=1):
        _check(_lib.lqcd_net_forward(self.h, _ptr(out), _ptr(inp), int(batch)), "lqcd_net_forward")

    def train_step(self, r, e, batch, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        loss = C.c_double()
        _check(_lib.lqcd_net_train_step(self.h, _ptr(r), _ptr(e), int(batch), lr, beta1, beta2, eps,
                                        C.byref(loss)), "lqcd_net_train_step")
        return loss.value


# --------------------------------------------------------------- convenience

class Lattice:
    """One context + its workspace (a torch uint8 tensor on ``device``)."""

    def __init__(self, dims, t_antiperiodic=1, recon=12, precisions=("f64", "f32", "f16", "bf16",
                                                                     "f16links", "bf16links"),
                 max_nrhs=1, gcr_nkrylov=0, device="cuda", stream=None, part=(1, 1, 1, 1),
                 coord=(0, 0, 0, 0)):
        self.dims = tuple(int(d) for d in dims)
        self.device = torch.device(device)
        self.stream = stream
        with torch.cuda.device(self.device):
            self.ctx = lqcd_create(self.dims, t_antiperiodic, recon, precisions, max_nrhs,
                                   gcr_nkrylov, stream, part, coord)
            n = lqcd_workspace_size(self.ctx)
            self.workspace = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
            off = (-self.workspace.data_ptr()) % 256
            self._ws_view = self.workspace[off:off + n]
            lqcd_set_workspace(self.ctx, self._ws_view)
        self.volume = int(np.prod(self.dims))
        self.max_nrhs = int(max_nrhs)
        self.kappa, self.csw = 0.0, 0.0

    def close(self):
        if self.ctx is not None:
            lqcd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def field_bytes(self, prec):
        return lqcd_field_bytes(self.ctx, prec)

    def new_field(self, prec, nrhs=1, full=False):
        """Uninitialised internal field(s) as a uint8 device tensor."""
        n = self.field_bytes(prec) * (2 if full else 1) * nrhs
        return torch.empty(n, dtype=torch.uint8, device=self.device)

    def canonical_spinor(self, nrhs=1, host=False, pin=False):
        lx, ly, lz, lt = self.dims
        shp = ((nrhs,) if nrhs > 1 else ()) + (lt, lz, ly, lx, 4, 3)
        if host:
            return torch.zeros(shp, dtype=torch.complex128, pin_memory=pin)
        return torch.zeros(shp, dtype=torch.complex128, device=self.device)

    def gauge_load(self, links):
        lqcd_gauge_load(self.ctx, _as_tensor(links, self.device))

    def clover_compute(self, kappa, csw):
        lqcd_clover_compute(self.ctx, kappa, csw)
        self.kappa, self.csw = float(kappa), float(csw)

    def pack(self, internal, canonical, parity, prec, nrhs=1):
        lqcd_pack(self.ctx, internal, _as_tensor(canonical, self.device), parity, prec, nrhs)

    def unpack(self, canonical, internal, parity, prec, nrhs=1):
        lqcd_unpack(self.ctx, canonical, internal, parity, prec, nrhs)

    def dslash(self, out, inp, parity, kappa=0.0, csw=0.0, op=OP_HOP, dag=False, prec="f32", nrhs=1):
        lqcd_dslash(self.ctx, out, inp, parity, kappa, csw, op | (DAG if dag else 0), prec, nrhs)

    def clover_apply(self, out, inp, parity, inverse, prec="f32", nrhs=1):
        lqcd_clover_apply(self.ctx, out, inp, parity, inverse, prec, nrhs)

    def solve(self, x, b, tol=1e-10, nrhs=1, raise_on_error=True, **kw):
        return lqcd_solve(self.ctx, x, b, tol, nrhs, solver_params(**kw), raise_on_error)

    def sap_apply(self, z, r, block, ncycle=1, nmr=4):
        lqcd_sap_apply(self.ctx, z, r, block, ncycle, nmr)

    def set_sap(self, block, ncycle=1, nmr=4):
        lqcd_set_preconditioner_sap(self.ctx, block, ncycle, nmr)

    def sync(self):
        lqcd_sync(self.ctx)


def _as_tensor(a, device):
    """numpy complex128 -> device tensor; tensors pass through."""
    if isinstance(a, torch.Tensor):
        return a.contiguous()
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)
