"""Thin ctypes binding of the dlz C ABI (include/dlz.h); argument marshalling only.

Every function carries the name of its C counterpart without the `dlz_`
prefix.  Vectors are torch tensors (CUDA or CPU) or numpy arrays of complex128
(complex64 for FP32 `apply`) laid out as [..., V, 4, 3]; the library itself
detects host or device memory and does every step of the computation in its
CUDA kernels.  There is no fallback: if libdlz.so is missing, importing this
module raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdlz.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "dlz.h")

OK = 0
ERR_BADARG = -1
ERR_BAD_GAUGE = -2
ERR_NONFINITE = -3
ERR_NOT_CONVERGED = -4
ERR_BREAKDOWN = -5
ERR_DEVICE_TIMEOUT = -6
ERR_CUDA = -7
ERR_OOM = -8
ERR_IO = -9

D, DDAG, Q, DDAGD = 0, 1, 2, 3
F64, F32, BF16 = 0, 1, 2


class Params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("k", ctypes.c_int), ("tol", ctypes.c_double),
                ("tol_eig", ctypes.c_double), ("oversolve", ctypes.c_double),
                ("max_cycles", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("reorth_period", ctypes.c_int), ("precision", ctypes.c_int),
                ("reliable_delta", ctypes.c_double), ("check_every", ctypes.c_int),
                ("profile", ctypes.c_int), ("finish", ctypes.c_int), ("eig_only", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("iterations", ctypes.c_int), ("cycles", ctypes.c_int),
                ("mvps", ctypes.c_longlong), ("true_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("stencil_ms", ctypes.c_double),
                ("stencil_launches", ctypes.c_longlong), ("stencil_bytes", ctypes.c_double),
                ("gpu_launches", ctypes.c_longlong), ("kernel_ms", ctypes.c_double * 3),
                ("kernel_bytes", ctypes.c_double * 3), ("kernel_launches", ctypes.c_longlong * 3)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k.startswith("kernel_") else getattr(self, k))
                for k, _ in self._fields_}


class DlzError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_0901_3163_gb300.build.build()")
lib = ctypes.CDLL(LIB_PATH)

_vp = ctypes.c_void_p
_ip = ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "dlz_params_default": ([ctypes.POINTER(Params)], _ip),
    "dlz_strerror": ([_ip], ctypes.c_char_p),
    "dlz_last_error": ([], ctypes.c_char_p),
    "dlz_create_operator": ([ctypes.POINTER(ctypes.c_int), _vp, ctypes.c_double, _ip, _vp,
                             ctypes.POINTER(_vp)], _ip),
    "dlz_destroy_operator": ([_vp], _ip),
    "dlz_op_volume": ([_vp, ctypes.POINTER(ctypes.c_longlong)], _ip),
    "dlz_apply": ([_vp, _ip, _vp, _vp, _ip, _ip], _ip),
    "dlz_create_operator_eo": ([ctypes.POINTER(ctypes.c_int), _vp, ctypes.c_double, _ip, _vp,
                                ctypes.POINTER(_vp)], _ip),
    "dlz_eo_prepare": ([_vp, _vp, _vp, _ip], _ip),
    "dlz_basis_combine": ([_vp, ctypes.c_longlong, _ip, ctypes.c_longlong, _vp, _ip, _ip, _vp, ctypes.c_longlong], _ip),
    "dlz_basis_dots": ([_vp, ctypes.c_longlong, _ip, _vp, ctypes.c_longlong, _ip, ctypes.c_longlong, _vp], _ip),
    "dlz_batch_last_choice": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int)], _ip),
    "dlz_eo_reconstruct": ([_vp, _vp, _vp, _vp, _ip], _ip),
    "dlz_apply_noalloc": ([_vp, _ip, _vp, _vp, _ip, _ip], _ip),
    "dlz_landr": ([_vp, _vp, _vp, ctypes.POINTER(Params), ctypes.POINTER(_vp),
                   ctypes.POINTER(Stats)], _ip),
    "dlz_minresdr": ([_vp, _vp, _vp, ctypes.POINTER(Params), ctypes.POINTER(_vp),
                      ctypes.POINTER(Stats)], _ip),
    "dlz_dcg": ([_vp, _vp, _vp, _vp, _ip, ctypes.POINTER(Params), ctypes.POINTER(Stats)], _ip),
    "dlz_dminres": ([_vp, _vp, _vp, _vp, _ip, ctypes.POINTER(Params), ctypes.POINTER(Stats)], _ip),
    "dlz_gmresdr": ([_vp, _vp, _vp, ctypes.POINTER(Params), ctypes.POINTER(_vp), ctypes.POINTER(Stats)], _ip),
    "dlz_dgmres": ([_vp, _vp, _vp, _vp, _ip, ctypes.POINTER(Params), ctypes.POINTER(Stats)], _ip),
    "dlz_defl_value_complex": ([_vp, _ip, _dp, _dp], _ip),
    "dlz_defl_count": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], _ip),
    "dlz_defl_get": ([_vp, _ip, _vp, _dp, _dp], _ip),
    "dlz_defl_save": ([_vp, ctypes.c_char_p], _ip),
    "dlz_defl_load": ([_vp, ctypes.c_char_p, ctypes.POINTER(_vp)], _ip),
    "dlz_defl_destroy": ([_vp], _ip),
    "dlz_stencil_bench": ([_vp, _ip, _ip, _ip, _ip, _vp, _dp], _ip),
    "dlz_batch_dminres": ([_ip, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                           ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Params),
                           ctypes.POINTER(Stats)], _ip),
    "dlz_net_create": ([_vp, _ip, ctypes.POINTER(ctypes.c_int), _vp, ctypes.POINTER(_vp)], _ip),
    "dlz_net_destroy": ([_vp], _ip),
    "dlz_net_weight_count": ([_vp, ctypes.POINTER(ctypes.c_longlong)], _ip),
    "dlz_net_bind": ([_vp, _vp], _ip),
    "dlz_net_forward": ([_vp, _vp, _ip, _vp], _ip),
    "dlz_net_backward": ([_vp, _vp, _ip, _vp], _ip),
    "dlz_net_get": ([_vp, _ip, _vp], _ip),
    "dlz_net_set_weights": ([_vp, _vp], _ip),
    "dlz_net_zero_grad": ([_vp], _ip),
    "dlz_net_adam_step": ([_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double], _ip),
    "dlz_subspace_loss": ([_vp, _vp, _ip, ctypes.c_double, _dp, _vp], _ip),
    "dlz_seed_deflation": ([_vp, _ip, _vp, _ip, _ip, ctypes.POINTER(_vp)], _ip),
    "dlz_host_symeig": ([_ip, _vp, _vp, _vp], _ip),
    "dlz_host_sym_extremes": ([_ip, _vp, _vp, _vp], _ip),
    "dlz_host_lstsq": ([_ip, _ip, _vp, _vp, _vp, _vp], _ip),
    "dlz_host_zgeev": ([_ip, _vp, _vp, _vp], _ip),
    "dlz_host_rayleigh_ritz": ([_ip, _vp, _vp, _vp, _vp], _ip),
    "dlz_host_zlstsq": ([_ip, _ip, _vp, _vp, _vp, _vp], _ip),
    "dlz_host_restart_plan": ([_ip, _ip, _ip, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _ip),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def header_symbols():
    """Function names declared in include/dlz.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|const char \*)\s*(dlz_\w+)\s*\(", txt, re.M)))


def strerror(code):
    return lib.dlz_strerror(code).decode()


def last_error():
    return lib.dlz_last_error().decode()


def _check(rc, allow=()):
    if rc != OK and rc not in allow:
        raise DlzError(rc, last_error() or strerror(rc))
    return rc


def _ptr(a):
    """Data pointer of a contiguous torch tensor or numpy array."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr()


def _empty_like(a, dtype=None):
    if isinstance(a, np.ndarray):
        return np.empty(a.shape, dtype=dtype or a.dtype)
    import torch
    return torch.empty(a.shape, dtype=dtype or a.dtype, device=a.device)


def _empty_shape(a, shape):
    """Uninitialised array of `shape` with a's dtype, on a's device."""
    if isinstance(a, np.ndarray):
        return np.empty(shape, dtype=a.dtype)
    import torch
    return torch.empty(shape, dtype=a.dtype, device=a.device)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def params_default(**overrides):
    p = Params()
    _check(lib.dlz_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class Operator:
    """Handle of a dlz_op_t (dlz_create_operator / dlz_destroy_operator)."""

    def __init__(self, handle, dims, kappa, bc_t):
        self.handle = handle
        self.dims = tuple(dims)
        self.kappa = kappa
        self.bc_t = bc_t

    @property
    def volume(self):
        v = ctypes.c_longlong()
        _check(lib.dlz_op_volume(self.handle, ctypes.byref(v)))
        return v.value

    def __del__(self):
        if getattr(self, "handle", None):
            lib.dlz_destroy_operator(self.handle)
            self.handle = None


class Deflation:
    """Handle of a dlz_defl_t (the k eigenvectors passed to D-CG / D-MinRes)."""

    def __init__(self, handle, op):
        self.handle = handle
        self.op = op            # keeps the operator alive

    def __del__(self):
        if getattr(self, "handle", None):
            lib.dlz_defl_destroy(self.handle)
            self.handle = None


def create_operator(dims, gauge, kappa, bc_t=1, stream=None):
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    h = _vp()
    _check(lib.dlz_create_operator(d, _ptr(gauge), float(kappa), int(bc_t),
                                   _stream_handle(stream), ctypes.byref(h)))
    return Operator(h, dims, kappa, bc_t)


def create_operator_eo(dims, gauge, kappa, bc_t=1, stream=None):
    """Even-odd (Schur complement) operator on the even sites; its vectors are [V/2, 4, 3]."""
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    h = _vp()
    _check(lib.dlz_create_operator_eo(d, _ptr(gauge), float(kappa), int(bc_t),
                                      _stream_handle(stream), ctypes.byref(h)))
    op = Operator(h, dims, kappa, bc_t)
    op.eo = True
    return op


def eo_prepare(op, b, out=None):
    """b_e + kappa H_eo b_o for full-lattice b [nrhs?, V, 4, 3] -> [nrhs?, V/2, 4, 3]."""
    nrhs = int(np.prod(b.shape)) // (24 * op.volume)
    if out is None:
        out = _empty_shape(b, tuple(b.shape[:-3]) + (op.volume, 4, 3))
    _check(lib.dlz_eo_prepare(op.handle, _ptr(b), _ptr(out), nrhs))
    return out


def eo_reconstruct(op, x_e, b, out=None):
    """Full solution (x_e, b_o + kappa H_oe x_e) [nrhs?, V, 4, 3] from x_e and b."""
    nrhs = int(np.prod(b.shape)) // (24 * op.volume)
    if out is None:
        out = _empty_like(b)
    _check(lib.dlz_eo_reconstruct(op.handle, _ptr(x_e), _ptr(b), _ptr(out), nrhs))
    return out


def apply(op, which, x, out=None, dtype=None):
    """out = A x for A in {D, DDAG, Q, DDAGD}; x is [nrhs?, V, 4, 3]."""
    if dtype is None:
        dtype = F32 if str(x.dtype).endswith("complex64") else F64
    if out is None:
        out = _empty_like(x)
    V = op.volume
    nrhs = int(np.prod(x.shape)) // (12 * V) if np.prod(x.shape) else 0
    _check(lib.dlz_apply(op.handle, int(which), _ptr(x), _ptr(out), int(dtype), nrhs))
    return out


def _dr(fn, op, b, params, x, deflate):
    p = params if params is not None else params_default()
    if x is None:
        x = _empty_like(b)
    st = Stats()
    h = _vp()
    rc = _check(fn(op.handle, _ptr(b), _ptr(x), ctypes.byref(p),
                   ctypes.byref(h) if deflate else None, ctypes.byref(st)),
                allow=(ERR_NOT_CONVERGED,))
    defl = Deflation(h, op) if (deflate and h.value) else None
    return x, defl, st


def landr(op, b, params=None, x=None, deflate=True):
    """Lan-DR(m,k) on D^dagger D for D x = b: returns (x, Deflation, Stats)."""
    return _dr(lib.dlz_landr, op, b, params, x, deflate)


def minresdr(op, b, params=None, x=None, deflate=True):
    """MinRes-DR(m,k) on gamma5 D for D x = b: returns (x, Deflation, Stats)."""
    return _dr(lib.dlz_minresdr, op, b, params, x, deflate)


def _dsolve(fn, op, defl, B, params, X):
    p = params if params is not None else params_default()
    if X is None:
        X = _empty_like(B)
    V = op.volume
    nrhs = int(np.prod(B.shape)) // (12 * V)
    st = (Stats * max(nrhs, 1))()
    _check(fn(op.handle, defl.handle if defl is not None else None, _ptr(B), _ptr(X), nrhs,
              ctypes.byref(p), st), allow=(ERR_NOT_CONVERGED,))
    return X, [st[i] for i in range(nrhs)]


def gmresdr(op, b, params=None, x=None, deflate=True):
    """GMRES-DR(m,k) on D for D x = b (FP64): returns (x, Deflation, Stats)."""
    return _dr(lib.dlz_gmresdr, op, b, params, x, deflate)


def dgmres(op, defl, B, params=None, X=None):
    """D-GMRES(m) over a GMRES-DR set (None: plain GMRES(m)); returns (X, [Stats])."""
    return _dsolve(lib.dlz_dgmres, op, defl, B, params, X)


def defl_value_complex(defl, i):
    """The i-th value of a deflation set as a complex number (GMRES-DR: theta_i)."""
    re, im = ctypes.c_double(), ctypes.c_double()
    _check(lib.dlz_defl_value_complex(defl.handle, int(i), ctypes.byref(re), ctypes.byref(im)))
    return complex(re.value, im.value)


def dcg(op, defl, B, params=None, X=None):
    """D-CG (Galerkin projection over defl, then CG on D^dagger D); returns (X, [Stats])."""
    return _dsolve(lib.dlz_dcg, op, defl, B, params, X)


def dminres(op, defl, B, params=None, X=None):
    """D-MinRes (Galerkin projection over defl, then MinRes on gamma5 D); returns (X, [Stats])."""
    return _dsolve(lib.dlz_dminres, op, defl, B, params, X)


def batch_dminres(ops, defls, Bs, params=None, Xs=None):
    """dlz_batch_dminres: D-MinRes on several lattices at once.  ops, defls (or None
    entries), Bs: per lattice [nrhs, V, 4, 3] complex128.  Returns (Xs, [[Stats]])."""
    nlat = len(ops)
    p = params if params is not None else params_default()
    if Xs is None:
        Xs = [_empty_like(b) for b in Bs]
    nr = [int(np.prod(b.shape)) // (12 * o.volume) for b, o in zip(Bs, ops)]
    oa = (_vp * nlat)(*[o.handle for o in ops])
    da = (_vp * nlat)(*[(d.handle if d is not None else None) for d in defls])
    ba = (_vp * nlat)(*[_ptr(b) for b in Bs])
    xa = (_vp * nlat)(*[_ptr(x) for x in Xs])
    na = (ctypes.c_int * nlat)(*nr)
    st = (Stats * max(sum(nr), 1))()
    _check(lib.dlz_batch_dminres(nlat, oa, da, ba, xa, na, ctypes.byref(p), st), allow=(ERR_NOT_CONVERGED,))
    out, q = [], 0
    for r in nr:
        out.append([st[q + i] for i in range(r)])
        q += r
    return Xs, out


def basis_combine(V, coef, out=None):
    """out[j] = sum_i coef[i, j] V[i] on the tensor cores.  V: device float32 [nin, len]
    (real coef, float64 [nin, nout]) or complex64 [nin, L] (complex coef, complex128
    [nin, nout])."""
    import torch
    cplx = V.dtype == torch.complex64
    nin = V.shape[0]
    nout = coef.shape[1]
    Vf = torch.view_as_real(V).reshape(nin, -1) if cplx else V
    ln = Vf.shape[1]
    if out is None:
        out = torch.empty((nout,) + tuple(V.shape[1:]), dtype=V.dtype, device=V.device)
    of = torch.view_as_real(out).reshape(nout, -1) if cplx else out
    c = np.ascontiguousarray(coef, dtype=np.complex128 if cplx else np.float64)
    _check(lib.dlz_basis_combine(_ptr(Vf), ln, nin, ln, c.ctypes.data, nout, int(cplx), _ptr(of), ln))
    return out


def basis_dots(V, R):
    """C[q, i] = <V_i, R_q> (complex) on the tensor cores; V, R: device complex64 [n?, L]."""
    import torch
    nin, nq = V.shape[0], R.shape[0]
    Vf = torch.view_as_real(V).reshape(nin, -1)
    Rf = torch.view_as_real(R).reshape(nq, -1)
    ln = Vf.shape[1]
    C = np.empty((nq, nin), dtype=np.complex128)
    _check(lib.dlz_basis_dots(_ptr(Vf), ln, nin, _ptr(Rf), ln, nq, ln, C.ctypes.data))
    return C


def batch_last_choice(op):
    """(form, chunks per block, half grid) the last FP32 batch_dminres call on op chose."""
    f, c, h = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib.dlz_batch_last_choice(op.handle, ctypes.byref(f), ctypes.byref(c), ctypes.byref(h)))
    return f.value, c.value, h.value


def defl_count(defl):
    k, w = ctypes.c_int(), ctypes.c_int()
    _check(lib.dlz_defl_count(defl.handle, ctypes.byref(k), ctypes.byref(w)))
    return k.value, w.value


def defl_get(defl, i, vec_out=None):
    """(value, residual) of Rayleigh-Ritz pair i; fills vec_out ([V,4,3]) if given."""
    v, r = ctypes.c_double(), ctypes.c_double()
    _check(lib.dlz_defl_get(defl.handle, int(i), _ptr(vec_out), ctypes.byref(v), ctypes.byref(r)))
    return v.value, r.value


def defl_save(defl, path):
    _check(lib.dlz_defl_save(defl.handle, str(path).encode()))


def defl_load(op, path):
    h = _vp()
    _check(lib.dlz_defl_load(op.handle, str(path).encode(), ctypes.byref(h)))
    return Deflation(h, op)


def apply_noalloc(op, which, x, out=None):
    """dlz_apply_noalloc: out = A x like apply(), with device tensors only and the
    library's static device scratch instead of temporary allocations."""
    dtype = F32 if str(x.dtype).endswith("complex64") else F64
    nrhs = int(np.prod(x.shape)) // (12 * op.volume)
    if out is None:
        out = _empty_like(x)
    _check(lib.dlz_apply_noalloc(op.handle, int(which), _ptr(x), _ptr(out), dtype, nrhs))
    return out


def stencil_bench(op, x, iters=50, which=D, dtype=None):
    """Average device time of one stencil launch over x's right-hand sides ([nrhs, V, 4, 3]);
    dtype BF16 stores the complex64 x as bfloat16."""
    if dtype is None:
        dtype = F32 if str(x.dtype).endswith("complex64") else F64
    nrhs = int(np.prod(x.shape)) // (12 * op.volume)
    ms = ctypes.c_double()
    _check(lib.dlz_stencil_bench(op.handle, dtype, int(which), nrhs, int(iters), _ptr(x), ctypes.byref(ms)))
    return {"ms": ms.value, "nrhs": nrhs}


class Network:
    """Handle of a dlz_net_t: the parallel-transport convolution network."""

    def __init__(self, handle, op, widths):
        self.handle = handle
        self.op = op
        self.widths = tuple(widths)

    def __del__(self):
        if getattr(self, "handle", None) and lib is not None:
            lib.dlz_net_destroy(self.handle)
            self.handle = None


def net_weight_shapes(widths):
    """Shapes of the layers' weights: (9, w[l+1], w[l], 4, 4)."""
    return [(9, widths[i + 1], widths[i], 4, 4) for i in range(len(widths) - 1)]


def _flat_weights(Ws):
    return np.ascontiguousarray(np.concatenate([np.asarray(w).reshape(-1) for w in Ws]).astype(np.complex64))


def _split_weights(flat, widths):
    out, o = [], 0
    for shp in net_weight_shapes(widths):
        n = int(np.prod(shp))
        out.append(flat[o:o + n].reshape(shp))
        o += n
    return out


def net_create(op, widths, Ws):
    """dlz_net_create with per-layer complex weights Ws (shapes net_weight_shapes(widths))."""
    w = (ctypes.c_int * len(widths))(*widths)
    flat = _flat_weights(Ws)
    h = _vp()
    _check(lib.dlz_net_create(op.handle, len(widths) - 1, w, flat.ctypes.data, ctypes.byref(h)))
    return Network(h, op, widths)


def net_bind(net, op):
    """Use op's links from now on (same lattice)."""
    _check(lib.dlz_net_bind(net.handle, op.handle))
    net.op = op


def net_forward(net, x, out=None):
    """f = N x for device complex64 x [nvec, V, 4, 3] (or [V, 4, 3])."""
    nvec = int(np.prod(x.shape)) // (12 * net.op.volume)
    if out is None:
        out = _empty_like(x)
    _check(lib.dlz_net_forward(net.handle, _ptr(x), nvec, _ptr(out)))
    return out


def net_backward(net, grad_out, want_input_grad=False):
    """Adds G(W) of the last forward to the gradients; returns G(x) if asked."""
    nvec = int(np.prod(grad_out.shape)) // (12 * net.op.volume)
    gin = _empty_like(grad_out) if want_input_grad else None
    _check(lib.dlz_net_backward(net.handle, _ptr(grad_out), nvec, _ptr(gin)))
    return gin


def _net_count(net):
    c = ctypes.c_longlong()
    _check(lib.dlz_net_weight_count(net.handle, ctypes.byref(c)))
    return c.value


def net_get(net, what=0):
    """Per-layer arrays: what = 0 master weights, 1 gradients, 2 bfloat16 weights in use."""
    flat = np.empty(_net_count(net), dtype=np.complex64)
    _check(lib.dlz_net_get(net.handle, int(what), flat.ctypes.data))
    return _split_weights(flat, net.widths)


def net_set_weights(net, Ws):
    flat = _flat_weights(Ws)
    _check(lib.dlz_net_set_weights(net.handle, flat.ctypes.data))


def net_zero_grad(net):
    _check(lib.dlz_net_zero_grad(net.handle))


def net_adam_step(net, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(lib.dlz_net_adam_step(net.handle, float(lr), float(beta1), float(beta2), float(eps)))


def subspace_loss(defl, f, want_grad=True, grad_scale=1.0):
    """Per-vector ||(1 - V V^dag) f||^2 / ||f||^2 against defl, and grad_scale * G(f)
    (device complex64)."""
    nvec = int(np.prod(f.shape)) // (12 * defl.op.volume)
    loss = np.empty(nvec)
    g = _empty_like(f) if want_grad else None
    _check(lib.dlz_subspace_loss(defl.handle, _ptr(f), nvec, ctypes.c_double(grad_scale),
                                 loss.ctypes.data_as(_dp), _ptr(g)))
    return loss, g


def seed_deflation(op, vecs, which=DDAGD):
    """Deflation set from the span of k device vectors [k, V, 4, 3] (Rayleigh-Ritz with A)."""
    dtype = F32 if str(vecs.dtype).endswith("complex64") else F64
    k = int(np.prod(vecs.shape)) // (12 * op.volume)
    h = _vp()
    _check(lib.dlz_seed_deflation(op.handle, int(which), _ptr(vecs), dtype, k, ctypes.byref(h)))
    return Deflation(h, op)


def host_symeig(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.empty(n)
    Z = np.empty((n, n))
    _check(lib.dlz_host_symeig(n, A.ctypes.data, w.ctypes.data, Z.ctypes.data))
    return w, Z


def host_sym_extremes(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib.dlz_host_sym_extremes(A.shape[0], A.ctypes.data, ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def host_restart_plan(T, c, k, harmonic, anorm=0.0):
    """dlz_host_restart_plan on Tbar ((m+1) x m) and c; returns a dict of y, P, Tn,
    cn, theta, ritz_res, anorm."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    m = T.shape[1]
    out = dict(y=np.empty(m), P=np.empty((m + 1, k + 1)), Tn=np.empty((m + 1, m)), cn=np.empty(m + 1),
               theta=np.empty(k), ritz_res=np.empty(k))
    an = ctypes.c_double(anorm)
    _check(lib.dlz_host_restart_plan(int(bool(harmonic)), m, k, T.ctypes.data, c.ctypes.data,
                                     *(out[key].ctypes.data for key in ("y", "P", "Tn", "cn", "theta", "ritz_res")),
                                     ctypes.byref(an)))
    out["anorm"] = an.value
    return out


def host_zgeev(A):
    """Eigenvalues and unit eigenvectors of a general complex matrix (library host code)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    n = A.shape[0]
    w = np.empty(n, dtype=np.complex128)
    Z = np.empty((n, n), dtype=np.complex128)
    _check(lib.dlz_host_zgeev(n, A.ctypes.data, w.ctypes.data, Z.ctypes.data))
    return w, Z


def host_rayleigh_ritz(H, G=None):
    """Rayleigh-Ritz pairs of a deflation set's H = V^dag A V, with the Gram matrix G =
    V^dag V of a basis orthonormal only to rounding (None: orthonormal): ascending values
    and vectors z (columns) with H z = value G z, z^dag G z = 1 (library host code)."""
    H = np.ascontiguousarray(H, dtype=np.complex128)
    k = H.shape[0]
    Gc = None if G is None else np.ascontiguousarray(G, dtype=np.complex128)
    w = np.empty(k, dtype=np.float64)
    Z = np.empty((k, k), dtype=np.complex128)
    _check(lib.dlz_host_rayleigh_ritz(k, H.ctypes.data, None if Gc is None else Gc.ctypes.data, w.ctypes.data,
                                      Z.ctypes.data))
    return w, Z


def host_zlstsq(A, c):
    """argmin ||c - A y|| (complex) and the unit vector spanning range(A)^perp (rows = cols + 1)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    c = np.ascontiguousarray(c, dtype=np.complex128)
    rows, cols = A.shape
    y = np.empty(cols, dtype=np.complex128)
    q = np.empty(rows, dtype=np.complex128)
    _check(lib.dlz_host_zlstsq(rows, cols, A.ctypes.data, c.ctypes.data, y.ctypes.data,
                               q.ctypes.data if rows == cols + 1 else None))
    return y, (q if rows == cols + 1 else None)


def host_lstsq(T, c):
    T = np.ascontiguousarray(T, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    rows, cols = T.shape
    y = np.empty(cols)
    q = np.empty(rows)
    _check(lib.dlz_host_lstsq(rows, cols, T.ctypes.data, c.ctypes.data, y.ctypes.data,
                              q.ctypes.data if rows == cols + 1 else None))
    return y, (q if rows == cols + 1 else None)
