"""ctypes binding of ``include/krr.h``: argument marshalling only.

Every function here takes tensors (device) or numpy arrays (host), passes
their pointers and sizes to the C ABI of the same name and raises
``KrrError`` on a non-zero status.  No arithmetic of the method happens in
Python.  The library must have been built (``paper_1611_03220_gb300.build()``);
a missing library raises ``ImportError`` at import time, there is no
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkrr_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run paper_1611_03220_gb300.build() first")
_lib = C.CDLL(LIB_PATH)

KRR_MAX_RHS = 16
STATUS = {0: "KRR_OK", 1: "KRR_EINVAL", 2: "KRR_ENOMEM", 3: "KRR_ECUDA", 4: "KRR_ECHOL",
          5: "KRR_ENOTCONV", 6: "KRR_EBREAKDOWN", 7: "KRR_ENAN", 8: "KRR_ETIMEOUT",
          9: "KRR_EUNSUPPORTED"}
KRR_OK, KRR_EINVAL, KRR_ENOMEM, KRR_ECUDA, KRR_ECHOL = 0, 1, 2, 3, 4
KRR_ENOTCONV, KRR_EBREAKDOWN, KRR_ENAN, KRR_ETIMEOUT, KRR_EUNSUPPORTED = 5, 6, 7, 8, 9
PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2, "hp": 3, "mixed": 4, "bf16x3": 5,
             "bf16p": 6, "fp16": 7}
APPLY_FORM = {"zl": 0, "u": 1}


class krr_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("lambda_p", C.c_double),
                ("precond", C.c_int), ("precision", C.c_int), ("apply_form", C.c_int),
                ("use_graph", C.c_int), ("inner_tol", C.c_double), ("max_outer", C.c_int),
                ("z_format", C.c_int), ("warm_start", C.c_int), ("inner_precision", C.c_int),
                ("batch_product", C.c_int), ("keep_direction", C.c_int),
                ("fuse_step", C.c_int)]


class krr_report(C.Structure):
    _fields_ = [("status", C.c_int), ("k", C.c_int), ("iters", C.c_int * KRR_MAX_RHS),
                ("rel_res", C.c_double * KRR_MAX_RHS), ("outer_steps", C.c_int),
                ("matvecs", C.c_int), ("ms_setup", C.c_double), ("ms_solve", C.c_double),
                ("ms_total", C.c_double), ("kappa", C.c_double * KRR_MAX_RHS),
                ("rel_res_rec", C.c_double * KRR_MAX_RHS)]

    def as_dict(self) -> dict:
        """The report's first k columns as plain Python values."""
        k = self.k
        return {"status": STATUS.get(self.status, self.status), "k": k,
                "iters": list(self.iters[:k]), "rel_res": list(self.rel_res[:k]),
                "outer_steps": self.outer_steps, "matvecs": self.matvecs,
                "ms_setup": self.ms_setup, "ms_solve": self.ms_solve, "ms_total": self.ms_total,
                "kappa": list(self.kappa[:k]), "rel_res_rec": list(self.rel_res_rec[:k])}


class krr_problem(C.Structure):
    _fields_ = [("X", C.c_void_p), ("n", C.c_int), ("d", C.c_int), ("ldx", C.c_int),
                ("sigma", C.c_double), ("lam", C.c_double), ("W", C.c_void_p),
                ("b", C.c_void_p), ("s", C.c_int), ("Y", C.c_void_p), ("k", C.c_int),
                ("ldy", C.c_int), ("C", C.c_void_p), ("ldc", C.c_int)]


class krr_matvec_problem(C.Structure):
    _fields_ = [("X", C.c_void_p), ("n", C.c_int), ("d", C.c_int), ("ldx", C.c_int),
                ("sigma", C.c_double), ("shift", C.c_double), ("V", C.c_void_p),
                ("Q", C.c_void_p)]


_vp, _i, _d = C.c_void_p, C.c_int, C.c_double
_SIGS = {
    "krr_default_opts": (None, [C.POINTER(krr_opts)]),
    "krr_create": (_i, [C.POINTER(_vp), _vp]),
    "krr_destroy": (_i, [_vp]),
    "krr_set_stream": (_i, [_vp, _vp]),
    "krr_last_error": (C.c_char_p, [_vp]),
    "krr_status_string": (C.c_char_p, [_i]),
    "krr_set_autotune": (_i, [_vp, _i, C.POINTER(_i)]),
    "krr_rff_features": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp, _i, _vp, _i]),
    "krr_rff_features_fixed": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp, _i, _vp, _i,
                                    C.POINTER(_i)]),
    "krr_kernel_matvec": (_i, [_vp, _vp, _i, _i, _vp, _i, _i, _i, _d, _d, _vp, _i, _i, _vp, _i, _i]),
    "krr_precond_setup": (_i, [_vp, _vp, _i, _i, _i, _d, _i, _i]),
    "krr_precond_apply": (_i, [_vp, _vp, _i, _i, _vp, _i]),
    "krr_pcg_solve": (_i, [_vp, _vp, _i, _i, _i, _d, _d, _vp, _vp, _i, _vp, _i, _i, _vp, _i,
                           C.POINTER(krr_opts), C.POINTER(krr_report)]),
    "krr_pcg_solve_batched": (_i, [_vp, C.POINTER(krr_problem), _i, C.POINTER(krr_opts),
                                   C.POINTER(krr_report)]),
    "krr_predict": (_i, [_vp, _vp, _i, _i, _vp, _i, _i, _i, _d, _vp, _i, _i, _vp, _i, _i]),
    "krr_rfm_fit": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp, _i, _d, _vp, _i, _i, _vp, _i]),
    "krr_rfm_predict": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp, _i, _vp, _i, _i, _vp, _i]),
    "krr_kernel_matvec_fp64_noalloc": (_i, [_vp, _i, _i, _vp, _i, _i, _i, _d, _d, _vp, _i, _i,
                                            _vp, _i, _vp]),
    "krr_kernel_dsigma_matvec": (_i, [_vp, _vp, _i, _i, _vp, _i, _i, _i, _d, _vp, _i, _i, _vp,
                                      _i, _i]),
    "krr_hypergrad": (_i, [_vp, _vp, _i, _i, _i, _vp, _i, _i, _d, _d, _vp, _vp, _i, _vp, _i, _vp,
                           _i, _i, C.POINTER(krr_opts), C.POINTER(_d), _vp, _i,
                           C.POINTER(krr_report)]),
    "krr_tensorsketch_features": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp, _i, _i, _d, _d, _vp,
                                       _i]),
    "krr_kernel_matvec_poly": (_i, [_vp, _vp, _i, _i, _vp, _i, _i, _i, _d, _d, _i, _d, _vp, _i,
                                    _i, _vp, _i, _i]),
    "krr_poly_pcg_solve": (_i, [_vp, _vp, _i, _i, _i, _d, _d, _i, _d, _vp, _vp, _i, _vp, _i, _i,
                                _vp, _i, C.POINTER(krr_opts), C.POINTER(krr_report)]),
    "krr_multilevel_features": (_i, [_vp, _vp, _i, _i, _i, _vp, _i, _vp, _i, _vp, _i, _vp, _i]),
    "krr_precond_setup_adaptive": (_i, [_vp, _vp, _i, _i, _i, _d, _d, _vp, _vp, _i, _i, _vp, _i,
                                        _i, _i, _d, _i, _i, C.POINTER(_i), C.POINTER(_d),
                                        C.POINTER(_i)]),
    "krr_kernel_matvec_batched": (_i, [_vp, C.POINTER(krr_matvec_problem), _i]),
    "krr_launch_count": (C.c_longlong, []),
    "krr_bench_ex2": (_i, [_vp, _i, C.POINTER(_d), C.POINTER(_d)]),
    "krr_bench_ex2_mix": (_i, [_vp, _i, _i, C.POINTER(_d), C.POINTER(_d)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class KrrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(a) -> int:
    """Data pointer of a torch tensor or a numpy array (no copy)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _ld(a) -> int:
    """Leading dimension (elements) of a row-major 2-D array."""
    if isinstance(a, np.ndarray):
        assert a.shape[1] == 1 or a.strides[1] == a.itemsize, "inner stride must be 1"
        return a.strides[0] // a.itemsize
    assert a.shape[1] == 1 or a.stride(1) == 1, "inner stride must be 1"
    return a.stride(0)


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Handle:
    """Owns a ``krr_handle`` bound to a CUDA stream (torch's current one by default)."""

    def __init__(self, stream=None):
        self._h = _vp()
        st = _lib.krr_create(C.byref(self._h), _stream_ptr(stream))
        if st != KRR_OK:
            raise KrrError(st, "krr_create failed")

    @property
    def ptr(self):
        """The ``krr_handle*`` to pass to the C functions."""
        return self._h

    def set_stream(self, stream=None):
        """Bind the handle to ``stream`` (a torch stream; None: torch's current one)."""
        self._check(_lib.krr_set_stream(self._h, _stream_ptr(stream)))

    def set_autotune(self, on=True) -> int:
        """Tile-plan selection: False/0 the fixed rule, True/1 autotune, 2 the
        symmetric product where it applies (16 epilogue warps), 3 the same with 8;
        returns the shapes tuned so far."""
        n = _i(0)
        mode = int(on) if not isinstance(on, bool) else (1 if on else 0)
        st = _lib.krr_set_autotune(self._h, mode, C.byref(n))
        if st != KRR_OK:
            raise KrrError(st, "krr_set_autotune: mode must be 0, 1, 2 or 3")
        return n.value

    def _check(self, st: int):
        if st != KRR_OK:
            raise KrrError(st, _lib.krr_last_error(self._h).decode())

    def close(self):
        """Destroy the handle (synchronises its stream, frees its workspace)."""
        if self._h:
            _lib.krr_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def default_opts(**kw) -> krr_opts:
    """``krr_default_opts`` with the given fields overridden; ``precision`` and
    ``inner_precision`` may be names ("fp64", "fp32", "mixed", "fp16", "bf16", ...),
    ``apply_form`` "zl" or "u"."""
    o = krr_opts()
    _lib.krr_default_opts(C.byref(o))
    for k, v in kw.items():
        if k in ("precision", "inner_precision") and isinstance(v, str):
            v = PRECISION[v]
        if k == "apply_form" and isinstance(v, str):
            v = APPLY_FORM[v]
        setattr(o, k, v)
    return o


def krr_rff_features(h: Handle, X, W, b, Z):
    """Z = sqrt(2/s) cos(X W + b) into the caller's Z (n x s float32, device)."""
    n, d = X.shape
    s = W.shape[1]
    h._check(_lib.krr_rff_features(h.ptr, _ptr(X), n, d, _ld(X), _ptr(W), _ptr(b), s,
                                   _ptr(Z), _ld(Z)))
    return Z


def krr_kernel_matvec(h: Handle, Xr, Xc, sigma: float, shift: float, V, Q, precision="fp64"):
    """Q = K(Xr, Xc) V + shift V into the caller's Q (device tensors)."""
    nr, d = Xr.shape
    nc = Xc.shape[0]
    k = V.shape[1]
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    h._check(_lib.krr_kernel_matvec(h.ptr, _ptr(Xr), nr, _ld(Xr), _ptr(Xc), nc, _ld(Xc), d,
                                    float(sigma), float(shift), _ptr(V), k, _ld(V), _ptr(Q),
                                    _ld(Q), prec))
    return Q


def krr_kernel_matvec_fp64_noalloc(Xr, Xc, sigma: float, shift: float, V, Q, stream=None) -> int:
    """FP64 Q = K(Xr, Xc) V + shift V without any device allocation; returns the status.

    For callers that cannot allocate (see include/krr.h); no handle needed.
    """
    nr, d = Xr.shape
    nc = Xc.shape[0]
    k = V.shape[1]
    return _lib.krr_kernel_matvec_fp64_noalloc(_ptr(Xr), nr, _ld(Xr), _ptr(Xc), nc, _ld(Xc), d,
                                               float(sigma), float(shift), _ptr(V), k, _ld(V),
                                               _ptr(Q), _ld(Q), _stream_ptr(stream))


Z_FORMAT = {"fp32": 0, "bf16": 1, "fixed": 2}


def krr_precond_setup(h: Handle, Z, lambda_p: float, apply_form="zl", z_format="fp32"):
    """Preconditioner set-up from the features Z (n x s float32): G = Z^T Z + lambda_p I,
    its Cholesky factor and the factors of the apply form ("zl" or "u"); the handle
    stores Z as ``z_format`` ("fp32", "bf16" or "fixed": 7-bit fixed point with an
    exact tensor-core Gram)."""
    n, s = Z.shape
    form = APPLY_FORM[apply_form] if isinstance(apply_form, str) else int(apply_form)
    zf = Z_FORMAT[z_format] if isinstance(z_format, str) else int(z_format)
    h._check(_lib.krr_precond_setup(h.ptr, _ptr(Z), n, s, _ld(Z), float(lambda_p), form, zf))


def krr_rff_features_fixed(h: Handle, X, W, b, Zq) -> int:
    """Fixed-point random Fourier features on the tensor cores: Zq (n x s torch.int8)
    holds q with Z ~= 2^(e-7) q; returns e."""
    n, d = X.shape
    s = W.shape[1]
    e = C.c_int()
    h._check(_lib.krr_rff_features_fixed(h.ptr, _ptr(X), n, d, _ld(X), _ptr(W), _ptr(b), s,
                                         _ptr(Zq), _ld(Zq), C.byref(e)))
    return e.value


def krr_precond_apply(h: Handle, R, Zout):
    """Zout = (Z Z^T + lambda_p I)^-1 R by the Woodbury identity (R, Zout n x k float64)."""
    k = R.shape[1]
    h._check(_lib.krr_precond_apply(h.ptr, _ptr(R), k, _ld(R), _ptr(Zout), _ld(Zout)))
    return Zout


def krr_pcg_solve(h: Handle, X, sigma: float, lam: float, W, b, Y, C_out, opts: krr_opts | None = None,
                  check: bool = True) -> dict:
    """Algorithm 1 end to end into C_out; host (numpy) or device (torch) buffers.

    Returns the report as a dict.  With ``check`` a non-OK status raises
    (KRR_ENOTCONV included); otherwise the status is only reported.
    """
    n, d = X.shape
    k = Y.shape[1]
    s = W.shape[1] if W is not None else 0
    rep = krr_report()
    o = opts if opts is not None else default_opts()
    st = _lib.krr_pcg_solve(h.ptr, _ptr(X), n, d, _ld(X), float(sigma), float(lam),
                            _ptr(W) if W is not None else None,
                            _ptr(b) if b is not None else None, s,
                            _ptr(Y), k, _ld(Y), _ptr(C_out), _ld(C_out), C.byref(o), C.byref(rep))
    if check:
        h._check(st)
    out = rep.as_dict()
    out["status_code"] = st
    return out


def krr_tensorsketch_features(h: Handle, X, hash_, sign, s: int, gamma: float, c: float, Z):
    """TensorSketch features of the polynomial kernel (gamma x.z + c)^q into Z (n x s
    float32); hash_ (q x d~ int32) and sign (q x d~ int8) are the q CountSketches."""
    n, d = X.shape
    q = hash_.shape[0]
    h._check(_lib.krr_tensorsketch_features(h.ptr, _ptr(X), n, d, _ld(X), _ptr(hash_),
                                            _ptr(sign), q, int(s), float(gamma), float(c),
                                            _ptr(Z), _ld(Z)))
    return Z


def krr_kernel_matvec_poly(h: Handle, Xr, Xc, gamma: float, c: float, q: int, shift: float, V, Q,
                           precision="fp64"):
    """Q = (gamma Xr Xc^T + c)^q V + shift V (float64 for "fp64", float32 for the
    tensor-core precisions "fp16", "bf16", "bf16x3")."""
    nr, d = Xr.shape
    nc = Xc.shape[0]
    k = V.shape[1]
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    h._check(_lib.krr_kernel_matvec_poly(h.ptr, _ptr(Xr), nr, _ld(Xr), _ptr(Xc), nc, _ld(Xc), d,
                                         float(gamma), float(c), int(q), float(shift), _ptr(V),
                                         k, _ld(V), _ptr(Q), _ld(Q), prec))
    return Q


def krr_poly_pcg_solve(h: Handle, X, gamma: float, c: float, q: int, lam: float, hash_, sign,
                       s: int, Y, C_out, opts: krr_opts | None = None, check: bool = True) -> dict:
    """Algorithm 1 for the polynomial kernel with the TensorSketch preconditioner."""
    n, d = X.shape
    k = Y.shape[1]
    rep = krr_report()
    o = opts if opts is not None else default_opts()
    st = _lib.krr_poly_pcg_solve(h.ptr, _ptr(X), n, d, _ld(X), float(gamma), float(c), int(q),
                                 float(lam), _ptr(hash_) if hash_ is not None else None,
                                 _ptr(sign) if sign is not None else None, int(s), _ptr(Y), k,
                                 _ld(Y), _ptr(C_out), _ld(C_out), C.byref(o), C.byref(rep))
    if check:
        h._check(st)
    out = rep.as_dict()
    out["status_code"] = st
    return out


def krr_multilevel_features(h: Handle, Z1, signs, rows, G, Z3):
    """Algorithm 2's features: Z3 = s3^-1/2 (Z1 S2^T) G^T with the SRHT S2 = s2^-1/2 P H D
    (signs: m int8, rows: s2 int32) and G (s3 x s2 float32); Z1, Z3 float32."""
    n, s1 = Z1.shape
    s3, s2 = G.shape
    h._check(_lib.krr_multilevel_features(h.ptr, _ptr(Z1), n, s1, _ld(Z1), _ptr(signs),
                                          len(signs), _ptr(rows), s2, _ptr(G), s3, _ptr(Z3),
                                          _ld(Z3)))
    return Z3


def krr_precond_setup_adaptive(h: Handle, X, sigma: float, lam: float, W, b, s0: int, x0,
                               power_iters: int = 30, ns_iters: int = 25, precision="fp64",
                               lambda_p: float = 0.0, apply_form="zl", z_format=-1) -> dict:
    """Theorem 4's adaptive sketch size: double s from s0 (up to W's columns) until
    ||(I - P) K (I - P)|| <= 0.1 lambda; sets up the handle's preconditioner with the
    chosen features.  Returns {"s", "estimates", "tests"}."""
    n, d = X.shape
    s_max = W.shape[1]
    est = (C.c_double * 64)()
    s_out, tests = C.c_int(), C.c_int()
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    form = APPLY_FORM[apply_form] if isinstance(apply_form, str) else int(apply_form)
    zf = Z_FORMAT[z_format] if isinstance(z_format, str) else int(z_format)
    h._check(_lib.krr_precond_setup_adaptive(h.ptr, _ptr(X), n, d, _ld(X), float(sigma),
                                             float(lam), _ptr(W), _ptr(b), s_max, int(s0),
                                             _ptr(x0), int(power_iters), int(ns_iters), prec,
                                             float(lambda_p), form, zf, C.byref(s_out), est,
                                             C.byref(tests)))
    return {"s": s_out.value, "estimates": [est[i] for i in range(tests.value)],
            "tests": tests.value}


def krr_kernel_matvec_batched(h: Handle, problems):
    """Kernel products of independent problems in one persistent launch:
    ``problems`` is a sequence of ``(X, sigma, shift, V, Q)`` with device tensors
    (X n x d float32, V and Q n x 1 float32); Q_p = K_p V_p + shift_p V_p on
    FP16 points."""
    arr = (krr_matvec_problem * len(problems))()
    for i, (X, sigma, shift, V, Q) in enumerate(problems):
        n, d = X.shape
        arr[i] = krr_matvec_problem(_ptr(X), n, d, _ld(X), float(sigma), float(shift), _ptr(V),
                                    _ptr(Q))
    h._check(_lib.krr_kernel_matvec_batched(h.ptr, arr, len(problems)))


def krr_pcg_solve_batched(h: Handle, problems, opts: krr_opts | None = None,
                          check: bool = True) -> list[dict]:
    """Algorithm 1 for independent problems in lockstep (one graph launch per round).

    ``problems``: a sequence of ``(X, sigma, lam, W, b, Y, C_out)`` tuples of
    host (numpy) or device (torch) buffers, shapes as for ``krr_pcg_solve``.
    Returns one report dict per problem; with ``check`` a non-OK status raises.
    """
    arr = (krr_problem * len(problems))()
    for i, (X, sigma, lam, W, b, Y, Cout) in enumerate(problems):
        n, d = X.shape
        arr[i] = krr_problem(_ptr(X), n, d, _ld(X), float(sigma), float(lam),
                             _ptr(W) if W is not None else None,
                             _ptr(b) if b is not None else None,
                             W.shape[1] if W is not None else 0,
                             _ptr(Y), Y.shape[1], _ld(Y), _ptr(Cout), _ld(Cout))
    reps = (krr_report * len(problems))()
    o = opts if opts is not None else default_opts()
    st = _lib.krr_pcg_solve_batched(h.ptr, arr, len(problems), C.byref(o), reps)
    if check:
        h._check(st)
    out = []
    for r in reps:
        dct = r.as_dict()
        dct["status_code"] = r.status
        out.append(dct)
    return out


def krr_predict(h: Handle, Xtr, Xte, sigma: float, Cc, F, precision="fp64"):
    """F = K(Xte, Xtr) Cc, the kernel ridge regression predictor at the rows of Xte."""
    n, d = Xtr.shape
    m = Xte.shape[0]
    k = Cc.shape[1]
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    h._check(_lib.krr_predict(h.ptr, _ptr(Xtr), n, _ld(Xtr), _ptr(Xte), m, _ld(Xte), d,
                              float(sigma), _ptr(Cc), k, _ld(Cc), _ptr(F), _ld(F), prec))
    return F


def krr_rfm_fit(h: Handle, X, W, b, lam: float, Y, Wf):
    """Random-features ridge solution Wf = (Z^T Z + lam I)^-1 Z^T Y into Wf (s x k)."""
    n, d = X.shape
    s = W.shape[1]
    k = Y.shape[1]
    h._check(_lib.krr_rfm_fit(h.ptr, _ptr(X), n, d, _ld(X), _ptr(W), _ptr(b), s, float(lam),
                              _ptr(Y), k, _ld(Y), _ptr(Wf), _ld(Wf)))


def krr_rfm_predict(h: Handle, Xte, W, b, Wf, F):
    """F = phi(Xte) Wf, the random-features predictor."""
    m, d = Xte.shape
    s = W.shape[1]
    k = Wf.shape[1]
    h._check(_lib.krr_rfm_predict(h.ptr, _ptr(Xte), m, d, _ld(Xte), _ptr(W), _ptr(b), s,
                                  _ptr(Wf), k, _ld(Wf), _ptr(F), _ld(F)))


def krr_kernel_dsigma_matvec(h: Handle, Xr, Xc, sigma: float, V, Q, precision="fp64"):
    """Q = (D o K)(Xr, Xc) V, the derivative of the product with respect to log sigma."""
    nr, d = Xr.shape
    nc = Xc.shape[0]
    k = V.shape[1]
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    h._check(_lib.krr_kernel_dsigma_matvec(h.ptr, _ptr(Xr), nr, _ld(Xr), _ptr(Xc), nc, _ld(Xc),
                                           d, float(sigma), _ptr(V), k, _ld(V), _ptr(Q), _ld(Q),
                                           prec))
    return Q


def krr_hypergrad(h: Handle, X, Xte, sigma: float, lam: float, W, b, Cc, GF,
                  opts: krr_opts | None = None, Wadj=None, check: bool = True):
    """(dL/dlog sigma, dL/dlog lambda) for dL/dF = GF at F = K(Xte, X) Cc.

    Returns ``(grad, report)``: grad a 2-tuple, report the adjoint solve's dict.
    """
    n, d = X.shape
    m = Xte.shape[0]
    k = GF.shape[1]
    s = W.shape[1] if W is not None else 0
    rep = krr_report()
    g = (_d * 2)()
    o = opts if opts is not None else default_opts()
    st = _lib.krr_hypergrad(h.ptr, _ptr(X), n, d, _ld(X), _ptr(Xte), m, _ld(Xte), float(sigma),
                            float(lam), _ptr(W) if W is not None else None,
                            _ptr(b) if b is not None else None, s, _ptr(Cc), _ld(Cc), _ptr(GF), k,
                            _ld(GF), C.byref(o), g, _ptr(Wadj) if Wadj is not None else None,
                            _ld(Wadj) if Wadj is not None else k, C.byref(rep))
    if check:
        h._check(st)
    out = rep.as_dict()
    out["status_code"] = st
    return (g[0], g[1]), out
