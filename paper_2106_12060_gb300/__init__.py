"""GB300 (sm_103a) sketch-preconditioned Riemannian CCA / Fisher LDA.

Thin Python binding over libgbcca.so with the names of the C ABI
(include/gbcca.h).  Device memory and streams come from PyTorch; every step
of the method runs in the library's CUDA kernels.  Importing works without a
GPU; calls need CUDA tensors on the current device.

Method: Shustin & Avron, "Faster Randomized Methods for Orthogonality
Constrained Problems" - Alg. 1 (CCA) and Alg. 2 (FDA).
"""
from __future__ import annotations

import ctypes as C

from . import _lib
from ._lib import (  # noqa: F401
    BF16, FP32, FP64, COUNTSKETCH, SRHT, IDENTITY, EXACT, Options, Info, GbccaError,
    Q_SKETCH_X, Q_SKETCH_Y, Q_R_X, Q_R_Y, Q_WARM_U, Q_WARM_V, Q_HISTORY, Q_CLASS_MEANS, Q_RITZ,
    OK, ERR_MAXITER, ERR_NOT_SPD, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_STATE, ERR_TIMEOUT, ERR_CUDA, ERR_OOM,
)

_DTYPE_NAMES = {"bf16": BF16, "f32": FP32, "fp32": FP32, "f64": FP64, "fp64": FP64}
STATUS_NAMES = {0: "ok", -1: "invalid_arg", -2: "unsupported", -3: "oom", -4: "not_spd", -5: "maxiter",
                -6: "timeout", -7: "cuda", -8: "state"}


def _torch():
    import torch
    return torch


def dtype_code(dtype) -> int:
    """Library dtype code of a torch dtype or a name ('bf16', 'f32', 'f64')."""
    if isinstance(dtype, int):
        return dtype
    if isinstance(dtype, str):
        return _DTYPE_NAMES[dtype]
    torch = _torch()
    return {torch.bfloat16: BF16, torch.float32: FP32, torch.float64: FP64}[dtype]


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _check_dev(name, t, dtype=None, rows=None, cols=None):
    """Reject, before any call into the library, a tensor that is not on the
    current CUDA device, has the wrong dtype, or is smaller than the shape the
    call reads or writes through its raw pointer."""
    torch = _torch()
    if t is None:
        raise ValueError(f"{name} is required")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} must be a CUDA tensor on the current device")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if rows is not None or cols is not None:
        if t.dim() != 2 or (rows is not None and t.shape[0] != rows) or (cols is not None and t.shape[1] != cols):
            raise ValueError(f"{name} must be ({rows}, {cols}), got {tuple(t.shape)}")
        if t.stride(1) != 1 or (t.shape[0] > 1 and t.stride(0) < t.shape[1]):
            raise ValueError(f"{name} must have unit column stride and row stride >= its columns")


_STORAGE = {0: "bfloat16", 1: "float32", 2: "float64"}


def _storage_dtype(code):
    return getattr(_torch(), _STORAGE[code])


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def default_options(**kw) -> Options:
    lib = _lib.load()
    o = Options()
    _lib.check(lib.gbcca_default_options(C.byref(o)), "gbcca_default_options")
    for key, val in kw.items():
        setattr(o, key, val)
    return o


class Plan:
    """Owns a gbcca_plan_t; frees it on close() / garbage collection."""

    def __init__(self, handle, kind, n, dims, k, dtype, opt, l=0):
        self.handle = handle
        self.kind = kind
        self.n = n
        self.dims = dims
        self.k = k
        self.dtype = dtype
        self.opt = opt
        self.l = l

    def close(self):
        if self.handle is not None:
            _lib.load().gbcca_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cca_plan(n, dx, dy, k, dtype, opt: Options | None = None) -> Plan:
    lib = _lib.load()
    h = C.c_void_p()
    code = dtype_code(dtype)
    _lib.check(lib.cca_plan(C.byref(h), n, dx, dy, k, code, C.byref(opt) if opt else None), "cca_plan")
    return Plan(h, "cca", n, (dx, dy), k, code, opt)


def lda_plan(n, d, n_classes, k, dtype, opt: Options | None = None) -> Plan:
    lib = _lib.load()
    h = C.c_void_p()
    code = dtype_code(dtype)
    _lib.check(lib.lda_plan(C.byref(h), n, d, n_classes, k, code, C.byref(opt) if opt else None), "lda_plan")
    return Plan(h, "lda", n, (d,), k, code, opt, l=n_classes)


def cca_precondition(plan: Plan, X, Y, lambda_x, lambda_y, sketch_h=None, sketch_g=None, stream=None):
    """X (n x dx), Y (n x dy): CUDA tensors of the plan's dtype, rows contiguous."""
    lib = _lib.load()
    torch = _torch()
    dx, dy = plan.dims
    dt = _storage_dtype(plan.dtype)
    _check_dev("X", X, dt, plan.n, dx)
    _check_dev("Y", Y, dt, plan.n, dy)
    for name, t in (("sketch_h", sketch_h), ("sketch_g", sketch_g)):
        if t is not None:
            _check_dev(name, t, torch.int32 if name == "sketch_h" else torch.int8)
    _lib.check(lib.cca_precondition(plan.handle, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0), float(lambda_x),
                                    float(lambda_y), _ptr(sketch_h), _ptr(sketch_g), _stream(stream)),
               "cca_precondition")
    plan._data = (X, Y, sketch_h, sketch_g)  # keep the caller's buffers alive with the plan


def cca_solve(plan: Plan, mu=None, tol=0.0, U=None, V=None, sigma=None, stream=None, allow_maxiter=True):
    """Returns (sigma, U, V, info dict).  U/V (float64, dx x k / dy x k) are
    also the start when the plan was made with warm_start = 0."""
    torch = _torch()
    lib = _lib.load()
    dx, dy = plan.dims
    dev = torch.device("cuda", torch.cuda.current_device())
    U = U if U is not None else torch.empty(dx, plan.k, dtype=torch.float64, device=dev)
    V = V if V is not None else torch.empty(dy, plan.k, dtype=torch.float64, device=dev)
    sigma = sigma if sigma is not None else torch.empty(plan.k, dtype=torch.float64, device=dev)
    _check_dev("U", U, torch.float64, dx, plan.k)
    _check_dev("V", V, torch.float64, dy, plan.k)
    _check_dev("sigma", sigma, torch.float64)
    if not (U.is_contiguous() and V.is_contiguous() and sigma.numel() >= plan.k):
        raise ValueError("U, V must be contiguous and sigma must hold k entries")
    info = Info()
    mu_arr = (C.c_double * plan.k)(*mu) if mu is not None else None
    allow = (OK, ERR_MAXITER) if allow_maxiter else (OK,)
    _lib.check(lib.cca_solve(plan.handle, mu_arr, float(tol), _ptr(U), _ptr(V), _ptr(sigma), C.byref(info),
                             _stream(stream)), "cca_solve", allow)
    return sigma, U, V, info.as_dict()


def lda_solve(plan: Plan, X, labels, lam, mu=None, tol=0.0, W=None, rho=None, sketch_h=None, sketch_g=None,
              stream=None, allow_maxiter=True):
    """X (n x d) CUDA tensor of the plan's dtype, labels int32 (n).  Returns
    (rho, W, info dict)."""
    torch = _torch()
    lib = _lib.load()
    (d,) = plan.dims
    dev = X.device
    W = W if W is not None else torch.empty(d, plan.k, dtype=torch.float64, device=dev)
    rho = rho if rho is not None else torch.empty(plan.k, dtype=torch.float64, device=dev)
    info = Info()
    mu_arr = (C.c_double * plan.k)(*mu) if mu is not None else None
    allow = (OK, ERR_MAXITER) if allow_maxiter else (OK,)
    _check_dev("X", X, _storage_dtype(plan.dtype), plan.n, d)
    _check_dev("labels", labels, torch.int32)
    if labels.dim() != 1 or labels.shape[0] != plan.n or not labels.is_contiguous():
        raise ValueError("labels must be a contiguous int32 vector of n entries")
    _check_dev("W", W, torch.float64, d, plan.k)
    _check_dev("rho", rho, torch.float64)
    _lib.check(lib.lda_solve(plan.handle, _ptr(X), X.stride(0), _ptr(labels), float(lam), mu_arr, float(tol),
                             _ptr(sketch_h), _ptr(sketch_g), _ptr(W), _ptr(rho), C.byref(info), _stream(stream)),
               "lda_solve", allow)
    plan._data = (X, labels)
    return rho, W, info.as_dict()


def gbcca_fused_pass(plan: Plan, Phi_x, Phi_y=None, stream=None):
    """One fused data pass at Phi_x (dx x 2k) / Phi_y (dy x 2k).  Returns
    (Gx, Gy, Gram) as float64 CUDA tensors (Gy None for an FDA plan)."""
    torch = _torch()
    lib = _lib.load()
    dev = Phi_x.device
    k2 = 2 * plan.k
    nc = (2 if plan.kind == "cca" else 1) * k2
    Gx = torch.empty(plan.dims[0], nc, dtype=torch.float64, device=dev)
    Gy = torch.empty(plan.dims[1], nc, dtype=torch.float64, device=dev) if plan.kind == "cca" else None
    Gram = torch.empty(nc, nc, dtype=torch.float64, device=dev)
    _lib.check(lib.gbcca_fused_pass(plan.handle, _ptr(Phi_x.contiguous()),
                                    _ptr(Phi_y.contiguous() if Phi_y is not None else None), _ptr(Gx), _ptr(Gy),
                                    _ptr(Gram), _stream(stream)), "gbcca_fused_pass")
    return Gx, Gy, Gram


fused_pass = gbcca_fused_pass


def gbcca_query(plan: Plan, what: int, stream=None):
    torch = _torch()
    lib = _lib.load()
    n = lib.gbcca_query_size(plan.handle, what)
    if n < 0:
        raise ValueError("query not available for this plan")
    out = torch.empty(n, dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
    _lib.check(lib.gbcca_query(plan.handle, what, _ptr(out), _stream(stream)), "gbcca_query")
    return out


query = gbcca_query


def gbcca_sketch_draws(kind, n, s, seed, stream=None):
    """Library-drawn sketch randomness: CountSketch -> (h[n], g[n]);
    SRHT (n a power of two) -> (rows[s], signs[n])."""
    torch = _torch()
    lib = _lib.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    if kind == COUNTSKETCH:
        h = torch.empty(n, dtype=torch.int32, device=dev)
        g = torch.empty(n, dtype=torch.int8, device=dev)
    else:
        h = torch.empty(s, dtype=torch.int32, device=dev)
        g = torch.empty(n, dtype=torch.int8, device=dev)
    _lib.check(lib.gbcca_sketch_draws(kind, n, s, seed, _ptr(h), _ptr(g), _stream(stream)), "gbcca_sketch_draws")
    return h, g


sketch_draws = gbcca_sketch_draws


def gbcca_sketch_gram_noalloc(A, lam, C, stream=None):
    """C = A^T A + lam I without any device allocation by the library (the
    split-K partials use its static scratch).  A: CUDA float64 (m, d) with
    unit column stride; C: caller-provided CUDA float64 (d, d), contiguous."""
    torch = _torch()
    if A.dim() != 2 or A.stride(1) != 1 or C.dim() != 2 or not C.is_contiguous():
        raise ValueError("A must be (m, d) with unit column stride and C a contiguous (d, d) tensor")
    m, d = A.shape
    if tuple(C.shape) != (d, d):
        raise ValueError("C must be (d, d)")
    _check_dev("A", A, torch.float64, m, d)
    _check_dev("C", C, torch.float64, d, d)
    lib = _lib.load()
    _lib.check(lib.gbcca_sketch_gram_noalloc(_ptr(A), A.stride(0), m, d, float(lam), _ptr(C), _stream(stream)),
               "gbcca_sketch_gram_noalloc")
    return C


sketch_gram_noalloc = gbcca_sketch_gram_noalloc


def gbcca_sketch_gram_noalloc_max_d() -> int:
    """Largest d the allocation-free Gram accepts."""
    return int(_lib.load().gbcca_sketch_gram_noalloc_max_d())


sketch_gram_noalloc_max_d = gbcca_sketch_gram_noalloc_max_d


def gbcca_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(_lib.load().gbcca_launch_count())


launch_count = gbcca_launch_count


def default_batch_options(**kw) -> _lib.BatchOptions:
    lib = _lib.load()
    o = _lib.BatchOptions()
    _lib.check(lib.gbcca_default_batch_options(C.byref(o)), "gbcca_default_batch_options")
    for key, val in kw.items():
        setattr(o, key, val)
    return o


class Batch:
    """Owns a gbcca_batch_t over prepared plans (each bound to its data);
    keeps the plans alive while it exists."""

    def __init__(self, plans, opt=None):
        lib = _lib.load()
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = C.c_void_p()
        _lib.check(lib.gbcca_batch_create(C.byref(h), arr, len(self.plans), C.byref(opt) if opt else None),
                   "gbcca_batch_create")
        self.handle = h

    def close(self):
        if self.handle is not None:
            _lib.load().gbcca_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gbcca_batch_create(plans, opt=None) -> Batch:
    return Batch(plans, opt)


batch_create = gbcca_batch_create


def gbcca_batch_solve(batch: Batch, stream=None, allow_maxiter=True):
    """Solves every plan of the batch.  Returns (results, report): results[i]
    = (sigma, U, V, info) for a CCA plan, (rho, W, None, info) for an FDA
    plan; report a dict of the batched launch."""
    torch = _torch()
    lib = _lib.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    n = len(batch.plans)
    outs = []
    for p in batch.plans:
        U = torch.empty(p.dims[0], p.k, dtype=torch.float64, device=dev)
        V = torch.empty(p.dims[1], p.k, dtype=torch.float64, device=dev) if p.kind == "cca" else None
        s = torch.empty(p.k, dtype=torch.float64, device=dev)
        outs.append((s, U, V))
    Ua = (C.c_void_p * n)(*[o[1].data_ptr() for o in outs])
    Va = (C.c_void_p * n)(*[o[2].data_ptr() if o[2] is not None else 0 for o in outs])
    Sa = (C.c_void_p * n)(*[o[0].data_ptr() for o in outs])
    infos = (Info * n)()
    rep = _lib.BatchReport()
    allow = (OK, ERR_MAXITER) if allow_maxiter else (OK,)
    _lib.check(lib.gbcca_batch_solve(batch.handle, Ua, Va, Sa, infos, C.byref(rep), _stream(stream)),
               "gbcca_batch_solve", allow)
    res = [(o[0], o[1], o[2], infos[i].as_dict()) for i, o in enumerate(outs)]
    report = {f: getattr(rep, f) for f, _ in _lib.BatchReport._fields_ if f != "reserved"}
    return res, report


batch_solve = gbcca_batch_solve


def gbcca_batch_fused_pass(batch: Batch, Phi_x, Phi_y, stream=None):
    """One batched pass: Phi_x[i] (dx_i x 2k_i), Phi_y[i] (dy_i x 2k_i) float64
    CUDA tensors.  Returns lists (G[i] ((dx + dy) x 4k), Gram[i] (4k x 4k))."""
    torch = _torch()
    lib = _lib.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    n = len(batch.plans)
    Px = [t.contiguous() for t in Phi_x]
    Py = [t.contiguous() for t in Phi_y]
    for i, p in enumerate(batch.plans):
        _check_dev(f"Phi_x[{i}]", Px[i], torch.float64, p.dims[0], 2 * p.k)
        _check_dev(f"Phi_y[{i}]", Py[i], torch.float64, p.dims[1], 2 * p.k)
    G = [torch.empty(sum(p.dims), 4 * p.k, dtype=torch.float64, device=dev) for p in batch.plans]
    Gram = [torch.empty(4 * p.k, 4 * p.k, dtype=torch.float64, device=dev) for p in batch.plans]
    arr = lambda ts: (C.c_void_p * n)(*[t.data_ptr() for t in ts])  # noqa: E731
    _lib.check(lib.gbcca_batch_fused_pass(batch.handle, arr(Px), arr(Py), arr(G), arr(Gram), _stream(stream)),
               "gbcca_batch_fused_pass")
    return G, Gram


batch_fused_pass = gbcca_batch_fused_pass


def default_server_options(**kw) -> _lib.ServerOptions:
    lib = _lib.load()
    o = _lib.ServerOptions()
    _lib.check(lib.gbcca_default_server_options(C.byref(o)), "gbcca_default_server_options")
    for key, val in kw.items():
        setattr(o, key, val)
    return o


class Server:
    """Owns a gbcca_server_t.  Submitted tensors are kept alive until their
    request's result is taken (the server reads them at admission)."""

    QUEUED, RUNNING, FINISHED, FAILED = 0, 1, 2, 3

    def __init__(self, opt=None):
        lib = _lib.load()
        h = C.c_void_p()
        _lib.check(lib.gbcca_server_create(C.byref(h), C.byref(opt) if opt else None), "gbcca_server_create")
        self.handle = h
        self._keep = {}
        self._shape = {}

    def _submit(self, req, keep, shape):
        rid = C.c_int64()
        _lib.check(_lib.load().gbcca_server_submit(self.handle, C.byref(req), C.byref(rid)), "gbcca_server_submit")
        self._keep[rid.value] = keep
        self._shape[rid.value] = shape
        return rid.value

    def submit_cca(self, X, Y, k, lambda_x, lambda_y, opt=None):
        """X (n x dx), Y (n x dy): CUDA tensors, or pinned host tensors, of
        one storage dtype, unit column stride."""
        n, dx = X.shape
        dy = Y.shape[1]
        for name, t in (("X", X), ("Y", Y)):
            if t.stride(1) != 1 or t.shape[0] != n or t.dtype != X.dtype:
                raise ValueError(f"{name} must be n x d with unit column stride and X's dtype")
        r = _lib.Request(kind=0, dtype=dtype_code(X.dtype), n=n, dx=dx, dy=dy, k=k, n_classes=0,
                         lambda_x=float(lambda_x), lambda_y=float(lambda_y), X=X.data_ptr(), ldx=X.stride(0),
                         Y=Y.data_ptr(), ldy=Y.stride(0), labels=None, opt=opt or default_options())
        return self._submit(r, (X, Y), ("cca", dx, dy, k))

    def submit_lda(self, X, labels, n_classes, k, lam, opt=None):
        n, d = X.shape
        if X.stride(1) != 1 or labels.dtype != _torch().int32 or labels.numel() != n:
            raise ValueError("X must be n x d with unit column stride and labels int32 of n entries")
        r = _lib.Request(kind=1, dtype=dtype_code(X.dtype), n=n, dx=d, dy=0, k=k, n_classes=n_classes,
                         lambda_x=float(lam), lambda_y=0.0, X=X.data_ptr(), ldx=X.stride(0), Y=None, ldy=0,
                         labels=labels.data_ptr(), opt=opt or default_options())
        return self._submit(r, (X, labels), ("lda", d, 0, k))

    def step(self, stream=None):
        q, r = C.c_int32(), C.c_int32()
        _lib.check(_lib.load().gbcca_server_step(self.handle, C.byref(q), C.byref(r), _stream(stream)),
                   "gbcca_server_step")
        return q.value, r.value

    def state(self, rid):
        return int(_lib.load().gbcca_server_state(self.handle, rid))

    def result(self, rid):
        """(vals, U, V, info, times) of a finished request as float64 CUDA
        tensors (V None for FDA); raises GbccaError if it failed."""
        torch = _torch()
        kind, d0, d1, k = self._shape[rid]
        dev = torch.device("cuda", torch.cuda.current_device())
        U = torch.empty(d0, k, dtype=torch.float64, device=dev)
        V = torch.empty(d1, k, dtype=torch.float64, device=dev) if kind == "cca" else None
        vals = torch.empty(k, dtype=torch.float64, device=dev)
        info, times = Info(), _lib.RequestTimes()
        rc = _lib.load().gbcca_server_result(self.handle, rid, _ptr(U), _ptr(V), _ptr(vals), C.byref(info),
                                             C.byref(times))
        self._keep.pop(rid, None)
        self._shape.pop(rid, None)
        _lib.check(rc, "gbcca_server_result", (OK, ERR_MAXITER))
        return vals, U, V, info.as_dict(), {f: getattr(times, f) for f, _ in times._fields_}

    def close(self):
        if self.handle is not None:
            _lib.load().gbcca_server_destroy(self.handle)
            self.handle = None
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
