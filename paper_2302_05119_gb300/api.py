"""Python front end of libcncpd: argument marshalling around the C ABI of
include/cncpd.h.  Every computation runs in the library's CUDA kernels.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); they must be C-contiguous float32 or float64.
"""

import ctypes

import numpy as np

from . import _lib as C


def _torch():
    try:
        import torch
        return torch
    except ImportError:  # pragma: no cover
        return None


def _is_torch(a):
    t = _torch()
    return t is not None and isinstance(a, t.Tensor)


def _dtype_code(a):
    if _is_torch(a):
        t = _torch()
        if a.dtype == t.float64:
            return C.CNCPD_F64
        if a.dtype == t.float32:
            return C.CNCPD_F32
        raise TypeError(f"unsupported tensor dtype {a.dtype}")
    if a.dtype == np.float64:
        return C.CNCPD_F64
    if a.dtype == np.float32:
        return C.CNCPD_F32
    raise TypeError(f"unsupported array dtype {a.dtype}")


def _prep(a, dtype=None):
    """Contiguous array/tensor (optionally cast); returns (obj, pointer, code)."""
    if _is_torch(a):
        t = _torch()
        if dtype is not None:
            a = a.to({np.float64: t.float64, np.float32: t.float32}[dtype])
        a = a.contiguous()
        return a, ctypes.c_void_p(a.data_ptr()), _dtype_code(a)
    a = np.asarray(a)
    if dtype is not None:
        a = a.astype(dtype, copy=False)
    if a.dtype not in (np.float32, np.float64):
        a = a.astype(np.float64)
    a = np.ascontiguousarray(a)
    return a, ctypes.c_void_p(a.ctypes.data), _dtype_code(a)


_STORAGE = {None: -1, "f64": C.CNCPD_F64, "f32": C.CNCPD_F32, "bf16": C.CNCPD_BF16, "bf16x2": C.CNCPD_BF16X2}


def default_opts():
    o = C.cncpd_opts()
    C.cncpd_default_opts(ctypes.byref(o))
    return o


class CoupledNCP:
    """K coupled nonnegative CP models solved by CoNCPD-APG / lraCoNCPD-APG.

    tensors: K arrays of shape (I_1, ..., I_N); R: rank (int or K ints);
    L: coupled columns per mode; nonneg: per-mode projection flags.
    The keyword options mirror cncpd_opts (include/cncpd.h): storage (None,
    "f64", "f32", "bf16", "bf16x2"), tensor_cores, autotune, tf32 (FP32
    data: trailing pass on the TF32 tensor cores, opt-in) and stream_x (one
    block of X on the device at a time; lraCoNCPD-APG only, the tensors are
    kept referenced by this object).
    """

    def __init__(self, tensors, R, L, nonneg=None, storage=None, use_core=False, reupdate=True,
                 eps=1e-8, max_it=1000, lra_eps=1e-4, lra_max_it=200, delta_w=0.9999,
                 use_graph=True, profile=False, tensor_cores=True, autotune=True, tf32=False, stream_x=False,
                 stream=None):
        self.K = len(tensors)
        self.N = len(tensors[0].shape)
        self.R = [int(r) for r in (R if np.ndim(R) else [R] * self.K)]
        self.L = [int(x) for x in L]
        self.dims = [tuple(int(s) for s in X.shape) for X in tensors]
        o = default_opts()
        o.eps, o.max_it, o.lra_eps, o.lra_max_it, o.delta_w = eps, max_it, lra_eps, lra_max_it, delta_w
        o.use_core, o.reupdate = int(use_core), int(reupdate)
        o.storage = _STORAGE[storage]
        o.use_graph, o.profile = int(use_graph), int(profile)
        o.tensor_cores = int(tensor_cores)
        o.autotune = int(autotune)
        o.tf32 = int(tf32)
        o.stream_x = int(stream_x)
        self.opts = o
        code0 = None
        keep, ptrs = [], []
        for X in tensors:
            obj, p, code = _prep(X)
            if code0 is None:
                code0 = code
            elif code != code0:
                obj, p, code = _prep(X, np.float64 if code0 == C.CNCPD_F64 else np.float32)
            keep.append(obj)
            ptrs.append(p.value)
        dims = (ctypes.c_int64 * (self.K * self.N))(*[d for dd in self.dims for d in dd])
        Xp = (ctypes.c_void_p * self.K)(*ptrs)
        Rp = (ctypes.c_int * self.K)(*self.R)
        Lp = (ctypes.c_int * self.N)(*self.L)
        nn = None if nonneg is None else (ctypes.c_ubyte * self.N)(*[1 if b else 0 for b in nonneg])
        h = ctypes.c_void_p()
        st = stream
        if st is None and any(_is_torch(x) and x.is_cuda for x in keep):
            st = _torch().cuda.current_stream().cuda_stream
        C.check(C.cncpd_create(ctypes.byref(h), self.K, self.N, dims, Xp, code0, Rp, Lp, nn,
                               ctypes.byref(o), ctypes.c_void_p(st) if st else None))
        self._h = h
        self.Rt = None
        # with stream_x the library reads the tensors again (LRA, global fit)
        self._x_keep = keep if stream_x else None

    # -------------------------------------------------------------- state --
    def close(self):
        if getattr(self, "_h", None):
            C.cncpd_destroy(self._h)
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

    def set_factors(self, U):
        """U[k][n]: initial factor of block k, mode n (I_n x R_k), all in
        one call (every factor in the first one's element type)."""
        keep, ptrs, code0 = [], [], None
        for k in range(self.K):
            for n in range(self.N):
                obj, p, code = _prep(U[k][n])
                if code0 is None:
                    code0 = code
                elif code != code0:
                    obj, p, code = _prep(U[k][n], np.float64 if code0 == C.CNCPD_F64 else np.float32)
                keep.append(obj)
                ptrs.append(p.value)
        arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
        C.check(C.cncpd_set_factors_all(self._h, arr, code0))

    def set_cores(self, lams):
        for k, lam in enumerate(lams):
            a = np.ascontiguousarray(np.asarray(lam, dtype=np.float64))
            C.check(C.cncpd_set_core(self._h, k, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    # ------------------------------------------------------------- solver --
    def step(self, n_iters=1):
        s = C.cncpd_stats()
        C.check(C.cncpd_step(self._h, int(n_iters), ctypes.byref(s)))
        return s.as_dict()

    def fit(self):
        s = C.cncpd_stats()
        C.check(C.cncpd_fit(self._h, ctypes.byref(s)))
        return s.as_dict()

    def lra(self, R_tilde, Ut0=None):
        Rt = [int(r) for r in (R_tilde if np.ndim(R_tilde) else [R_tilde] * self.K)]
        keep = []
        ptrs = None
        code = C.CNCPD_F64
        if Ut0 is not None:
            vals = []
            for k in range(self.K):
                for n in range(self.N):
                    obj, p, code = _prep(Ut0[k][n], np.float64)
                    keep.append(obj)
                    vals.append(p.value)
            ptrs = (ctypes.c_void_p * (self.K * self.N))(*vals)
        s = C.cncpd_stats()
        C.check(C.cncpd_lra(self._h, (ctypes.c_int * self.K)(*Rt), ptrs, code, ctypes.byref(s)))
        self.Rt = Rt
        return s.as_dict()

    # ------------------------------------------------------------ outputs --
    def factor(self, k, n, dtype=np.float64, out=None):
        if out is not None:
            obj, p, code = _prep(out)
            C.check(C.cncpd_factors(self._h, k, n, p, code))
            return out
        a = np.empty((self.dims[k][n], self.R[k]), dtype=dtype)
        C.check(C.cncpd_factors(self._h, k, n, ctypes.c_void_p(a.ctypes.data), _dtype_code(a)))
        return a

    def factors(self, dtype=np.float64):
        return [[self.factor(k, n, dtype) for n in range(self.N)] for k in range(self.K)]

    def core(self, k):
        a = np.empty(self.R[k], dtype=np.float64)
        C.check(C.cncpd_core(self._h, k, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return a

    def lra_factor(self, k, n, dtype=np.float64):
        a = np.empty((self.dims[k][n], self.Rt[k]), dtype=dtype)
        C.check(C.cncpd_lra_factors(self._h, k, n, ctypes.c_void_p(a.ctypes.data), _dtype_code(a)))
        return a

    def global_fit(self):
        f = ctypes.c_double()
        C.check(C.cncpd_global_fit(self._h, ctypes.byref(f)))
        return f.value

    def mttkrp(self, k, n, dtype=np.float64):
        a = np.empty((self.dims[k][n], self.R[k]), dtype=dtype)
        C.check(C.cncpd_mttkrp(self._h, k, n, ctypes.c_void_p(a.ctypes.data), _dtype_code(a)))
        return a

    def objective_grad(self, dtype=np.float64, want_grads=True):
        F = ctypes.c_double()
        if not want_grads:
            C.check(C.cncpd_objective_grad(self._h, ctypes.byref(F), None, None, C.CNCPD_F64))
            return F.value, None, None
        gU = [[np.empty((self.dims[k][n], self.R[k]), dtype=dtype) for n in range(self.N)]
              for k in range(self.K)]
        gC = [np.empty((self.dims[0][n], self.L[n]), dtype=dtype) if self.L[n] else None
              for n in range(self.N)]
        pu = (ctypes.c_void_p * (self.K * self.N))(*[gU[k][n].ctypes.data for k in range(self.K)
                                                     for n in range(self.N)])
        pc = (ctypes.c_void_p * self.N)(*[g.ctypes.data if g is not None else None for g in gC])
        C.check(C.cncpd_objective_grad(self._h, ctypes.byref(F), pu, pc,
                                       C.CNCPD_F64 if dtype == np.float64 else C.CNCPD_F32))
        return F.value, gU, gC

    def check_wait_timeout(self, limit_ms=1.0):
        """Run the bounded-wait self-test (cncpd_check_wait_timeout); returns
        the library's status code (CNCPD_ETIMEOUT = -5 is the expected one)."""
        code = C.cncpd_check_wait_timeout(self._h, float(limit_ms))
        return code, C.lib().cncpd_last_error().decode()

    def objective_grad_at(self, U, gU=None, gC=None, dtype=np.float64):
        """F and gradients at the factors U[k][n] (numpy or torch, host or
        device) without touching the solver's state.  gU[k][n] / gC[n]:
        preallocated outputs (numpy or torch, host or device; None entries
        skipped), or None to skip that family."""
        keep, ptrs = [], []
        code = None
        for k in range(self.K):
            for n in range(self.N):
                obj, p, c = _prep(U[k][n], None if code is None else (np.float64 if code == C.CNCPD_F64 else np.float32))
                code = c if code is None else code
                keep.append(obj)
                ptrs.append(p.value)
        Up = (ctypes.c_void_p * (self.K * self.N))(*ptrs)

        def out_ptrs(arrs, count):
            if arrs is None:
                return None
            vals = []
            for a in arrs:
                vals.append(None if a is None else (a.data_ptr() if _is_torch(a) else a.ctypes.data))
            assert len(vals) == count
            return (ctypes.c_void_p * count)(*vals)

        pu = out_ptrs(None if gU is None else [gU[k][n] for k in range(self.K) for n in range(self.N)],
                      self.K * self.N)
        pc = out_ptrs(gC, self.N)
        F = ctypes.c_double()
        C.check(C.cncpd_objective_grad_at(self._h, Up, code, ctypes.byref(F), pu, pc,
                                          C.CNCPD_F64 if dtype in (np.float64, "float64") else C.CNCPD_F32))
        return F.value

    def save_state(self):
        p = ctypes.c_void_p()
        n = ctypes.c_size_t()
        C.check(C.cncpd_save_state(self._h, ctypes.byref(p), ctypes.byref(n)))
        try:
            return ctypes.string_at(p, n.value)
        finally:
            C.cncpd_free_blob(p)

    def load_state(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        C.check(C.cncpd_load_state(self._h, ctypes.cast(buf, ctypes.c_void_p), len(blob)))


def lipschitz(H):
    """Largest eigenvalue of a symmetric PSD matrix as the GPU solver
    computes it (Eqs. eqLipsLd/eqLipsLu)."""
    H = np.ascontiguousarray(np.asarray(H, dtype=np.float64))
    out = ctypes.c_double()
    C.check(C.cncpd_lipschitz(H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), H.shape[0], ctypes.byref(out)))
    return out.value


def _autograd_function():
    torch = _torch()
    if torch is None:  # pragma: no cover
        return None

    class CoupledCPLoss(torch.autograd.Function):
        """F of Eq. costfunc as a differentiable function of the factors.

        ``F = CoupledCPLoss.apply(model, *factors)`` with ``factors`` the
        K*N tensors U^(n,k) (block-major, I_n x R_k).  The value and the
        gradient (Eq. solbpgU) are computed by the library at these factors.
        As in ``set_factors``, the shared first L_n columns come from block
        0: their gradient is the sum over blocks (App. A) and lands on block
        0's columns; the other blocks' copies get zero.  The factors may be
        CPU or CUDA tensors; the gradients are written by the library into
        tensors on the same device, and the model's own iterate and APG
        history are not changed (``cncpd_objective_grad_at``).
        """

        @staticmethod
        def forward(ctx, model, *factors):
            K, N = model.K, model.N
            U = [[factors[k * N + n].detach().contiguous() for n in range(N)] for k in range(K)]
            dt = factors[0].dtype
            if dt not in (torch.float32, torch.float64):
                raise TypeError(f"factors must be float32 or float64, not {dt}")
            # gradients written by the library straight into tensors on the
            # factors' device; the solver state of `model` is left untouched
            gU = [[torch.empty_like(U[k][n]) for n in range(N)] for k in range(K)]
            gC = [torch.empty((model.dims[0][n], model.L[n]), dtype=dt, device=factors[0].device)
                  if model.L[n] else None for n in range(N)]
            F = model.objective_grad_at(U, gU, gC, np.float64 if dt == torch.float64 else np.float32)
            grads = []
            for k in range(K):
                for n in range(N):
                    g = gU[k][n]
                    Ln = model.L[n]
                    if Ln:
                        g[:, :Ln] = gC[n] if k == 0 else 0.0
                    grads.append(g)
            ctx.save_for_backward(*grads)
            return torch.tensor(F, dtype=dt, device=factors[0].device)

        @staticmethod
        def backward(ctx, gF):
            return (None, *[gF * g for g in ctx.saved_tensors])

    return CoupledCPLoss


CoupledCPLoss = _autograd_function()

