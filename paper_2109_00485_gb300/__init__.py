"""GB300-native block LOBPCG for a sparse symmetric matrix stored as one triangle.

Thin ctypes binding over the C ABI declared in ``include/lobpcg.h``: the
functions and methods here only marshal arguments; every step of the
computation runs in the CUDA kernels of ``liblobpcg.so``.  PyTorch supplies
device memory and streams.  There is no CPU fallback: if the library is not
built, importing the binding raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

_lib = None

LOBPCG_OK = 0
STATUS = {
    0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_BREAKDOWN", 5: "ERR_NONFINITE",
    6: "ERR_NOT_CONVERGED", 7: "ERR_TIMEOUT", 8: "ERR_BOUNDS", 9: "ERR_UNSUPPORTED",
}
MEM_DEVICE, MEM_HOST = 0, 1
MLP_NPARAM = 49728      # W1 [256][129] | b1 [256] | W2 [64][256] | b2 [64]
PRECOND = {"none": 0, "diag": 1, "bjacobi": 2, "mlp": 3, "fom": 4}


class LobpcgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Matrix(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("val_is_fp64", ctypes.c_int32),
                ("mem", ctypes.c_int32)]


class _Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("nev", ctypes.c_int32), ("maxiter", ctypes.c_int32),
                ("tol", ctypes.c_double), ("precond", ctypes.c_int32), ("resid_mode", ctypes.c_int32),
                ("polish_fp64", ctypes.c_int32), ("tile_format", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("fom_steps", ctypes.c_int32), ("reserved", ctypes.c_int32), ("fom_tile_ptr", ctypes.c_void_p),
                ("fom_ntiles", ctypes.c_int64)]


class _Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("iters_fp64", ctypes.c_int32), ("used_fp64", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("p_dropped", ctypes.c_int32), ("svqb_used", ctypes.c_int32),
                ("explicit_restarts", ctypes.c_int32), ("spmm_calls", ctypes.c_int32), ("time_ms", ctypes.c_double),
                ("spmm_ms", ctypes.c_double)]


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_blocks", ctypes.c_int64),
                ("chunks", ctypes.c_int64), ("padded_nnz", ctypes.c_int64), ("full_chunks", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("gershgorin", ctypes.c_double), ("num_sms", ctypes.c_int32),
                ("warps", ctypes.c_int32), ("tile_format", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("stream_bytes", ctypes.c_int64)]


def library_path() -> str:
    return _build.SO


def load():
    """Load ``liblobpcg.so``; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.SO):
        raise ImportError(f"{_build.SO} is missing: run __graft_entry__.build() (or python -m "
                          "paper_2109_00485_gb300._build) first; there is no CPU fallback")
    L = ctypes.CDLL(_build.SO)
    vp, i32, st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int
    L.lobpcg_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Matrix), ctypes.POINTER(_Params), vp]
    L.lobpcg_create.restype = st
    L.lobpcg_destroy.argtypes = [vp]
    L.lobpcg_destroy.restype = st
    L.lobpcg_last_error.argtypes = [vp]
    L.lobpcg_last_error.restype = ctypes.c_char_p
    L.lobpcg_matrix_info.argtypes = [vp, ctypes.POINTER(_Info)]
    L.lobpcg_matrix_info.restype = st
    L.lobpcg_sync.argtypes = [vp]
    L.lobpcg_sync.restype = st
    L.lobpcg_spmm_sym.argtypes = [vp, vp, vp, i32]
    L.lobpcg_spmm_sym.restype = st
    L.lobpcg_spmm_sym_f64.argtypes = [vp, vp, vp, i32]
    L.lobpcg_spmm_sym_f64.restype = st
    L.lobpcg_precond_apply.argtypes = [vp, vp, vp, vp, i32, i32]
    L.lobpcg_precond_apply.restype = st
    L.lobpcg_rayleigh_ritz.argtypes = [vp, vp, vp, i32, i32, vp, vp]
    L.lobpcg_rayleigh_ritz.restype = st
    L.lobpcg_rayleigh_ritz_noalloc.argtypes = [vp, vp, vp, i32, i32, vp, vp]
    L.lobpcg_rayleigh_ritz_noalloc.restype = st
    L.lobpcg_test_set_device_ordinal.argtypes = [vp, i32]
    L.lobpcg_test_set_device_ordinal.restype = st
    L.lobpcg_solve.argtypes = [vp, vp, vp, vp, ctypes.POINTER(_Stats)]
    L.lobpcg_solve.restype = st
    L.lobpcg_davidson.argtypes = [vp, vp, i32, vp, vp, ctypes.POINTER(_Stats)]
    L.lobpcg_davidson.restype = st
    L.lobpcg_iterate.argtypes = [vp, vp, i32, vp, ctypes.POINTER(_Stats)]
    L.lobpcg_iterate.restype = st
    L.lobpcg_get_x_f64.argtypes = [vp, vp]
    L.lobpcg_get_x_f64.restype = st
    i64 = ctypes.c_int64
    L.lobpcg_mlp_set_params.argtypes = [vp, vp, i64]
    L.lobpcg_mlp_set_params.restype = st
    L.lobpcg_mlp_get_params.argtypes = [vp, vp, i64, i32]
    L.lobpcg_mlp_get_params.restype = st
    L.lobpcg_mlp_forward.argtypes = [vp, vp, i64, vp]
    L.lobpcg_mlp_forward.restype = st
    L.lobpcg_mlp_grad.argtypes = [vp, vp, vp, i64, vp]
    L.lobpcg_mlp_grad.restype = st
    L.lobpcg_mlp_adam.argtypes = [vp, ctypes.c_float]
    L.lobpcg_mlp_adam.restype = st
    L.lobpcg_precond_train.argtypes = [vp, i32, i64, i32, vp, ctypes.c_float, vp, vp]
    L.lobpcg_precond_train.restype = st
    _lib = L
    return L


def _check(h, status):
    if status != LOBPCG_OK:
        msg = load().lobpcg_last_error(h)
        raise LobpcgError(status, msg.decode() if msg else "")


def _ptr(t) -> int:
    """Data pointer of a torch tensor or numpy array."""
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _dev_block(t, dtype_name: str, n: int, k: int):
    import torch
    want = {"f32": torch.float32, "f64": torch.float64}[dtype_name]
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != want or t.shape != (n, k) or not t.is_contiguous():
        raise ValueError(f"expected a contiguous {want} tensor of shape ({n}, {k}), got {t.dtype} {tuple(t.shape)}")


class Handle:
    """A created lobpcg handle (``lobpcg_create``)."""

    def __init__(self, ptr: int, n: int, params: _Params, stream, keep=()):
        self._h = ctypes.c_void_p(ptr)
        self.n = n
        self.params = params
        self.stream = stream
        self._keep = keep

    # -- C ABI entry points ------------------------------------------------
    def lobpcg_spmm_sym(self, X, Y=None, k: int | None = None):
        """Y = H X (float32, device tensors n x k row-major)."""
        import torch
        k = X.shape[1] if k is None else k
        _dev_block(X, "f32", self.n, k)
        if Y is None:
            Y = torch.empty_like(X)
        _dev_block(Y, "f32", self.n, k)
        _check(self._h, load().lobpcg_spmm_sym(self._h, _ptr(X), _ptr(Y), k))
        return Y

    def spmm_sym_host(self, Xh, Yh):
        """``lobpcg_spmm_sym`` with HOST X and Y (pinned torch CPU tensors or
        numpy arrays, float32 n x k); Y is valid after ``sync()``."""
        for t in (Xh, Yh):
            shape, ok = tuple(t.shape), (t.dtype == np.float32 if isinstance(t, np.ndarray) else str(t.dtype) == "torch.float32")
            if shape[0] != self.n or len(shape) != 2 or not ok:
                raise ValueError("host blocks must be float32 (n, k)")
        k = Xh.shape[1]
        _check(self._h, load().lobpcg_spmm_sym(self._h, _ptr(Xh), _ptr(Yh), k))
        return Yh

    def lobpcg_spmm_sym_f64(self, X, Y=None, k: int | None = None):
        """Y = H X with float64 vectors and accumulation."""
        import torch
        k = X.shape[1] if k is None else k
        _dev_block(X, "f64", self.n, k)
        if Y is None:
            Y = torch.empty_like(X)
        _dev_block(Y, "f64", self.n, k)
        _check(self._h, load().lobpcg_spmm_sym_f64(self._h, _ptr(X), _ptr(Y), k))
        return Y

    def lobpcg_precond_apply(self, R, theta, W=None, mode="diag"):
        """W = K^{-1} R (float32 device n x k); theta: float64 device tensor (k)."""
        import torch
        k = R.shape[1]
        _dev_block(R, "f32", self.n, k)
        if W is None:
            W = torch.empty_like(R)
        _dev_block(W, "f32", self.n, k)
        if not (theta.is_cuda and theta.dtype == torch.float64 and theta.numel() == k and theta.is_contiguous()):
            raise ValueError("theta must be a contiguous CUDA float64 tensor of length k")
        m = PRECOND[mode] if isinstance(mode, str) else int(mode)
        _check(self._h, load().lobpcg_precond_apply(self._h, _ptr(R), _ptr(theta), _ptr(W), k, m))
        return W

    def lobpcg_rayleigh_ritz(self, S, HS, k: int):
        """(C, theta) of the k leftmost Ritz pairs in span(S): S, HS float32
        device n x m; returns float64 device tensors C (m x k), theta (k)."""
        import torch
        m = S.shape[1]
        _dev_block(S, "f32", self.n, m)
        _dev_block(HS, "f32", self.n, m)
        C = torch.empty((m, k), dtype=torch.float64, device=S.device)
        th = torch.empty((k,), dtype=torch.float64, device=S.device)
        _check(self._h, load().lobpcg_rayleigh_ritz(self._h, _ptr(S), _ptr(HS), m, k, _ptr(C), _ptr(th)))
        return C, th

    def lobpcg_rayleigh_ritz_noalloc(self, S, HS, k: int, C, theta):
        """``lobpcg_rayleigh_ritz`` into caller-provided C (float64 device
        m x k) and theta (float64 device k); the library allocates nothing."""
        import torch
        m = S.shape[1]
        _dev_block(S, "f32", self.n, m)
        _dev_block(HS, "f32", self.n, m)
        for t, shape in ((C, (m, k)), (theta, (k,))):
            if not (t.is_cuda and t.dtype == torch.float64 and tuple(t.shape) == shape and t.is_contiguous()):
                raise ValueError(f"expected a contiguous CUDA float64 tensor of shape {shape}")
        _check(self._h, load().lobpcg_rayleigh_ritz_noalloc(self._h, _ptr(S), _ptr(HS), m, k, _ptr(C), _ptr(theta)))
        return C, theta

    def lobpcg_solve(self, X0):
        """Run LOBPCG from X0 (float32 n x k: CUDA tensor, or host numpy / CPU
        tensor).  Returns (X, evals, resid, stats) with X of the same kind;
        raises LobpcgError on failure (NOT_CONVERGED carries .result)."""
        return self._run(X0, lambda X, ev, rs, stats: load().lobpcg_solve(
            self._h, _ptr(X), ev.ctypes.data, rs.ctypes.data, ctypes.byref(stats)))

    def lobpcg_davidson(self, X0, max_blocks: int = 0):
        """Block Davidson from X0 on the same SpMM and preconditioner (basis
        of at most max_blocks blocks of k columns; 0: min(6, 96 // k)).
        Returns and raises as lobpcg_solve."""
        mb = int(max_blocks) if max_blocks else min(6, 96 // self.params.k)
        return self._run(X0, lambda X, ev, rs, stats: load().lobpcg_davidson(
            self._h, _ptr(X), mb, ev.ctypes.data, rs.ctypes.data, ctypes.byref(stats)))

    def _run(self, X0, call):
        k = self.params.k
        nev = self.params.nev
        if isinstance(X0, np.ndarray):
            X = np.ascontiguousarray(X0, dtype=np.float32).copy()
            if X.shape != (self.n, k):
                raise ValueError(f"X0 must be ({self.n}, {k})")
        else:
            import torch
            if X0.is_cuda and self.stream is not None:
                # the copy on the handle's stream, after the caller's stream
                # has produced X0
                self.stream.wait_stream(torch.cuda.current_stream(X0.device))
                with torch.cuda.stream(self.stream):
                    X = X0.detach().clone().contiguous()
            else:
                X = X0.detach().clone().contiguous()
            if tuple(X.shape) != (self.n, k) or str(X.dtype) != "torch.float32":
                raise ValueError(f"X0 must be float32 ({self.n}, {k})")
        ev = np.zeros(nev)
        rs = np.zeros(nev)
        stats = _Stats()
        status = call(X, ev, rs, stats)
        result = (X, ev, rs, {f: getattr(stats, f) for f, _ in _Stats._fields_})
        if status != LOBPCG_OK:
            err = LobpcgError(status, self.lobpcg_last_error())
            err.result = result
            raise err
        return result

    def lobpcg_iterate(self, steps: int, X0=None):
        """Run `steps` float32 iterations (X0 starts a new run; None
        continues).  Returns (theta, stats)."""
        th = np.zeros(self.params.k)
        stats = _Stats()
        _check(self._h, load().lobpcg_iterate(self._h, _ptr(X0) if X0 is not None else None, int(steps),
                                              th.ctypes.data, ctypes.byref(stats)))
        return th, {f: getattr(stats, f) for f, _ in _Stats._fields_}

    def lobpcg_get_x_f64(self, out=None):
        import torch
        k = self.params.k
        if out is None:
            out = torch.empty((self.n, k), dtype=torch.float64, device="cuda")
        _check(self._h, load().lobpcg_get_x_f64(self._h, _ptr(out)))
        return out

    def lobpcg_sync(self):
        _check(self._h, load().lobpcg_sync(self._h))

    # -- learned tile preconditioner (mode 3) --------------------------------
    def lobpcg_mlp_set_params(self, params):
        """Load weights: float32 vector of MLP_NPARAM (numpy or CUDA tensor)."""
        if isinstance(params, np.ndarray):
            params = np.ascontiguousarray(params, dtype=np.float32)
        _check(self._h, load().lobpcg_mlp_set_params(self._h, _ptr(params), int(params.size if isinstance(
            params, np.ndarray) else params.numel())))

    def lobpcg_mlp_get_params(self, which: str = "weights") -> np.ndarray:
        """Weights (or 'grads', the gradients of the last batch) as float32 numpy."""
        out = np.zeros(MLP_NPARAM, dtype=np.float32)
        _check(self._h, load().lobpcg_mlp_get_params(self._h, out.ctypes.data, MLP_NPARAM,
                                                     {"weights": 0, "grads": 1}[which]))
        return out

    def lobpcg_mlp_forward(self, Xin, Y=None):
        """Y (B x 64) = network(Xin (B x 129)), float32 CUDA tensors."""
        import torch
        B = Xin.shape[0]
        if tuple(Xin.shape) != (B, 129) or Xin.dtype != torch.float32 or not Xin.is_cuda or not Xin.is_contiguous():
            raise ValueError("Xin must be a contiguous CUDA float32 (B, 129) tensor")
        if Y is None:
            Y = torch.empty((B, 64), dtype=torch.float32, device=Xin.device)
        _check(self._h, load().lobpcg_mlp_forward(self._h, _ptr(Xin), B, _ptr(Y)))
        return Y

    def lobpcg_mlp_grad(self, Xin, T) -> float:
        """Batch MSE loss of Xin (B x 129) against T (B x 64); gradients kept
        on the handle (``mlp_get_params('grads')``)."""
        B = Xin.shape[0]
        if tuple(T.shape) != (B, 64) or tuple(Xin.shape) != (B, 129):
            raise ValueError("Xin must be (B, 129) and T (B, 64)")
        loss = ctypes.c_double(0.0)
        _check(self._h, load().lobpcg_mlp_grad(self._h, _ptr(Xin), _ptr(T), B, ctypes.addressof(loss)))
        return loss.value

    def lobpcg_mlp_adam(self, lr: float = 1e-3):
        _check(self._h, load().lobpcg_mlp_adam(self._h, float(lr)))

    def lobpcg_precond_train(self, X0, harvest_iters: int = 20, n_pairs: int = 1 << 20, epochs: int = 5,
                             lr: float = 1e-3):
        """Harvest (residual, exact tile solve) pairs from block-Jacobi
        iterations from X0, then train the network.  Returns (held-out loss
        before training and after each epoch, pairs used)."""
        if isinstance(X0, np.ndarray):
            X0 = np.ascontiguousarray(X0, dtype=np.float32)
        hist = np.zeros(epochs + 1)
        used = ctypes.c_int64(0)
        _check(self._h, load().lobpcg_precond_train(self._h, int(harvest_iters), int(n_pairs), int(epochs),
                                                    _ptr(X0), float(lr), hist.ctypes.data, ctypes.addressof(used)))
        return hist, used.value

    def lobpcg_matrix_info(self) -> dict:
        info = _Info()
        _check(self._h, load().lobpcg_matrix_info(self._h, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in _Info._fields_}

    def lobpcg_last_error(self) -> str:
        msg = load().lobpcg_last_error(self._h)
        return msg.decode() if msg else ""

    def lobpcg_destroy(self):
        if self._h:
            load().lobpcg_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def lobpcg_test_set_device_ordinal(self, device: int):
        """Test hook: overwrite the device ordinal recorded in the handle."""
        _check(self._h, load().lobpcg_test_set_device_ordinal(self._h, int(device)))

    # -- conveniences with the same meaning ---------------------------------
    spmm_sym = lobpcg_spmm_sym
    spmm_sym_f64 = lobpcg_spmm_sym_f64
    precond_apply = lobpcg_precond_apply
    rayleigh_ritz = lobpcg_rayleigh_ritz
    rayleigh_ritz_noalloc = lobpcg_rayleigh_ritz_noalloc
    solve = lobpcg_solve
    davidson = lobpcg_davidson
    iterate = lobpcg_iterate
    get_x_f64 = lobpcg_get_x_f64
    sync = lobpcg_sync
    mlp_set_params = lobpcg_mlp_set_params
    mlp_get_params = lobpcg_mlp_get_params
    mlp_forward = lobpcg_mlp_forward
    mlp_grad = lobpcg_mlp_grad
    mlp_adam = lobpcg_mlp_adam
    precond_train = lobpcg_precond_train
    info = lobpcg_matrix_info
    destroy = lobpcg_destroy

    def __del__(self):
        try:
            self.lobpcg_destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.lobpcg_destroy()


def lobpcg_last_error() -> str:
    """Text of the last failed ``lobpcg_create`` on this thread."""
    msg = load().lobpcg_last_error(None)
    return msg.decode() if msg else ""


def make_params(k: int, nev: int | None = None, maxiter: int = 1000, tol: float = 1e-6, precond="diag",
                resid_mode: int = 0, polish_fp64: int = 1, seed: int = 0, tile_format: int = 0,
                fom_steps: int = 0, fom_tile_ptr=None) -> _Params:
    p = _Params()
    p.k = k
    p.nev = k if nev is None else nev
    p.maxiter = maxiter
    p.tol = tol
    p.precond = PRECOND[precond] if isinstance(precond, str) else int(precond)
    p.resid_mode = resid_mode
    p.polish_fp64 = polish_fp64
    p.tile_format = tile_format
    p.seed = seed & (2 ** 64 - 1)
    p.fom_steps = fom_steps
    if fom_tile_ptr is not None:
        tp = np.ascontiguousarray(fom_tile_ptr, dtype=np.int64)
        p._keep = tp                       # the array must outlive the create call
        p.fom_tile_ptr = tp.ctypes.data
        p.fom_ntiles = tp.size - 1
    return p


def lobpcg_create(n: int, row_ptr, col, val, params: _Params | None = None, stream=None, **kw) -> Handle:
    """Create a handle from a lower-triangle CSR.

    ``row_ptr`` (int64[n+1]), ``col`` (int32[nnz]) and ``val`` (float32 or
    float64[nnz]) are either all numpy arrays (host) or all CUDA tensors.
    ``stream`` is a ``torch.cuda.Stream`` (default: the current stream)."""
    import torch
    L = load()
    if params is None:
        params = make_params(**kw)
    m = _Matrix()
    m.n = int(n)
    if isinstance(row_ptr, np.ndarray):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        if val.dtype not in (np.float32, np.float64):
            raise TypeError("val must be float32 or float64")
        val = np.ascontiguousarray(val)
        m.mem = MEM_HOST
        m.val_is_fp64 = 1 if val.dtype == np.float64 else 0
        m.nnz = int(col.size)
    else:
        for t, dt in ((row_ptr, torch.int64), (col, torch.int32)):
            if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
                raise TypeError("device CSR: row_ptr int64, col int32, contiguous CUDA tensors")
        if val.dtype not in (torch.float32, torch.float64) or not val.is_cuda or not val.is_contiguous():
            raise TypeError("val must be a contiguous CUDA float32/float64 tensor")
        m.mem = MEM_DEVICE
        m.val_is_fp64 = 1 if val.dtype == torch.float64 else 0
        m.nnz = int(col.numel())
    m.row_ptr, m.col, m.val = _ptr(row_ptr), _ptr(col), _ptr(val)
    if stream is None and torch.cuda.is_available():
        stream = torch.cuda.current_stream()
    sh = stream.cuda_stream if stream is not None else 0
    out = ctypes.c_void_p(0)
    st = L.lobpcg_create(ctypes.byref(out), ctypes.byref(m), ctypes.byref(params), ctypes.c_void_p(sh))
    if st != LOBPCG_OK:
        msg = L.lobpcg_last_error(None)
        raise LobpcgError(st, msg.decode() if msg else "")
    return Handle(out.value, int(n), params, stream)


def from_csr(A, params: _Params | None = None, stream=None, **kw) -> Handle:
    """``lobpcg_create`` from an object with ``n, row_ptr, col, val`` (host arrays)."""
    return lobpcg_create(A.n, A.row_ptr, A.col, A.val, params=params, stream=stream, **kw)
