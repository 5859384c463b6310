"""Python binding of libmera (ctypes; argument marshalling only).

Every computation runs in the CUDA library; this module converts arrays to
pointers and back.  Arrays may be NumPy arrays (host memory) or torch
tensors (host or CUDA); outputs are NumPy arrays unless ``device=True``, in
which case they are CUDA torch tensors.  If the compiled library is missing
the import fails: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmera.so")

MERA_F64, MERA_C128 = 0, 1
MERA_BINARY, MERA_TERNARY, MERA_MPS = 0, 1, 2
PREC_FP64, PREC_3XTF32, PREC_SPLIT_BF16, PREC_SPLIT_FP16 = 0, 1, 2, 3

ERRORS = {
    -1: "MERA_ERR_ARG", -2: "MERA_ERR_OOM", -3: "MERA_ERR_NONFINITE", -4: "MERA_ERR_NOCONV",
    -5: "MERA_ERR_DEVICE_TIMEOUT", -6: "MERA_ERR_NOT_ISOMETRIC", -7: "MERA_ERR_CUDA",
    -8: "MERA_ERR_UNSUPPORTED",
}


class MeraError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("d_b", C.c_int), ("chi", C.c_int), ("n_trans", C.c_int), ("dtype", C.c_int),
                ("prec", C.c_int), ("w_stiefel", C.c_int), ("precond", C.c_int),
                ("krylov_dim", C.c_int), ("krylov_maxiter", C.c_int), ("krylov_tol", C.c_double),
                ("recompute_env", C.c_int), ("lbfgs_m", C.c_int), ("b_chunk", C.c_int), ("network", C.c_int),
                ("z2", C.c_int), ("device_wait_s", C.c_double)]


class IterInfo(C.Structure):
    _fields_ = [("iter", C.c_int), ("energy", C.c_double), ("gnorm", C.c_double),
                ("alpha", C.c_double), ("n_evals", C.c_int), ("ls_ok", C.c_int),
                ("krylov_matvecs", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("gett_launches", C.c_int64), ("gett_flops", C.c_double),
                ("gett_timed", C.c_int64), ("gett_ms", C.c_double),
                ("energy_grad_calls", C.c_int64), ("krylov_matvecs", C.c_int64)]


class RequestStatus(C.Structure):
    _fields_ = [("state", C.c_int), ("error", C.c_int), ("iters", C.c_int), ("n_evals", C.c_int),
                ("energy", C.c_double), ("gnorm", C.c_double), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("bytes", C.c_size_t),
                ("message", C.c_char * 160), ("deferred", C.c_int), ("batched_evals", C.c_int)]


# device allocator callbacks of mera_set_allocator
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_allocator_refs = None  # the installed callbacks, kept alive while installed


def set_allocator(alloc=None, free=None):
    """Route every device buffer the library allocates through alloc(nbytes)
    -> int device pointer (0 when it cannot) and free(ptr) (see
    mera_set_allocator in mera.h); set_allocator() restores cudaMalloc.
    The callbacks run on whichever thread allocates, with the GIL taken."""
    global _allocator_refs
    L = load()
    if alloc is None:
        rc = L.mera_set_allocator(C.cast(None, ALLOC_FN), C.cast(None, FREE_FN), None)
        _allocator_refs = None
    else:
        a = ALLOC_FN(lambda n, user: alloc(int(n)) or None)
        f = FREE_FN(lambda p, user: free(int(p)))
        rc = L.mera_set_allocator(a, f, None)
        _allocator_refs = (a, f)
    if rc != 0:
        raise MeraError(rc, L.mera_strerror(rc).decode())


def use_torch_allocator():
    """Route the library's device memory through PyTorch's caching allocator
    on the current device (its memory then shows in torch.cuda's statistics
    and is reused across objects)."""
    import torch
    dev = torch.cuda.current_device()

    def alloc(n):
        try:
            return torch.cuda.caching_allocator_alloc(n, device=dev)
        except RuntimeError:  # out of memory: the library reports MERA_ERR_OOM
            return 0
    set_allocator(alloc, lambda p: torch.cuda.caching_allocator_delete(p))


class SolveOpts(C.Structure):
    _fields_ = [("method", C.c_int), ("maxiter", C.c_int), ("gtol", C.c_double)]


class SolveResult(C.Structure):
    _fields_ = [("iters", C.c_int), ("n_evals", C.c_int), ("energy", C.c_double),
                ("gnorm", C.c_double), ("converged", C.c_int)]


EXPORTS = ["mera_config_default", "mera_create", "mera_destroy", "mera_num_tensors", "mera_energy",
           "mera_tensor_shape", "mera_set_tensors", "mera_get_tensors", "mera_init_random", "mera_energy_grad",
           "mera_project", "mera_inner", "mera_transport", "mera_retract", "mera_precondition",
           "mera_lbfgs_step", "mera_cg_step", "mera_gd_step", "mera_ev_sweep", "mera_solve", "mera_footprint_bytes",
           "mera_launch_count", "mera_get_stats", "mera_profile", "mera_profile_dump", "mera_dots_noalloc",
           "mera_gemm", "mera_strerror", "mera_last_error", "mera_server_create", "mera_set_device_wait",
           "mera_set_allocator", "mera_reset_warm_starts",
           "mera_server_submit", "mera_server_poll", "mera_server_wait", "mera_server_destroy"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libmera.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmera.so not built ({path}); run paper_2007_03638_gb300.build.build()")
    L = C.CDLL(path)
    vpp = C.POINTER(C.c_void_p)
    sig = {
        "mera_config_default": (None, [C.POINTER(Config), C.c_int, C.c_int, C.c_int]),
        "mera_create": (C.c_int, [C.POINTER(Config), C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
        "mera_destroy": (C.c_int, [C.c_void_p]),
        "mera_num_tensors": (C.c_int, [C.c_void_p]),
        "mera_tensor_shape": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "mera_set_tensors": (C.c_int, [C.c_void_p, vpp]),
        "mera_get_tensors": (C.c_int, [C.c_void_p, vpp]),
        "mera_init_random": (C.c_int, [C.c_void_p, C.c_uint64]),
        "mera_energy_grad": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), vpp, vpp]),
        "mera_energy": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
        "mera_project": (C.c_int, [C.c_void_p, vpp, vpp]),
        "mera_inner": (C.c_int, [C.c_void_p, vpp, vpp, C.POINTER(C.c_double)]),
        "mera_transport": (C.c_int, [C.c_void_p, vpp, C.c_double, vpp]),
        "mera_retract": (C.c_int, [C.c_void_p, vpp, C.c_double, vpp]),
        "mera_precondition": (C.c_int, [C.c_void_p, vpp, vpp]),
        "mera_lbfgs_step": (C.c_int, [C.c_void_p, C.POINTER(IterInfo)]),
        "mera_cg_step": (C.c_int, [C.c_void_p, C.POINTER(IterInfo)]),
        "mera_gd_step": (C.c_int, [C.c_void_p, C.POINTER(IterInfo)]),
        "mera_ev_sweep": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(IterInfo)]),
        "mera_solve": (C.c_int, [C.c_void_p, C.POINTER(SolveOpts), C.POINTER(SolveResult)]),
        "mera_footprint_bytes": (C.c_size_t, [C.POINTER(Config)]),
        "mera_launch_count": (C.c_int64, [C.c_void_p]),
        "mera_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats), C.c_int]),
        "mera_profile": (C.c_int, [C.c_void_p, C.c_int]),
        "mera_profile_dump": (C.c_int, [C.c_void_p, C.c_char_p]),
        "mera_dots_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64,
                                        C.c_void_p, C.c_void_p]),
        "mera_gemm": (C.c_int, [C.c_int, C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p]),
        "mera_server_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(C.c_void_p)]),
        "mera_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Config), C.c_void_p, vpp, C.c_int,
                                         C.c_double, C.c_int, C.POINTER(C.c_int64)]),
        "mera_server_poll": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(RequestStatus)]),
        "mera_server_wait": (C.c_int, [C.c_void_p, C.c_double]),
        "mera_server_destroy": (C.c_int, [C.c_void_p]),
        "mera_set_device_wait": (C.c_int, [C.c_void_p, C.c_double]),
        "mera_reset_warm_starts": (C.c_int, [C.c_void_p]),
        "mera_set_allocator": (C.c_int, [ALLOC_FN, FREE_FN, C.c_void_p]),
        "mera_strerror": (C.c_char_p, [C.c_int]),
        "mera_last_error": (C.c_char_p, [C.c_void_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def default_config(d_b, chi, n_trans, **kw) -> Config:
    L = load()
    cfg = Config()
    L.mera_config_default(C.byref(cfg), d_b, chi, n_trans)
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def footprint_bytes(cfg: Config) -> int:
    return int(load().mera_footprint_bytes(C.byref(cfg)))


def dots_noalloc(X, y, k, n, ldx, out, stream=0):
    """Allocation-free batched dot products (see mera_dots_noalloc in mera.h):
    X, y float64 device arrays (torch CUDA tensors, or raw pointers whose
    sizes the caller vouches for), out: host or device float64 array of at
    least k elements.  Raises ValueError when an array is too short and
    MeraError on a size the library rejects."""
    L = load()
    k, n, ldx = int(k), int(n), int(ldx)
    if k >= 1 and n >= 0:
        need_x = (k - 1) * ldx + n if k > 1 else n
        for name, a, need in (("X", X, need_x), ("y", y, n), ("out", out, k)):
            size = None if isinstance(a, int) else (a.numel() if hasattr(a, "numel") else a.size)
            if size is not None and size < need:
                raise ValueError(f"dots_noalloc: {name} holds {size} elements, needs {need}")
    xp = X if isinstance(X, int) else _ptr(X, np.float64)
    yp = y if isinstance(y, int) else _ptr(y, np.float64)
    rc = L.mera_dots_noalloc(C.c_void_p(xp), ldx, k, C.c_void_p(yp), n,
                             C.c_void_p(_ptr(out, np.float64)), C.c_void_p(stream))
    if rc != 0:
        raise MeraError(rc, L.mera_strerror(rc).decode())
    return out


def gemm(prec, A, B, out, stream=0):
    """out = A B (device float64 row-major tensors) in the arithmetic of ``prec``.
    A is M x K and B K x N; out holds M N elements (ValueError otherwise: the
    library reads and writes exactly those extents)."""
    L = load()
    if len(A.shape) != 2 or len(B.shape) != 2:
        raise ValueError("gemm: A and B must be matrices")
    M, K = A.shape
    if B.shape[0] != K:
        raise ValueError(f"gemm: B has {B.shape[0]} rows, A has {K} columns")
    N = B.shape[1]
    if _numel(out) != M * N:
        raise ValueError(f"gemm: out holds {_numel(out)} elements, the product has {M * N}")
    rc = L.mera_gemm(int(prec), M, N, K, C.c_void_p(_ptr(A, np.float64)), C.c_void_p(_ptr(B, np.float64)),
                     C.c_void_p(_ptr(out, np.float64)), C.c_void_p(stream))
    if rc != 0:
        raise MeraError(rc, L.mera_strerror(rc).decode())
    return out


def C_void(a):
    return C.c_void_p(_ptr(a))


def _ptr(a, dtype=None):
    """Data pointer of a contiguous numpy array or torch tensor of float64
    (or complex128) elements; ``dtype`` (a numpy dtype) pins the type."""
    ok = (np.dtype(np.float64), np.dtype(np.complex128)) if dtype is None else (np.dtype(dtype),)
    if isinstance(a, np.ndarray):
        if a.dtype not in ok or not a.flags.c_contiguous:
            raise TypeError(f"expected a C-contiguous {' or '.join(map(str, ok))} array")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        tmap = {torch.float64: np.dtype(np.float64), torch.complex128: np.dtype(np.complex128)}
        if tmap.get(a.dtype) not in ok or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {' or '.join(map(str, ok))} tensor")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _numel(a):
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _ptrs(arrs, keep, dtype=np.float64, sizes=None):
    """ctypes array of the arrays' data pointers.  With ``sizes`` (elements
    per array) the list must hold exactly that many arrays of those sizes:
    the library reads and writes that many elements behind each pointer."""
    if sizes is not None:
        if len(arrs) != len(sizes):
            raise ValueError(f"expected {len(sizes)} tensors, got {len(arrs)}")
        for i, (a, n) in enumerate(zip(arrs, sizes)):
            if _numel(a) != n:
                raise ValueError(f"tensor {i} has {_numel(a)} elements, expected {n}")
    out = (C.c_void_p * len(arrs))()
    for i, a in enumerate(arrs):
        if isinstance(a, np.ndarray) and (a.dtype != dtype or not a.flags.c_contiguous):
            a = np.ascontiguousarray(a, dtype=dtype)
        keep.append(a)
        out[i] = _ptr(a, dtype)
    return out


class Mera:
    """One optimisation problem (a ``mera_t``) bound to a CUDA stream."""

    def __init__(self, cfg: Config, h3, stream=None):
        self.L = load()
        self.cfg = cfg
        self.dtype = np.dtype(np.complex128 if cfg.dtype == MERA_C128 else np.float64)
        h = np.ascontiguousarray(h3, dtype=self.dtype) if isinstance(h3, np.ndarray) else h3
        n_op = int(cfg.d_b) ** (6 if cfg.network == MERA_BINARY else 4)  # three- or two-site term
        if _numel(h) != n_op:
            raise ValueError(f"the Hamiltonian term has {_numel(h)} elements, expected {n_op}")
        handle = C.c_void_p()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except ImportError:
                stream = 0
        rc = self.L.mera_create(C.byref(cfg), C.c_void_p(_ptr(h, self.dtype)), C.c_void_p(stream),
                                C.byref(handle))
        if rc != 0:
            raise MeraError(rc, self.L.mera_strerror(rc).decode())
        self.h = handle
        self.n = self.L.mera_num_tensors(self.h)
        self.shapes = []
        for i in range(self.n):
            r, c = C.c_int64(), C.c_int64()
            self.L.mera_tensor_shape(self.h, i, C.byref(r), C.byref(c))
            self.shapes.append((r.value, c.value))
        self.sizes = [r * c for r, c in self.shapes]

    def _check(self, rc):
        if rc != 0:
            raise MeraError(rc, self.L.mera_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.mera_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _alloc(self, device):
        if device:
            import torch
            tdt = torch.complex128 if self.dtype == np.complex128 else torch.float64
            return [torch.empty(s, dtype=tdt, device="cuda") for s in self.shapes]
        return [np.empty(s, dtype=self.dtype) for s in self.shapes]

    # ---- C ABI mirrors ------------------------------------------------------
    def set_tensors(self, tensors):
        keep = []
        self._check(self.L.mera_set_tensors(self.h, _ptrs(tensors, keep, self.dtype, self.sizes)))

    def init_random(self, seed):
        """Seeded sign-fixed QR-of-Gaussian point (see mera_init_random in mera.h)."""
        self._check(self.L.mera_init_random(self.h, int(seed)))

    def get_tensors(self, device=False):
        out = self._alloc(device)
        keep = []
        self._check(self.L.mera_get_tensors(self.h, _ptrs(out, keep, self.dtype, self.sizes)))
        return out

    def energy_grad(self, device=False, deriv=False):
        e = C.c_double()
        G = self._alloc(device)
        keep = []
        D = self._alloc(device) if deriv else None
        self._check(self.L.mera_energy_grad(self.h, C.byref(e), _ptrs(G, keep, self.dtype, self.sizes),
                                            _ptrs(D, keep, self.dtype, self.sizes) if deriv else None))
        return (e.value, G, D) if deriv else (e.value, G)

    def reset_warm_starts(self):
        """Next evaluation starts its Krylov solves afresh (mera_reset_warm_starts)."""
        self._check(self.L.mera_reset_warm_starts(self.h))

    def set_device_wait(self, seconds):
        """Limit of each tensor-core pipeline wait (mera_set_device_wait)."""
        self._check(self.L.mera_set_device_wait(self.h, float(seconds)))

    def energy_grad_into(self, G):
        """Energy, with the gradient written into the given arrays (host or device)."""
        e = C.c_double()
        keep = []
        self._check(self.L.mera_energy_grad(self.h, C.byref(e), _ptrs(G, keep, self.dtype, self.sizes), None))
        return e.value

    def energy(self):
        """Energy and gradient at the current point; returns the energy."""
        e = C.c_double()
        self._check(self.L.mera_energy_grad(self.h, C.byref(e), None, None))
        return e.value

    def energy_only(self):
        """Energy alone (no environments)."""
        e = C.c_double()
        self._check(self.L.mera_energy(self.h, C.byref(e)))
        return e.value

    def project(self, D, device=False):
        G = self._alloc(device)
        keep = []
        self._check(self.L.mera_project(self.h, _ptrs(D, keep, self.dtype, self.sizes), _ptrs(G, keep, self.dtype, self.sizes)))
        return G

    def inner(self, X, Y):
        out = C.c_double()
        keep = []
        self._check(self.L.mera_inner(self.h, _ptrs(X, keep, self.dtype, self.sizes), _ptrs(Y, keep, self.dtype, self.sizes),
                                      C.byref(out)))
        return out.value

    def transport(self, X, alpha, Y):
        keep = []
        Yc = [np.array(y, dtype=self.dtype, copy=True) if isinstance(y, np.ndarray) else y.clone() for y in Y]
        self._check(self.L.mera_transport(self.h, _ptrs(X, keep, self.dtype, self.sizes), float(alpha),
                                          _ptrs(Yc, keep, self.dtype, self.sizes)))
        return Yc

    def retract(self, X, alpha, want_xprime=False):
        keep = []
        Xp = self._alloc(False) if want_xprime else None
        self._check(self.L.mera_retract(self.h, _ptrs(X, keep, self.dtype, self.sizes), float(alpha),
                                        _ptrs(Xp, keep, self.dtype, self.sizes) if want_xprime else None))
        return Xp

    def precondition(self, X):
        keep = []
        out = self._alloc(False)
        self._check(self.L.mera_precondition(self.h, _ptrs(X, keep, self.dtype, self.sizes),
                                             _ptrs(out, keep, self.dtype, self.sizes)))
        return out

    def lbfgs_step(self):
        info = IterInfo()
        self._check(self.L.mera_lbfgs_step(self.h, C.byref(info)))
        return {f: getattr(info, f) for f, _ in IterInfo._fields_}

    def cg_step(self):
        info = IterInfo()
        self._check(self.L.mera_cg_step(self.h, C.byref(info)))
        return {f: getattr(info, f) for f, _ in IterInfo._fields_}

    def gd_step(self):
        """One Riemannian gradient-descent iteration (negative preconditioned gradient)."""
        info = IterInfo()
        self._check(self.L.mera_gd_step(self.h, C.byref(info)))
        return {f: getattr(info, f) for f, _ in IterInfo._fields_}

    def ev_sweep(self, gamma):
        """One Evenbly-Vidal sweep with the Hamiltonian shifted by -gamma."""
        info = IterInfo()
        self._check(self.L.mera_ev_sweep(self.h, float(gamma), C.byref(info)))
        return {f: getattr(info, f) for f, _ in IterInfo._fields_}

    def solve(self, maxiter=100, gtol=1e-6, method=0):
        o = SolveOpts(method, maxiter, gtol)
        r = SolveResult()
        self._check(self.L.mera_solve(self.h, C.byref(o), C.byref(r)))
        return {f: getattr(r, f) for f, _ in SolveResult._fields_}

    def launch_count(self):
        return int(self.L.mera_launch_count(self.h))

    def stats(self, reset=False):
        st = Stats()
        self._check(self.L.mera_get_stats(self.h, C.byref(st), int(reset)))
        return {f: getattr(st, f) for f, _ in Stats._fields_}

    def profile(self, enable=True):
        self._check(self.L.mera_profile(self.h, int(enable)))

    def profile_dump(self, path):
        """Per-shape table of the contractions timed while profiling (CSV)."""
        self._check(self.L.mera_profile_dump(self.h, str(path).encode()))
