"""ctypes binding of libpase.so (include/pase.h): argument marshalling only.

Array arguments may be numpy arrays (host memory), CPU torch tensors, or CUDA torch
tensors (device memory); they must be C-contiguous float64 (int64/int32 for CSR index
arrays).  Multivectors are row-major [N][m].
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpase.so")

PASE_OK = 0
PASE_ERR_NAN = -5
PASE_ERR_NOT_CONVERGED = -6
PASE_ERR_TIMEOUT = -7
PASE_PREC_FP64 = 0
PASE_PREC_MIXED = 1
PASE_SOLVER_VCYCLE = 0
PASE_SOLVER_CG = 1
PASE_SOLVER_MGCG = 2
PASE_SMOOTHER_JACOBI = 0
PASE_SMOOTHER_LEARNED = 1
PASE_AUG_PLAIN = 0
PASE_AUG_PRECOND_A = 1
PASE_AUG_PRECOND_B = 2
PASE_AUG_PRECOND_BA = 3


class PaseCSR(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("on_device", ctypes.c_int)]


class PaseOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("linear_solver", ctypes.c_int),
                ("inner_steps", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("omega", ctypes.c_double), ("coarse_level", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("aug_max_iter", ctypes.c_int),
                ("aug_tol", ctypes.c_double), ("aug_adaptive", ctypes.c_int),
                ("verbose", ctypes.c_int), ("use_graphs", ctypes.c_int), ("autotune", ctypes.c_int),
                ("smoother", ctypes.c_int), ("split_gemm", ctypes.c_int), ("stencil", ctypes.c_int),
                ("post_solve", ctypes.c_int), ("aug_transform", ctypes.c_int), ("spmm_df64", ctypes.c_int),
                ("graph_solve", ctypes.c_int), ("graph_pass_limit", ctypes.c_int),
                ("stencil_columns", ctypes.c_int), ("aug_factor", ctypes.c_double),
                ("sygv_tridiag", ctypes.c_int), ("sygv_cholesky", ctypes.c_int)]


class PaseTrainOptions(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("seed", ctypes.c_uint),
                ("max_cycles", ctypes.c_int)]


class PaseStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("max_residual", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("phase_ms", ctypes.c_double * 5), ("aug_iterations", ctypes.c_int),
                ("kernel_launches", ctypes.c_int), ("graph_launches", ctypes.c_int)]

    def as_dict(self):
        return {"iterations": self.iterations, "converged": self.converged,
                "max_residual": self.max_residual, "solve_ms": self.solve_ms,
                "phase_ms": list(self.phase_ms), "aug_iterations": self.aug_iterations,
                "kernel_launches": self.kernel_launches, "graph_launches": self.graph_launches}


class PaseError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pase error {code}: {msg}")
        self.code = code


_lib = None

EXPORTED = ["pase_default_options", "pase_create", "pase_setup", "pase_reserve", "pase_solve", "pase_solve_batches",
            "pase_solve_batched", "pase_profile_kernel", "pase_profile_read",
            "pase_residual", "pase_linear_solve", "pase_project", "pase_augmented_eig",
            "pase_prolongate", "pase_iterate", "pase_spmm_am", "pase_smooth", "pase_smoother_form",
            "pase_residual_noalloc",
            "pase_time_kernel", "pase_set_grid", "pase_smoother_nparams", "pase_smoother_state",
            "pase_smoother_apply", "pase_smoother_step", "pase_default_train_options",
            "pase_train_smoother",
            "pase_kernel_count", "pase_launch_counts",
            "pase_destroy", "pase_status_string", "pase_last_error"]


def load_library(path=LIB_PATH):
    """Load libpase.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(python paper_2502_04589_gb300/build.py); no CPU fallback exists")
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.pase_default_options.argtypes = [ctypes.POINTER(PaseOptions)]
    L.pase_default_options.restype = None
    L.pase_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(PaseOptions), vp]
    L.pase_setup.argtypes = [vp, ctypes.POINTER(PaseCSR), ctypes.POINTER(PaseCSR), i32,
                             ctypes.POINTER(PaseCSR), ctypes.POINTER(PaseCSR), ctypes.POINTER(PaseCSR)]
    L.pase_reserve.argtypes = [vp, i32]
    L.pase_solve.argtypes = [vp, i32, dbl, i32, vp, vp, vp, ctypes.POINTER(PaseStats)]
    L.pase_solve_batches.argtypes = [vp, i32, i32, i32, dbl, vp, vp, ctypes.POINTER(PaseStats)]
    L.pase_solve_batched.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(i32), ctypes.POINTER(dbl),
                                     ctypes.POINTER(i32), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(vp), ctypes.POINTER(PaseStats)]
    L.pase_residual.argtypes = [vp, i32, vp, vp, vp, vp]
    L.pase_linear_solve.argtypes = [vp, i32, vp, vp, vp, vp]
    L.pase_project.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.pase_augmented_eig.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(i32)]
    L.pase_prolongate.argtypes = [vp, i32, vp, vp, vp, vp]
    L.pase_iterate.argtypes = [vp, i32, i32, vp, vp, i32, vp]
    L.pase_spmm_am.argtypes = [vp, i32, vp, vp, vp]
    L.pase_smooth.argtypes = [vp, i32, i32, vp, vp]
    L.pase_smoother_form.argtypes = [vp]
    L.pase_residual_noalloc.argtypes = [i64, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.pase_time_kernel.argtypes = [vp, i32, i32, i32, ctypes.POINTER(dbl)]
    L.pase_profile_kernel.argtypes = [vp, i32]
    L.pase_profile_read.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(dbl)]
    L.pase_set_grid.argtypes = [vp, i32, i32, vp]
    L.pase_smoother_nparams.argtypes = [i32]
    L.pase_smoother_state.argtypes = [vp, vp, i64, i32]
    L.pase_smoother_apply.argtypes = [vp, i32, vp, vp]
    flt = ctypes.c_float
    L.pase_smoother_step.argtypes = [vp, vp, vp, i32, flt, flt, flt, flt, vp, vp]
    L.pase_default_train_options.argtypes = [ctypes.POINTER(PaseTrainOptions)]
    L.pase_default_train_options.restype = None
    L.pase_train_smoother.argtypes = [vp, ctypes.POINTER(PaseTrainOptions), vp]
    L.pase_kernel_count.argtypes = [vp]
    L.pase_kernel_count.restype = i64
    L.pase_launch_counts.argtypes = [vp, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.pase_destroy.argtypes = [vp]
    L.pase_status_string.argtypes = [i32]
    L.pase_status_string.restype = ctypes.c_char_p
    L.pase_last_error.argtypes = []
    L.pase_last_error.restype = ctypes.c_char_p
    for name in ["pase_create", "pase_setup", "pase_reserve", "pase_solve", "pase_solve_batched", "pase_solve_batches",
                 "pase_residual",
                 "pase_linear_solve", "pase_project", "pase_augmented_eig", "pase_prolongate",
                 "pase_iterate", "pase_spmm_am", "pase_smooth", "pase_smoother_form", "pase_residual_noalloc",
                 "pase_time_kernel",
                 "pase_profile_kernel", "pase_profile_read", "pase_set_grid", "pase_smoother_nparams",
                 "pase_smoother_state", "pase_smoother_apply", "pase_smoother_step", "pase_train_smoother",
                 "pase_launch_counts", "pase_destroy"]:
        getattr(L, name).restype = i32
    _lib = L
    return L


def _check(rc, allow=()):
    if rc != PASE_OK and rc not in allow:
        L = load_library()
        raise PaseError(rc, f"{L.pase_status_string(rc).decode()}: {L.pase_last_error().decode()}")
    return rc


def _ptr(a, dtype=np.float64):
    """Raw pointer of a contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array")
        return a.ctypes.data
    # torch tensor
    if not a.is_contiguous():
        raise TypeError("expected a contiguous tensor")
    want = {np.float64: "torch.float64", np.int64: "torch.int64", np.int32: "torch.int32"}[dtype]
    if str(a.dtype) != want:
        raise TypeError(f"expected {want}, got {a.dtype}")
    return a.data_ptr()


def _is_device(a):
    return (not isinstance(a, np.ndarray)) and getattr(a, "is_cuda", False)


def make_csr(indptr, indices, data, shape):
    """PaseCSR view of CSR arrays (numpy host arrays or torch tensors, all on one side).
    The caller keeps the arrays alive for the duration of the call."""
    dev = _is_device(data)
    return PaseCSR(int(shape[0]), int(shape[1]), int(len(indices)), _ptr(indptr, np.int64),
                   _ptr(indices, np.int32), _ptr(data, np.float64), 1 if dev else 0)


def csr_from_scipy(A):
    """(PaseCSR, keep-alive tuple) for a scipy CSR matrix."""
    indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(A.indices, dtype=np.int32)
    data = np.ascontiguousarray(A.data, dtype=np.float64)
    return make_csr(indptr, indices, data, A.shape), (indptr, indices, data)


def pase_default_options():
    o = PaseOptions()
    load_library().pase_default_options(ctypes.byref(o))
    return o


def pase_create(opt=None, stream=None):
    """Handle on the given CUDA stream (int handle, torch.cuda.Stream, or None)."""
    L = load_library()
    h = ctypes.c_void_p()
    s = getattr(stream, "cuda_stream", stream)
    _check(L.pase_create(ctypes.byref(h), ctypes.byref(opt) if opt is not None else None,
                         ctypes.c_void_p(s) if s else None))
    return h


def pase_setup(h, A_h, M_h, P, A_H=None, M_H=None):
    """A_h, M_h, A_H, M_H: scipy CSR; P: list of scipy CSR (the interpolation chain).
    A_H and M_H may both be None (the library forms the Galerkin coarse pencil)."""
    keep = []
    def conv(X):
        c, k = csr_from_scipy(X)
        keep.append(k)
        return c
    cA, cM = conv(A_h), conv(M_h)
    cAH = ctypes.byref(conv(A_H)) if A_H is not None else None
    cMH = ctypes.byref(conv(M_H)) if M_H is not None else None
    arr = (PaseCSR * len(P))(*[conv(p) for p in P])
    return _check(load_library().pase_setup(h, ctypes.byref(cA), ctypes.byref(cM), len(P), arr, cAH, cMH))


def pase_reserve(h, m):
    return _check(load_library().pase_reserve(h, m))


def pase_solve(h, nev, tol, m, U0, lam, U):
    """Returns (status, stats dict); status may be PASE_ERR_NOT_CONVERGED."""
    st = PaseStats()
    rc = _check(load_library().pase_solve(h, nev, tol, m, _ptr(U0), _ptr(lam), _ptr(U),
                                          ctypes.byref(st)), allow=(PASE_ERR_NOT_CONVERGED,))
    return rc, st.as_dict()


def pase_solve_batches(h, nev, k, m, tol, lam, U):
    """The batch scheme of §5 (Alg. 7): first nev pairs in batches of about k, block m.
    Returns (status, stats dict); status may be PASE_ERR_NOT_CONVERGED."""
    st = PaseStats()
    rc = _check(load_library().pase_solve_batches(h, nev, k, m, tol, _ptr(lam), _ptr(U), ctypes.byref(st)),
                allow=(PASE_ERR_NOT_CONVERGED,))
    return rc, st.as_dict()


def pase_solve_batched(handles, nev, tol, m, U0, lam, U):
    """Solve independent problems concurrently; lists of per-problem arguments (U0 entries may
    be None).  Returns (status, list of stats dicts)."""
    n = len(handles)
    H = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    NEV = (ctypes.c_int * n)(*nev)
    TOL = (ctypes.c_double * n)(*tol)
    M = (ctypes.c_int * n)(*m)
    U0p = (ctypes.c_void_p * n)(*[_ptr(x) for x in U0])
    Lp = (ctypes.c_void_p * n)(*[_ptr(x) for x in lam])
    Up = (ctypes.c_void_p * n)(*[_ptr(x) for x in U])
    st = (PaseStats * n)()
    rc = _check(load_library().pase_solve_batched(H, n, NEV, TOL, M, U0p, Lp, Up, st),
                allow=(PASE_ERR_NOT_CONVERGED,))
    return rc, [s.as_dict() for s in st]


def pase_residual(h, m, U, lam, R, relres):
    return _check(load_library().pase_residual(h, m, _ptr(U), _ptr(lam), _ptr(R), _ptr(relres)))


def pase_linear_solve(h, m, U, lam, R, W):
    return _check(load_library().pase_linear_solve(h, m, _ptr(U), _ptr(lam), _ptr(R), _ptr(W)))


def pase_project(h, m, W, aH, bH, GA, GM):
    return _check(load_library().pase_project(h, m, _ptr(W), _ptr(aH), _ptr(bH), _ptr(GA), _ptr(GM)))


def pase_augmented_eig(h, m, aH, bH, GA, GM, lam, C_H, C_W):
    it = ctypes.c_int(0)
    _check(load_library().pase_augmented_eig(h, m, _ptr(aH), _ptr(bH), _ptr(GA), _ptr(GM),
                                             _ptr(lam), _ptr(C_H), _ptr(C_W), ctypes.byref(it)))
    return it.value


def pase_prolongate(h, m, W, C_H, C_W, U):
    return _check(load_library().pase_prolongate(h, m, _ptr(W), _ptr(C_H), _ptr(C_W), _ptr(U)))


def pase_iterate(h, nev, m, U, lam, do_linear_solve=True, relres=None):
    return _check(load_library().pase_iterate(h, nev, m, _ptr(U), _ptr(lam),
                                              1 if do_linear_solve else 0, _ptr(relres)))


def pase_spmm_am(h, m, X, AX, MX):
    return _check(load_library().pase_spmm_am(h, m, _ptr(X), _ptr(AX), _ptr(MX)))


def pase_smooth(h, m, sweeps, B, X):
    return _check(load_library().pase_smooth(h, m, sweeps, _ptr(B), _ptr(X)))


def pase_smoother_form(h):
    return int(load_library().pase_smoother_form(h))


def pase_residual_noalloc(n, m, rowptr, colind, A_val, M_val, U, lam, R, relres, stream=None):
    """Residual without any device allocation; every array must be a CUDA tensor.
    Queued on `stream` (int handle, torch.cuda.Stream or None) without synchronising."""
    s = getattr(stream, "cuda_stream", stream)
    return _check(load_library().pase_residual_noalloc(
        int(n), int(m), _ptr(rowptr, np.int64), _ptr(colind, np.int32), _ptr(A_val), _ptr(M_val),
        _ptr(U), _ptr(lam), _ptr(R), _ptr(relres), ctypes.c_void_p(s) if s else None))


KERNELS = {"spmm_am_fp64": 0, "jacobi_fp64": 1, "jacobi_fp32": 2, "gram_fp64": 3,
           "prolong_fp64": 4, "sygv": 5, "sygv3": 6, "prolong_split": 7,
           "gram_split": 8, "jacobi_fp32_csr": 9, "fma_fp64": 10, "spmm_am_df64": 11}
FMA_FP64_FLOPS = 2.0 * 8 * 4096 * 256 * 152 * 8  # flops of one fma_fp64 launch


def pase_time_kernel(h, kernel, m, reps=10):
    """Average device milliseconds of one launch of a named hot kernel."""
    ms = ctypes.c_double(0.0)
    _check(load_library().pase_time_kernel(h, KERNELS.get(kernel, kernel), m, reps, ctypes.byref(ms)))
    return ms.value


def pase_profile_kernel(h, kernel):
    """Time every fine-level launch of `kernel` (name or id; None stops) while h works."""
    k = -1 if kernel is None else KERNELS.get(kernel, kernel)
    _check(load_library().pase_profile_kernel(h, k))


def pase_profile_read(h):
    """(launches, total_ms) timed since the last read."""
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    _check(load_library().pase_profile_read(h, ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def pase_set_grid(h, dim, n, log_kappa=None):
    """Fine level = interior grid of the uniform n^dim mesh; log_kappa per element (or None)."""
    lk = None if log_kappa is None else np.ascontiguousarray(log_kappa, dtype=np.float64)
    return _check(load_library().pase_set_grid(h, dim, n, _ptr(lk)))


def pase_smoother_nparams(dim):
    return int(load_library().pase_smoother_nparams(dim))


def pase_smoother_state(h, dim, state=None):
    """state None: returns the state (params, m, v, t); else sets it from a tuple
    (params[, m, v, t]) of float arrays (missing moments are zero)."""
    P = pase_smoother_nparams(dim)
    L = load_library()
    if state is None:
        buf = np.empty(3 * P + 1, dtype=np.float32)
        _check(L.pase_smoother_state(h, buf.ctypes.data, buf.size, 1))
        return buf[:P].copy(), buf[P:2 * P].copy(), buf[2 * P:3 * P].copy(), int(buf[3 * P])
    params = np.asarray(state[0], dtype=np.float32)
    m = np.asarray(state[1], dtype=np.float32) if len(state) > 1 else np.zeros(P, np.float32)
    v = np.asarray(state[2], dtype=np.float32) if len(state) > 2 else np.zeros(P, np.float32)
    t = float(state[3]) if len(state) > 3 else 0.0
    buf = np.concatenate([params, m, v, np.array([t], np.float32)]).astype(np.float32)
    return _check(L.pase_smoother_state(h, buf.ctypes.data, buf.size, 0))


def pase_smoother_apply(h, m, R, D):
    return _check(load_library().pase_smoother_apply(h, m, _ptr(R), _ptr(D)))


def pase_smoother_step(h, E, R, update=False, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, want_grad=False, P=None):
    """One training step on 8 columns; returns (loss8, grad or None)."""
    loss = np.empty(8)
    grad = np.empty(P) if want_grad else None
    _check(load_library().pase_smoother_step(h, _ptr(E), _ptr(R), int(update), lr, beta1, beta2, eps,
                                             loss.ctypes.data, None if grad is None else grad.ctypes.data))
    return loss, grad


def pase_default_train_options():
    o = PaseTrainOptions()
    load_library().pase_default_train_options(ctypes.byref(o))
    return o


def pase_train_smoother(h, opt=None, **kw):
    """Returns a dict: loss over the first 10 steps, over the last 10, damped Jacobi's on
    the last 10 steps' samples, and the two-V-cycle energy error factors with the network
    and with Jacobi (the handle keeps Jacobi unless the network's is smaller)."""
    o = opt or pase_default_train_options()
    for k, v in kw.items():
        setattr(o, k, v)
    out = np.empty(5)
    _check(load_library().pase_train_smoother(h, ctypes.byref(o), out.ctypes.data))
    return dict(loss_first=float(out[0]), loss_last=float(out[1]), loss_jacobi=float(out[2]),
                vcycle_factor=float(out[3]), vcycle_factor_jacobi=float(out[4]),
                accepted=bool(out[3] < out[4]))


def pase_kernel_count(h):
    return int(load_library().pase_kernel_count(h))


def pase_launch_counts(h):
    """(kernels, kernels run inside graph replays, graph launches) of the handle so far."""
    k, g, n = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().pase_launch_counts(h, ctypes.byref(k), ctypes.byref(g), ctypes.byref(n)))
    return k.value, g.value, n.value


def pase_destroy(h):
    return _check(load_library().pase_destroy(h))


def pase_status_string(code):
    return load_library().pase_status_string(code).decode()


def pase_last_error():
    return load_library().pase_last_error().decode()
