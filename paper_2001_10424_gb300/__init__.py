"""Python binding of the GB300 GKB saddle-point solver (``libgkb.so``).

Thin ctypes marshalling over the C ABI declared in ``include/gkb.h``: every
function here has the C name, converts its array arguments to raw pointers
(PyTorch CUDA or CPU tensors, or NumPy arrays, all float64 and contiguous)
and calls the library. All arithmetic runs in the library's CUDA kernels;
there is no Python or CPU fallback, and :func:`load` raises if the shared
library has not been built.
"""
import ctypes
import os

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = _build.LIB

GKB_OK = 0
GKB_ERR_INVALID_ARG = 1
GKB_ERR_NOT_SPD = 2
GKB_ERR_NOT_CONVERGED = 3
GKB_ERR_INNER_NOT_CONVERGED = 4
GKB_ERR_NAN = 5
GKB_ERR_TIMEOUT = 6
GKB_ERR_CUDA = 7
GKB_ERR_OOM = 8

GKB_BC_DIRICHLET = 0
GKB_BC_NATURAL = 1
GKB_PREC_FP64 = 0
GKB_PREC_MIXED = 1
GKB_INNER_CG = 0
GKB_INNER_GMG_PCG = 1
GKB_INNER_FCG_UNET = 2
GKB_INNER_FCG_UNET_MG = 3
GKB_INNER_FGMRES = 4
GKB_OP_W, GKB_OP_A, GKB_OP_AT, GKB_OP_M = 0, 1, 2, 3
GKB_VISC_LAPLACE, GKB_VISC_SYMGRAD = 0, 1
KERNEL_CLASSES = ["apply", "residual", "smooth", "restrict", "prolong", "coarse", "blas", "gkb", "layout", "unet"]

STATUS_NAMES = {
    0: "OK", 1: "INVALID_ARG", 2: "NOT_SPD", 3: "NOT_CONVERGED", 4: "INNER_NOT_CONVERGED",
    5: "NAN", 6: "TIMEOUT", 7: "CUDA", 8: "OOM",
}

# symbols declared in include/gkb.h
EXPORTED = [
    "gkb_default_options", "gkb_create", "gkb_set_problem", "gkb_set_problem_n", "gkb_layout", "gkb_boundary_rhs",
    "gkb_solve", "gkb_stats", "gkb_history", "gkb_apply", "gkb_precond", "gkb_last_error",
    "gkb_destroy", "gkb_apply_noalloc", "gkb_solve_batched",
    "gkb_unet_create", "gkb_unet_num_params", "gkb_unet_get_params", "gkb_unet_set_params",
    "gkb_unet_forward", "gkb_unet_loss_grad", "gkb_unet_adam_step", "gkb_unet_last_error", "gkb_unet_destroy",
    "gkb_unet_train", "gkb_unet_set_target_scale", "gkb_unet_get_target_scale", "gkb_set_unet", "gkb_harvest_pairs",
    "gkb_get_options", "gkb_solve_preconditioned",
]
GKB_NOALLOC_MAX_ELEMS = 1048576


class gkb_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double),
                ("bc", ctypes.c_int * 6)]


class gkb_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("inner", ctypes.c_int), ("tol_inner", ctypes.c_double),
                ("maxit", ctypes.c_int), ("maxit_inner", ctypes.c_int), ("smoother_degree", ctypes.c_int),
                ("coarse_max", ctypes.c_int), ("mixed_rtol", ctypes.c_double), ("use_graph", ctypes.c_int),
                ("profile", ctypes.c_int), ("kernel_variant", ctypes.c_int), ("unet_side", ctypes.c_int),
                ("fcg_rho", ctypes.c_double), ("fgmres_restart", ctypes.c_int), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("autotune", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("viscous_form", ctypes.c_int), ("batch_lockstep", ctypes.c_int), ("tail_side", ctypes.c_int)]


class gkb_stats_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iterations", ctypes.c_int), ("inner_solves", ctypes.c_int),
                ("inner_iterations", ctypes.c_int64), ("estimate", ctypes.c_double),
                ("setup_seconds", ctypes.c_double), ("solve_seconds", ctypes.c_double),
                ("levels", ctypes.c_int), ("inner_fallbacks", ctypes.c_int), ("tuned_inner_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64 * 10),
                ("kernel_units", ctypes.c_int64 * 10), ("kernel_ms", ctypes.c_double * 10),
                ("kernel_top_launches", ctypes.c_int64 * 10), ("kernel_top_units", ctypes.c_int64 * 10),
                ("kernel_top_ms", ctypes.c_double * 10)]


class GkbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(code, "?"), code, msg))
        self.code = code


_lib = None
_P = ctypes.c_void_p


def load(path=None):
    """Load ``libgkb.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libgkb.so is not built (%s); run paper_2001_10424_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    i, d = ctypes.c_int, ctypes.c_double
    sig = {
        "gkb_default_options": (i, [ctypes.POINTER(gkb_options)]),
        "gkb_create": (i, [ctypes.POINTER(_P), ctypes.POINTER(gkb_options)]),
        "gkb_set_problem": (i, [_P, ctypes.POINTER(gkb_grid), _P, d, d, d]),
        "gkb_set_problem_n": (i, [_P, ctypes.POINTER(gkb_grid), _P, d, d, _P]),
        "gkb_layout": (i, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "gkb_boundary_rhs": (i, [_P, i, _P, _P, _P]),
        "gkb_solve": (i, [_P, _P, _P, d, i, _P, _P, _P, _P]),
        "gkb_stats": (i, [_P, ctypes.POINTER(gkb_stats_t)]),
        "gkb_history": (i, [_P, _P, _P, _P, _P, _P, i]),
        "gkb_apply": (i, [_P, i, _P, _P]),
        "gkb_precond": (i, [_P, _P, _P]),
        "gkb_last_error": (ctypes.c_char_p, [_P]),
        "gkb_destroy": (i, [_P]),
        "gkb_apply_noalloc": (i, [ctypes.POINTER(gkb_grid), d, d, d, i, _P, _P, _P]),
        "gkb_solve_batched": (i, [ctypes.POINTER(_P), i, ctypes.POINTER(_P), ctypes.POINTER(_P), d, i,
                                  ctypes.POINTER(_P), ctypes.POINTER(_P)]),
        "gkb_unet_create": (i, [ctypes.POINTER(_P), i, i, i, i, ctypes.c_ulonglong, _P]),
        "gkb_unet_num_params": (i, [_P, ctypes.POINTER(ctypes.c_int64)]),
        "gkb_unet_get_params": (i, [_P, _P]),
        "gkb_unet_set_params": (i, [_P, _P]),
        "gkb_unet_forward": (i, [_P, _P, i, i, i, _P, i]),
        "gkb_unet_loss_grad": (i, [_P, _P, _P, i, i, i, ctypes.POINTER(d), _P]),
        "gkb_unet_adam_step": (i, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
        "gkb_unet_last_error": (ctypes.c_char_p, [_P]),
        "gkb_unet_destroy": (i, [_P]),
        "gkb_unet_train": (i, [_P, _P, _P, ctypes.c_int64, i, i, i, i, ctypes.c_float, ctypes.c_ulonglong, _P]),
        "gkb_unet_set_target_scale": (i, [_P, ctypes.c_float]),
        "gkb_unet_get_target_scale": (i, [_P, ctypes.POINTER(ctypes.c_float)]),
        "gkb_set_unet": (i, [_P, _P]),
        "gkb_get_options": (i, [_P, ctypes.POINTER(gkb_options)]),
        "gkb_solve_preconditioned": (i, [_P, _P, _P, d, i, i, d, i, _P, _P, ctypes.POINTER(i)]),
        "gkb_harvest_pairs": (i, [_P, _P, i, _P, _P, ctypes.POINTER(i)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a, dtype="float64"):
    """Raw pointer of a contiguous tensor / array of the given dtype (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        if a.dtype != getattr(torch, dtype) or not a.is_contiguous():
            raise TypeError("tensors must be contiguous %s" % dtype)
        return a.data_ptr()
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.dtype(dtype) or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("arrays must be C-contiguous %s numpy arrays" % dtype)
    return a.ctypes.data


def _check(h, rc, allow=()):
    if rc != GKB_OK and rc not in allow:
        raise GkbError(rc, gkb_last_error(h) if h else "")
    return rc


def make_grid(n, h, bc=None):
    """gkb_grid for ``n`` cells per axis (2 or 3 entries), spacing h, sides bc."""
    g = gkb_grid()
    g.dim = len(n)
    for a, v in enumerate(n):
        g.n[a] = int(v)
    g.h = float(h)
    bc = bc if bc is not None else (GKB_BC_DIRICHLET,) * (2 * len(n))
    for s, v in enumerate(bc):
        g.bc[s] = int(v)
    return g


def gkb_default_options():
    lib = load()
    o = gkb_options()
    _check(None, lib.gkb_default_options(ctypes.byref(o)))
    return o


def gkb_create(opt=None):
    lib = load()
    opt = opt or gkb_default_options()
    h = _P()
    _check(None, lib.gkb_create(ctypes.byref(h), ctypes.byref(opt)))
    return h


def gkb_set_problem(h, grid, viscosity=None, mu0=1.0, gamma=0.0, n_scale=0.0):
    return _check(h, load().gkb_set_problem(h, ctypes.byref(grid), _ptr(viscosity), mu0, gamma, n_scale))


def gkb_set_problem_n(h, grid, n_diag, viscosity=None, mu0=1.0, gamma=0.0):
    """N = diag(n_diag): n values in compact pressure ordering (host or device)."""
    return _check(h, load().gkb_set_problem_n(h, ctypes.byref(grid), _ptr(viscosity), mu0, gamma, _ptr(n_diag)))


def gkb_layout(h):
    m, n = ctypes.c_int64(), ctypes.c_int64()
    _check(h, load().gkb_layout(h, ctypes.byref(m), ctypes.byref(n)))
    return m.value, n.value


def gkb_boundary_rhs(h, side, normal_velocity, g, r):
    return _check(h, load().gkb_boundary_rhs(h, side, _ptr(normal_velocity), _ptr(g), _ptr(r)))


def gkb_solve(h, g, r, tol, delay, w_out, p_out, w0=None, p0=None):
    """Returns the status code; argument / CUDA errors raise GkbError."""
    rc = load().gkb_solve(h, _ptr(g), _ptr(r), tol, delay, _ptr(w_out), _ptr(p_out), _ptr(w0), _ptr(p0))
    return _check(h, rc, allow=(GKB_ERR_NOT_CONVERGED, GKB_ERR_INNER_NOT_CONVERGED, GKB_ERR_NOT_SPD, GKB_ERR_NAN))


def gkb_solve_batched(hs, g, r, tol, delay, w_out, p_out):
    """Batched solve of len(hs) problems in one graph launch; g, r, w_out,
    p_out are lists of per-problem arrays. Returns the status code."""
    n = len(hs)
    arr = lambda xs: (_P * n)(*[_ptr(x) for x in xs])
    H = (_P * n)(*[h.value if hasattr(h, "value") else h for h in hs])
    rc = load().gkb_solve_batched(H, n, arr(g), arr(r), tol, delay, arr(w_out), arr(p_out))
    return _check(hs[0], rc, allow=(GKB_ERR_NOT_CONVERGED, GKB_ERR_INNER_NOT_CONVERGED, GKB_ERR_NOT_SPD, GKB_ERR_NAN))


def gkb_stats(h):
    s = gkb_stats_t()
    _check(h, load().gkb_stats(h, ctypes.byref(s)))
    out = {f: getattr(s, f) for f, _ in s._fields_}
    out["kernel_launches"] = dict(zip(KERNEL_CLASSES, list(s.kernel_launches)))
    out["kernel_units"] = dict(zip(KERNEL_CLASSES, list(s.kernel_units)))
    out["kernel_ms"] = dict(zip(KERNEL_CLASSES, list(s.kernel_ms)))
    out["kernel_top_launches"] = dict(zip(KERNEL_CLASSES, list(s.kernel_top_launches)))
    out["kernel_top_units"] = dict(zip(KERNEL_CLASSES, list(s.kernel_top_units)))
    out["kernel_top_ms"] = dict(zip(KERNEL_CLASSES, list(s.kernel_top_ms)))
    return out


def gkb_history(h, capacity=4096):
    import numpy as np
    a = np.zeros(capacity)
    b = np.zeros(capacity)
    z = np.zeros(capacity)
    e = np.zeros(capacity)
    its = np.zeros(capacity, dtype=np.int32)
    n = load().gkb_history(h, a.ctypes.data, b.ctypes.data, z.ctypes.data, e.ctypes.data, its.ctypes.data, capacity)
    if n < 0:
        raise GkbError(-n, gkb_last_error(h))
    st = gkb_stats(h)
    k = st["outer_iterations"]
    return {"alpha": a[:n], "beta": b[:k + 1], "zeta": z[:n], "estimate": e[:k],
            "inner_iterations": its[:st["inner_solves"]]}


def gkb_apply(h, op, x, y):
    return _check(h, load().gkb_apply(h, op, _ptr(x), _ptr(y)))


def gkb_precond(h, r, z):
    return _check(h, load().gkb_precond(h, _ptr(r), _ptr(z)))


def gkb_apply_noalloc(grid, mu0, gamma, n_scale, op, x, y, stream=None):
    """y = op(x) without a handle or any device allocation (device arrays);
    returns the status code."""
    return load().gkb_apply_noalloc(ctypes.byref(grid), mu0, gamma, n_scale, op, _ptr(x), _ptr(y), stream)


def _ucheck(u, rc):
    if rc != GKB_OK:
        msg = load().gkb_unet_last_error(u)
        raise GkbError(rc, msg.decode() if msg else "")
    return rc


def gkb_unet_create(c_in=3, c1=16, c2=32, c_out=2, seed=0, stream=None):
    u = _P()
    rc = load().gkb_unet_create(ctypes.byref(u), c_in, c1, c2, c_out, seed, stream)
    if rc != GKB_OK:
        raise GkbError(rc, "gkb_unet_create")
    return u


def gkb_unet_num_params(u):
    n = ctypes.c_int64()
    _ucheck(u, load().gkb_unet_num_params(u, ctypes.byref(n)))
    return n.value


def gkb_unet_get_params(u, out):
    return _ucheck(u, load().gkb_unet_get_params(u, _ptr(out, "float32")))


def gkb_unet_set_params(u, params):
    return _ucheck(u, load().gkb_unet_set_params(u, _ptr(params, "float32")))


def gkb_unet_forward(u, x, n, h, w, y, tensor_cores=0):
    return _ucheck(u, load().gkb_unet_forward(u, _ptr(x, "float32"), n, h, w, _ptr(y, "float32"), tensor_cores))


def gkb_unet_loss_grad(u, x, target, n, h, w, grad=None):
    loss = ctypes.c_double()
    _ucheck(u, load().gkb_unet_loss_grad(u, _ptr(x, "float32"), _ptr(target, "float32"), n, h, w,
                                         ctypes.byref(loss), _ptr(grad, "float32")))
    return loss.value


def gkb_unet_adam_step(u, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    return _ucheck(u, load().gkb_unet_adam_step(u, lr, beta1, beta2, eps))


def gkb_unet_train(u, x_img, t_img, count, h, w, batch, steps, lr, seed=0, losses=None):
    """Adam training on device pairs; returns the per-step losses (numpy)."""
    import numpy as np
    out = np.zeros(max(steps, 1), dtype=np.float64) if losses is None else losses
    _ucheck(u, load().gkb_unet_train(u, _ptr(x_img, "float32"), _ptr(t_img, "float32"), count, h, w, batch, steps,
                                     lr, seed, _ptr(out)))
    return out[:steps]


def gkb_unet_set_target_scale(u, s):
    return _ucheck(u, load().gkb_unet_set_target_scale(u, s))


def gkb_unet_get_target_scale(u):
    v = ctypes.c_float()
    _ucheck(u, load().gkb_unet_get_target_scale(u, ctypes.byref(v)))
    return v.value


def gkb_solve_preconditioned(h, g, r, tol, w_out, p_out, restart=20, maxit=200, pc_tol=1e-2, delay=5):
    """FGMRES on the saddle system with GKB (to pc_tol) as preconditioner;
    returns (status, outer iterations)."""
    it = ctypes.c_int()
    rc = _check(h, load().gkb_solve_preconditioned(h, _ptr(g), _ptr(r), tol, restart, maxit, pc_tol, delay,
                                                    _ptr(w_out), _ptr(p_out), ctypes.byref(it)),
                allow=(GKB_ERR_NOT_CONVERGED,))
    return rc, it.value


def gkb_get_options(h):
    o = gkb_options()
    _check(h, load().gkb_get_options(h, ctypes.byref(o)))
    return o


def gkb_set_unet(h, u):
    return _check(h, load().gkb_set_unet(h, u))


def gkb_harvest_pairs(h, f, max_pairs, x_img, t_img):
    """Training pairs from GMG-PCG on M x = f; returns how many were written."""
    n = ctypes.c_int()
    _check(h, load().gkb_harvest_pairs(h, _ptr(f), max_pairs, _ptr(x_img, "float32"), _ptr(t_img, "float32"),
                                       ctypes.byref(n)))
    return n.value


def gkb_unet_last_error(u):
    msg = load().gkb_unet_last_error(u)
    return msg.decode() if msg else ""


def gkb_unet_destroy(u):
    return load().gkb_unet_destroy(u)


def gkb_last_error(h):
    msg = load().gkb_last_error(h)
    return msg.decode() if msg else ""


def gkb_destroy(h):
    return _check(None, load().gkb_destroy(h))
