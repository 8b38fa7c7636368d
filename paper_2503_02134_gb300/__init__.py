"""Python binding of libsem, the GB300 spectral-element Poisson library.

Argument marshalling only: every function forwards to the C-ABI entry point of
the same name in ``libsem.so`` (declared in ``include/sem.h``).  Arrays may be
PyTorch CUDA tensors (passed as device pointers, the normal case) or numpy
arrays / CPU tensors (host pointers, staged by the library).  There is no CPU
implementation behind these calls: if the compiled library is missing, import
fails loudly.

Operations (arXiv 2503.02134): the matrix-free operator ``ax`` (Sec. 3.1,
profiling table), the gather-scatter Sigma' = QQ^T (Sec. 3.3), the Jacobi
preconditioned CG loop in FP64 and in the paper's mixed FP32/FP64 strategy
(Sec. 3.3, 4.3).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsem.so")

SEM_FP64, SEM_MIXED_FP32, SEM_MIXED_TF32, SEM_MIXED_BF16X3, SEM_FP32_ALL = range(5)
SEM_OK, SEM_EINVAL, SEM_ECUDA, SEM_ENOMEM, SEM_ETIMEOUT = 0, -1, -2, -3, -4
SEM_MAXIT, SEM_STAGNATED, SEM_BREAKDOWN = 1, 2, 3

FIELD_G, FIELD_B, FIELD_MINV, FIELD_MULT, FIELD_MASK, FIELD_C, FIELD_COORDS = range(7)
FIELD_XI, FIELD_W, FIELD_D, FIELD_DETJ = 7, 8, 9, 10

RHS_SINE, RHS_UNIFORM = 0, 1


class sem_mesh(ctypes.Structure):
    _fields_ = [("kx", ctypes.c_int), ("ky", ctypes.c_int), ("kz", ctypes.c_int),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("deform_amp", ctypes.c_double), ("deform_kind", ctypes.c_int),
                ("gid", ctypes.POINTER(ctypes.c_int64)),
                ("coords", ctypes.POINTER(ctypes.c_double)),
                ("dirichlet_faces", ctypes.POINTER(ctypes.c_uint8))]


class sem_sizes(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("n", ctypes.c_int), ("E", ctypes.c_int64),
                ("L", ctypes.c_int64), ("U", ctypes.c_int64), ("n_shared", ctypes.c_int64),
                ("n_segments", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class sem_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refinements", ctypes.c_int), ("status", ctypes.c_int),
                ("relres", ctypes.c_double), ("relres_true", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("launches", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sem_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("precision", ctypes.c_int),
                ("fixed_iters", ctypes.c_int), ("no_refine", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_cycles", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("chunk", ctypes.c_int), ("precond", ctypes.c_int),
                ("history", ctypes.POINTER(ctypes.c_double)), ("refine_mode", ctypes.c_int),
                ("replace_factor", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsem.so not built ({LIB_PATH}); run "
                          "`python paper_2503_02134_gb300/build.py` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, h = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "sem_setup": (i, [ctypes.POINTER(sem_mesh), i, i, vp, ctypes.POINTER(h)]),
        "sem_destroy": (None, [h]),
        "sem_last_error": (ctypes.c_char_p, []),
        "sem_get_sizes": (i, [h, ctypes.POINTER(sem_sizes)]),
        "sem_ax": (i, [h, vp, vp, i]),
        "sem_ax_local": (i, [h, vp, vp, i]),
        "sem_gs": (i, [h, vp, i]),
        "sem_glsc3": (i, [h, vp, vp, i, ctypes.POINTER(d)]),
        "sem_get_field": (i, [h, i, vp]),
        "sem_rhs": (i, [h, i, ctypes.c_uint64, vp]),
        "sem_pcg_solve": (i, [h, vp, vp, vp, d, i, i, ctypes.POINTER(sem_info)]),
        "sem_pcg_solve_ex": (i, [h, vp, vp, vp, ctypes.POINTER(sem_solve_opts),
                                 ctypes.POINTER(sem_info)]),
        "sem_set_option": (i, [h, ctypes.c_char_p, ctypes.c_int64]),
        "sem_glsc3_noalloc": (i, [vp, vp, vp, ctypes.c_int64, vp, vp]),
        "sem_fma_peak": (i, [i, i, ctypes.POINTER(d)]),
        "sem_x0_set_option": (i, [vp, ctypes.c_char_p, ctypes.c_int64]),
        "sem_batch_setup": (i, [ctypes.POINTER(sem_mesh), ctypes.POINTER(i), i, vp,
                                ctypes.POINTER(h)]),
        "sem_batch_problem": (i, [h, i, ctypes.POINTER(h)]),
        "sem_batch_pcg_solve": (i, [h, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(sem_solve_opts), ctypes.POINTER(sem_info)]),
        "sem_batch_get_option": (i, [h, ctypes.c_char_p, ctypes.POINTER(d)]),
        "sem_batch_destroy": (None, [h]),
        "sem_rhs_fourier": (i, [h, ctypes.c_uint64, ctypes.c_uint64, vp]),
        "sem_x0_create": (i, [h, i, ctypes.c_uint64, ctypes.POINTER(h)]),
        "sem_x0_param_count": (i, [h, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "sem_x0_params": (i, [h, vp, i]),
        "sem_x0_features": (i, [h, vp, vp, vp]),
        "sem_x0_gradients": (i, [h, vp, vp, i, i, vp, ctypes.POINTER(d)]),
        "sem_x0_add_pair": (i, [h, vp, vp]),
        "sem_x0_train": (i, [h, i, i, ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(d)]),
        "sem_x0_predict": (i, [h, vp, vp, i]),
        "sem_x0_destroy": (None, [h]),
        "sem_get_option": (i, [h, ctypes.c_char_p, ctypes.POINTER(d)]),
        "sem_mg_apply": (i, [h, vp, vp, i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("sem_setup", "sem_destroy", "sem_last_error", "sem_get_sizes", "sem_ax",
            "sem_ax_local", "sem_gs", "sem_glsc3", "sem_get_field", "sem_rhs", "sem_pcg_solve",
            "sem_pcg_solve_ex", "sem_set_option", "sem_get_option", "sem_glsc3_noalloc",
            "sem_batch_setup", "sem_batch_problem", "sem_batch_pcg_solve", "sem_batch_get_option",
            "sem_batch_destroy", "sem_rhs_fourier", "sem_x0_create", "sem_x0_param_count",
            "sem_x0_params", "sem_x0_features", "sem_x0_gradients", "sem_x0_add_pair",
            "sem_x0_train", "sem_x0_predict", "sem_x0_destroy", "sem_mg_apply", "sem_fma_peak",
            "sem_x0_set_option")


class SemError(RuntimeError):
    def __init__(self, code, where):
        msg = _lib.sem_last_error().decode(errors="replace")
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


def _check(code, where):
    if code < 0:
        raise SemError(code, where)
    return code


def _ptr(a):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


# ----------------------------------------------------------------- C-ABI mirrors
def sem_setup(mesh: sem_mesh, N: int, geom_flags: int = 0, stream: int | None = None):
    h = ctypes.c_void_p()
    _check(_lib.sem_setup(ctypes.byref(mesh), N, geom_flags, stream, ctypes.byref(h)), "sem_setup")
    return h


def sem_destroy(h):
    _lib.sem_destroy(h)


def sem_last_error() -> str:
    return _lib.sem_last_error().decode(errors="replace")


def sem_get_sizes(h) -> sem_sizes:
    s = sem_sizes()
    _check(_lib.sem_get_sizes(h, ctypes.byref(s)), "sem_get_sizes")
    return s


def sem_ax(h, u, w, precision):
    return _check(_lib.sem_ax(h, _ptr(u), _ptr(w), precision), "sem_ax")


def sem_ax_local(h, u, w, precision):
    return _check(_lib.sem_ax_local(h, _ptr(u), _ptr(w), precision), "sem_ax_local")


def sem_gs(h, v, precision):
    return _check(_lib.sem_gs(h, _ptr(v), precision), "sem_gs")


def sem_mg_apply(h, r, z, precision):
    return _check(_lib.sem_mg_apply(h, _ptr(r), _ptr(z), precision), "sem_mg_apply")


def sem_glsc3(h, a, b, precision) -> float:
    out = ctypes.c_double()
    _check(_lib.sem_glsc3(h, _ptr(a), _ptr(b), precision, ctypes.byref(out)), "sem_glsc3")
    return out.value


def sem_get_field(h, which, out):
    return _check(_lib.sem_get_field(h, which, _ptr(out)), "sem_get_field")


def sem_rhs(h, kind, seed, b):
    return _check(_lib.sem_rhs(h, kind, seed, _ptr(b)), "sem_rhs")


def sem_pcg_solve(h, f, x0, x, tol, maxit, precision):
    info = sem_info()
    rc = _check(_lib.sem_pcg_solve(h, _ptr(f), _ptr(x0), _ptr(x), tol, maxit, precision,
                                   ctypes.byref(info)), "sem_pcg_solve")
    return rc, info


def sem_pcg_solve_ex(h, f, x0, x, opts: sem_solve_opts):
    info = sem_info()
    rc = _check(_lib.sem_pcg_solve_ex(h, _ptr(f), _ptr(x0), _ptr(x), ctypes.byref(opts),
                                      ctypes.byref(info)), "sem_pcg_solve_ex")
    return rc, info


def sem_glsc3_noalloc(a, b, c, n, result, stream=None):
    """Allocation-free sum_i a_i c_i b_i into the device double `result`."""
    return _check(_lib.sem_glsc3_noalloc(_ptr(a), _ptr(b), _ptr(c), int(n), _ptr(result), stream),
                  "sem_glsc3_noalloc")


def sem_fma_peak(fp64: bool, iters: int) -> float:
    """Measured FMA throughput of the CUDA cores in TFLOP/s (FP64 or FP32)."""
    out = ctypes.c_double()
    _check(_lib.sem_fma_peak(1 if fp64 else 0, int(iters), ctypes.byref(out)), "sem_fma_peak")
    return out.value


def sem_batch_setup(meshes, Ns, stream=None):
    count = len(meshes)
    arr = (sem_mesh * count)(*meshes)
    ns = (ctypes.c_int * count)(*Ns)
    b = ctypes.c_void_p()
    _check(_lib.sem_batch_setup(arr, ns, count, stream, ctypes.byref(b)), "sem_batch_setup")
    return b


def sem_batch_problem(b, i):
    h = ctypes.c_void_p()
    _check(_lib.sem_batch_problem(b, i, ctypes.byref(h)), "sem_batch_problem")
    return h


def sem_batch_pcg_solve(b, fs, xs, opts: sem_solve_opts):
    count = len(fs)
    fa = (ctypes.c_void_p * count)(*[_ptr(t) for t in fs])
    xa = (ctypes.c_void_p * count)(*[_ptr(t) for t in xs])
    infos = (sem_info * count)()
    rc = _check(_lib.sem_batch_pcg_solve(b, fa, xa, ctypes.byref(opts), infos),
                "sem_batch_pcg_solve")
    return rc, [infos[i].as_dict() for i in range(count)]


def sem_batch_get_option(b, key: str) -> float:
    out = ctypes.c_double()
    _check(_lib.sem_batch_get_option(b, key.encode(), ctypes.byref(out)), "sem_batch_get_option")
    return out.value


def sem_batch_destroy(b):
    _lib.sem_batch_destroy(b)


def sem_rhs_fourier(h, seed, sample, b):
    return _check(_lib.sem_rhs_fourier(h, seed, sample, _ptr(b)), "sem_rhs_fourier")


def sem_x0_create(h, hidden=256, seed=0):
    m = ctypes.c_void_p()
    _check(_lib.sem_x0_create(h, hidden, seed, ctypes.byref(m)), "sem_x0_create")
    return m


def sem_x0_param_count(m):
    sz = (ctypes.c_int64 * 6)()
    off = (ctypes.c_int64 * 6)()
    _check(_lib.sem_x0_param_count(m, sz, off), "sem_x0_param_count")
    return list(sz), list(off)


def sem_x0_params(m, host, set_=False):
    return _check(_lib.sem_x0_params(m, _ptr(host), 1 if set_ else 0), "sem_x0_params")


def sem_x0_features(m, b, X, scale=None):
    return _check(_lib.sem_x0_features(m, _ptr(b), _ptr(X), _ptr(scale)), "sem_x0_features")


def sem_x0_gradients(m, X, T, rows, bf16_mode, grads):
    loss = ctypes.c_double()
    _check(_lib.sem_x0_gradients(m, _ptr(X), _ptr(T), rows, bf16_mode, _ptr(grads), ctypes.byref(loss)),
           "sem_x0_gradients")
    return loss.value


def sem_x0_add_pair(m, b, x):
    return _check(_lib.sem_x0_add_pair(m, _ptr(b), _ptr(x)), "sem_x0_add_pair")


def sem_x0_train(m, epochs, batch, lr, seed=0):
    loss = ctypes.c_double()
    _check(_lib.sem_x0_train(m, epochs, batch, lr, seed, ctypes.byref(loss)), "sem_x0_train")
    return loss.value


def sem_x0_predict(m, b, x0, energy_scale=True):
    return _check(_lib.sem_x0_predict(m, _ptr(b), _ptr(x0), 1 if energy_scale else 0), "sem_x0_predict")


def sem_x0_set_option(m, key: str, value: int):
    return _check(_lib.sem_x0_set_option(m, key.encode(), int(value)), "sem_x0_set_option")


def sem_x0_destroy(m):
    _lib.sem_x0_destroy(m)


def sem_set_option(h, key: str, value: int):
    return _check(_lib.sem_set_option(h, key.encode(), int(value)), "sem_set_option")


def sem_get_option(h, key: str) -> float:
    out = ctypes.c_double()
    _check(_lib.sem_get_option(h, key.encode(), ctypes.byref(out)), "sem_get_option")
    return out.value


# ----------------------------------------------------------------- convenience
def box_mesh(kx, ky, kz, deform=False, amp=0.05, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    m = sem_mesh()
    m.kx, m.ky, m.kz = kx, ky, kz
    m.lo[:] = list(lo)
    m.hi[:] = list(hi)
    m.deform_amp = amp if deform else 0.0
    m.deform_kind = 1 if deform else 0
    return m


def user_mesh(E, gid: np.ndarray, coords: np.ndarray, faces: np.ndarray):
    """A general conforming hex mesh (arrays must stay alive during sem_setup)."""
    m = sem_mesh()
    m.kx, m.ky, m.kz = E, 1, 1
    m.gid = gid.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    m.coords = coords.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    m.dirichlet_faces = faces.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    return m


class Solver:
    """Owns one sem handle; thin wrapper used by the tests and the benchmark."""

    def __init__(self, kx, ky, kz, N, deform=False, amp=0.05, stream=None, mesh=None):
        self.mesh = mesh if mesh is not None else box_mesh(kx, ky, kz, deform, amp)
        self.h = sem_setup(self.mesh, N, 0, stream)
        s = sem_get_sizes(self.h)
        self.N, self.n, self.E, self.L, self.U = s.N, s.n, s.E, s.L, s.U
        self.sizes = s

    def close(self):
        if self.h is not None:
            sem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def field(self, which, count=None):
        import torch
        if count is None:
            count = {FIELD_G: 6 * self.L, FIELD_COORDS: 3 * self.L, FIELD_XI: self.n,
                     FIELD_W: self.n, FIELD_D: self.n * self.n}.get(which, self.L)
        out = torch.empty(count, dtype=torch.float64, device="cuda")
        sem_get_field(self.h, which, out)
        return out

    def solve(self, f, x0=None, tol=1e-8, maxit=1000, precision=SEM_FP64, fixed_iters=0,
              no_refine=False, history=False, use_graph=True, chunk=0, inner_tol=0.0,
              precond=True, x=None, refine_mode=0, replace_factor=0.0):
        import torch
        if x is None:
            x = torch.empty_like(f)
        o = sem_solve_opts()
        o.tol, o.maxit, o.precision = tol, maxit, precision
        o.fixed_iters = fixed_iters
        o.no_refine = 1 if no_refine else 0
        o.use_graph = 1 if use_graph else -1
        o.chunk = chunk
        o.inner_tol = inner_tol
        o.precond = 2 if precond == "mg" else (1 if precond else -1)
        o.refine_mode = refine_mode
        o.replace_factor = replace_factor
        hist = None
        if history:
            hist = np.zeros((fixed_iters or maxit) + 1)
            o.history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        rc, info = sem_pcg_solve_ex(self.h, f, x0, x, o)
        out = info.as_dict()
        out["rc"] = rc
        if history:
            out["history"] = hist[:info.iters + 1]
        return x, out
