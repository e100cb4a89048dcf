"""Thin Python binding of libmpcg (argument marshalling only).

The functions carry the names of the C entry points declared in
``include/mpcg.h``; every computation runs in the CUDA library.  Device
arrays are passed as raw pointers (``tensor.data_ptr()``); host arrays as
numpy buffers.  A missing library raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmpcg.so")

MPCG_OK = 0
MPCG_NOT_CONVERGED = 1
MPCG_ERR_ARG = -1
MPCG_ERR_CUDA = -2
MPCG_ERR_NOT_SPD = -3
MPCG_ERR_BREAKDOWN = -4
MPCG_ERR_TIMEOUT = -5
MPCG_ERR_OOM = -6
MPCG_FORMAT_STENCIL = 0
MPCG_SMOOTHER_JACOBI = 0
MPCG_SMOOTHER_SSOR = 1
MPCG_FP64 = 0
MPCG_MIXED = 1
MPCG_FP64_DW = 2   # FP64 data, double-word (2 x FP32) arithmetic
MPCG_MAX_COLS = 12
MPCG_MAX_WINDOW = 16
MPCG_AMG_A = 0
MPCG_AMG_P = 1
MPCG_AMG_R = 2


class MpcgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libmpcg status {status}: {msg}")
        self.status = status


MPCG_ALL_FACES = 0x3F


class mg_operator(C.Structure):
    _fields_ = [("dim", C.c_int), ("nodes", C.c_int), ("format", C.c_int), ("values_dev", C.c_void_p),
                ("dofs_per_node", C.c_int), ("dirichlet_faces", C.c_uint)]


class mpcg_options(C.Structure):
    _fields_ = [("m", C.c_int), ("nu", C.c_int), ("omega", C.c_double), ("pinv_tau", C.c_double),
                ("drop_delta", C.c_double), ("precision", C.c_int), ("inner_rtol", C.c_double),
                ("inner_pinv_tau", C.c_double), ("inner_drop_delta", C.c_double), ("max_outer", C.c_int),
                ("use_graph", C.c_int), ("sum_columns", C.c_int), ("smoother", C.c_int), ("ssor_omega", C.c_double),
                ("vcycle", C.c_int), ("half_stencil", C.c_int), ("stream", C.c_void_p)]


class mg_csr(C.Structure):
    _fields_ = [("n", C.c_int), ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class mg_amg_options(C.Structure):
    _fields_ = [("theta", C.c_double), ("w", C.c_double), ("max_levels", C.c_int), ("coarse_size", C.c_int)]


class mg_train_opts(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("seed", C.c_ulonglong)]


_lib = None

# name -> (restype, argtypes); mirrors include/mpcg.h
_SIGS = {
    "mpcg_default_options": (C.c_int, [C.POINTER(mpcg_options)]),
    "mg_hierarchy_setup": (C.c_int, [C.POINTER(mg_operator), C.c_int, C.POINTER(mpcg_options), C.POINTER(C.c_void_p)]),
    "mpcg_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int),
                             C.c_void_p, C.c_void_p]),
    "mg_num_levels": (C.c_int, [C.c_void_p]),
    "mg_num_columns": (C.c_int, [C.c_void_p]),
    "mg_level_size": (C.c_longlong, [C.c_void_p, C.c_int]),
    "mg_apply_operator": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "mg_corrections": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mg_apply_operator_f32": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "mg_corrections_f32": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mg_get_operator": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "mg_hierarchy_destroy": (None, [C.c_void_p]),
    "mpcg_last_error": (C.c_char_p, []),
    "mpcg_kernel_class_name": (C.c_char_p, [C.c_int]),
    "mpcg_solve_profiled": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                      C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_longlong, C.POINTER(C.c_longlong)]),
    "mg_last_launches": (C.c_longlong, [C.c_void_p]),
    "mg_last_solve_counters": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "mg_stencil_apply_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                           C.c_void_p]),
    "mg_hierarchy_setup_batched": (C.c_int, [C.POINTER(mg_operator), C.c_int, C.c_int, C.POINTER(mpcg_options),
                                             C.POINTER(C.c_void_p)]),
    "mg_num_problems": (C.c_int, [C.c_void_p]),
    "mg_amg_default_options": (C.c_int, [C.POINTER(mg_amg_options)]),
    "mg_hierarchy_setup_algebraic": (C.c_int, [C.POINTER(mg_csr), C.POINTER(mg_amg_options),
                                               C.POINTER(mpcg_options), C.POINTER(C.c_void_p)]),
    "mg_amg_aggregates": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "mg_amg_nnz": (C.c_longlong, [C.c_void_p, C.c_int, C.c_int]),
    "mg_amg_get": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mg_amg_setup_host": (C.c_int, [C.POINTER(mg_csr), C.POINTER(mg_amg_options), C.POINTER(C.c_void_p)]),
    "mg_amg_host_levels": (C.c_int, [C.c_void_p]),
    "mg_amg_host_size": (C.c_longlong, [C.c_void_p, C.c_int]),
    "mg_amg_host_nnz": (C.c_longlong, [C.c_void_p, C.c_int, C.c_int]),
    "mg_amg_host_aggregates": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "mg_amg_host_get": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mg_amg_host_destroy": (None, [C.c_void_p]),
    "mg_amg_host_ell_entries": (C.c_longlong, [C.c_void_p, C.c_int, C.c_int]),
    "mg_amg_host_ell": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "mpcg_solve_batched": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_void_p), C.c_double, C.c_int, C.POINTER(C.c_void_p)]),
    "mpcg_solve_batched_graph": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p),
                                           C.POINTER(C.c_void_p), C.c_double, C.c_int, C.POINTER(C.c_void_p)]),
    "mg_learned_num_params": (C.c_int, []),
    "mg_set_tensor_wait_limit": (C.c_int, [C.c_longlong]),
    "mg_learned_num_params_of": (C.c_int, [C.c_void_p]),
    "mg_learned_attach": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "mg_learned_detach": (C.c_int, [C.c_void_p]),
    "mg_attach_q1_kappa": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mg_detach_q1_kappa": (C.c_int, [C.c_void_p]),
    "mg_learned_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "mg_autotune": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_int)]),
    "mg_autotune_load": (C.c_int, [C.c_char_p, C.c_char_p, C.c_int, C.POINTER(C.c_int)]),
    "mg_autotune_save": (C.c_int, [C.c_char_p, C.c_char_p, C.c_int]),
    "mg_autotune_lookup": (C.c_int, [C.c_int, C.c_int, C.c_longlong, C.c_int, C.c_int]),
    "mg_autotune_set": (None, [C.c_int, C.c_int, C.c_longlong, C.c_int, C.c_int, C.c_int]),
    "mg_autotune_clear": (None, []),
    "mg_learned_forward_acts": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "mg_learned_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "mg_learned_train": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                   C.POINTER(mg_train_opts), C.c_void_p, C.c_void_p]),
}
MPCG_NUM_KERNEL_CLASSES = 17


def load(path: str = LIB_PATH):
    """Load libmpcg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2402_12833_gb300.build.build()")
        lib = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def mpcg_last_error() -> str:
    return load().mpcg_last_error().decode()


def _check(status: int, allow=(MPCG_OK,)) -> int:
    if status not in allow:
        raise MpcgError(status, mpcg_last_error())
    return status


def mpcg_default_options(**overrides) -> mpcg_options:
    o = mpcg_options()
    _check(load().mpcg_default_options(C.byref(o)))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(a) -> int:
    """Address of a torch tensor or numpy array (contiguous float64)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"] and not a.flags["F_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data
    raise TypeError(type(a))


def mg_hierarchy_setup(values_dev, dim: int, nodes: int, levels: int, options: mpcg_options | None = None,
                       dofs_per_node: int = 1, faces: int = MPCG_ALL_FACES) -> int:
    """Return an opaque hierarchy handle for the fine stencil ``values_dev``
    (device float64 array of shape (dofs_per_node * 3**dim, n))."""
    op = mg_operator(dim, nodes, MPCG_FORMAT_STENCIL, _ptr(values_dev), dofs_per_node, faces)
    h = C.c_void_p()
    opt = options if options is not None else mpcg_default_options()
    _check(load().mg_hierarchy_setup(C.byref(op), levels, C.byref(opt), C.byref(h)))
    return h.value


def mpcg_solve(h: int, b, x, rtol: float = 1e-8, maxit: int = 500, histories: bool = True,
               ncols: int | None = None):
    """Run the solver; returns (status, iterations, res_hist, alpha_hist).
    ``b`` and ``x`` are device tensors or host numpy arrays of n doubles."""
    it = C.c_int(0)
    ncols = mg_num_columns(h) if ncols is None else ncols
    rh = np.zeros(maxit + 1) if histories else None
    ah = np.zeros(maxit * ncols) if histories else None
    st = load().mpcg_solve(h, _ptr(b), _ptr(x), rtol, maxit, C.byref(it),
                           rh.ctypes.data if histories else None, ah.ctypes.data if histories else None)
    _check(st, allow=(MPCG_OK, MPCG_NOT_CONVERGED))
    k = it.value
    if histories:
        return st, k, rh[: k + 1].copy(), ah[: k * ncols].reshape(k, ncols).copy()
    return st, k, None, None


def mpcg_kernel_class_name(cls: int) -> str:
    return load().mpcg_kernel_class_name(cls).decode()


def mpcg_solve_profiled(h: int, b, x, rtol: float = 1e-8, maxit: int = 500, trace_cap: int = 1 << 16):
    """Solve with per-launch CUDA-event timing; returns (status, iterations,
    {class name: (total ms, launches)}, [(class name, ms) per launch]).
    iterations is an int, or an array with one count per problem for a
    batched hierarchy."""
    nprob = max(1, mg_num_problems(h))
    it = np.zeros(nprob, dtype=np.int32)
    ms = np.zeros(MPCG_NUM_KERNEL_CLASSES)
    cnt = np.zeros(MPCG_NUM_KERNEL_CLASSES, dtype=np.int64)
    tc = np.zeros(trace_cap, dtype=np.int32)
    tm = np.zeros(trace_cap, dtype=np.float32)
    tl = C.c_longlong(0)
    st = load().mpcg_solve_profiled(h, _ptr(b), _ptr(x), rtol, maxit, it.ctypes.data_as(C.POINTER(C.c_int)),
                                    ms.ctypes.data, cnt.ctypes.data, tc.ctypes.data, tm.ctypes.data, trace_cap,
                                    C.byref(tl))
    _check(st, allow=(MPCG_OK, MPCG_NOT_CONVERGED))
    names = [mpcg_kernel_class_name(i) for i in range(MPCG_NUM_KERNEL_CLASSES)]
    n = min(tl.value, trace_cap)
    trace = [(names[int(c)], float(t)) for c, t in zip(tc[:n], tm[:n])]
    iters = int(it[0]) if nprob == 1 else it.copy()
    return st, iters, {names[i]: (float(ms[i]), int(cnt[i])) for i in range(MPCG_NUM_KERNEL_CLASSES)}, trace


def mg_last_launches(h: int) -> int:
    return load().mg_last_launches(h)


def mg_last_solve_counters(h: int, problem: int = 0) -> dict:
    """Counters of the last solve: x updates, termination code, dropped
    columns, eigenvalue pseudo-inverse blocks."""
    out = np.zeros(4, dtype=np.int32)
    _check(load().mg_last_solve_counters(h, problem, out.ctypes.data))
    return {"iters": int(out[0]), "done": int(out[1]), "dropped": int(out[2]), "pinv_fallbacks": int(out[3])}


def mg_num_levels(h: int) -> int:
    return load().mg_num_levels(h)


def mg_num_columns(h: int) -> int:
    return load().mg_num_columns(h)


def mg_level_size(h: int, level: int) -> int:
    return load().mg_level_size(h, level)


def mg_apply_operator(h: int, level: int, X_dev, Y_dev, ncols: int) -> None:
    _check(load().mg_apply_operator(h, level, _ptr(X_dev), _ptr(Y_dev), ncols))


def mg_corrections(h: int, r_dev, Z_dev) -> None:
    _check(load().mg_corrections(h, _ptr(r_dev), _ptr(Z_dev)))


def mg_apply_operator_f32(h: int, level: int, X_dev, Y_dev, ncols: int) -> None:
    """mg_apply_operator in the FP32 arithmetic of the mixed inner solves."""
    _check(load().mg_apply_operator_f32(h, level, _ptr(X_dev), _ptr(Y_dev), ncols))


def mg_corrections_f32(h: int, r_dev, Z_dev) -> None:
    """mg_corrections in the FP32 arithmetic of the mixed inner solves."""
    _check(load().mg_corrections_f32(h, _ptr(r_dev), _ptr(Z_dev)))


def mg_get_operator(h: int, level: int, planes_dev) -> None:
    _check(load().mg_get_operator(h, level, _ptr(planes_dev)))


def mg_stencil_apply_noalloc(dim: int, nodes: int, values_dev, X_dev, Y_dev, ncols: int, stream: int = 0) -> None:
    """Y = A X on the fine grid without device allocation (static scratch;
    enqueued on ``stream``, not synchronised)."""
    _check(load().mg_stencil_apply_noalloc(dim, nodes, _ptr(values_dev), _ptr(X_dev), _ptr(Y_dev), ncols, stream))


def mg_learned_num_params() -> int:
    return load().mg_learned_num_params()


def mg_learned_num_params_of(h: int) -> int:
    """Parameter count of h's network (2D scalar or 3D vector problem)."""
    return load().mg_learned_num_params_of(h)


def mg_learned_attach(h: int, params) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32) if isinstance(params, np.ndarray) else params
    _check(load().mg_learned_attach(h, _ptr(p), mg_learned_num_params_of(h)))


MG_TENSOR_WAIT_DEFAULT = 1 << 22


def mg_set_tensor_wait_limit(polls: int) -> None:
    """Polls of the first bounded waits of the tensor-core kernels (0: give
    up at once, exercising the timeout path)."""
    _check(load().mg_set_tensor_wait_limit(polls))


def mg_learned_detach(h: int) -> None:
    _check(load().mg_learned_detach(h))


def mg_attach_q1_kappa(h: int, kappa_dev) -> None:
    """Matrix-free FP32 fine operator from the element coefficients (device
    tensor of (nodes - 1)^3 float64, x fastest); checked against the stored
    fine stencil."""
    _check(load().mg_attach_q1_kappa(h, _ptr(kappa_dev)))


def mg_detach_q1_kappa(h: int) -> None:
    _check(load().mg_detach_q1_kappa(h))


def mg_learned_forward(h: int, rhat_dev, y_dev, nimg: int = 1) -> None:
    _check(load().mg_learned_forward(h, _ptr(rhat_dev), _ptr(y_dev), nimg))


MG_TUNE_STREAM_BLOCKS, MG_TUNE_SPMM_BLOCKS, MG_TUNE_GRAM_CHUNKS, MG_TUNE_JACOBI_NARROW = 0, 1, 2, 3
MG_TUNE_ANY, MG_TUNE_F32, MG_TUNE_F64, MG_TUNE_DW = -1, 0, 1, 2


def mg_autotune(h: int, cache_path: str | None = None) -> int:
    """Tune the launch shapes for h (see mpcg.h); returns the number of
    candidates timed (0 when the cache served)."""
    timed = C.c_int(0)
    _check(load().mg_autotune(h, cache_path.encode() if cache_path else None, C.byref(timed)))
    return timed.value


def mg_autotune_load(path: str, device: str, sm_count: int) -> int:
    n = C.c_int(0)
    _check(load().mg_autotune_load(path.encode(), device.encode(), sm_count, C.byref(n)))
    return n.value


def mg_autotune_save(path: str, device: str, sm_count: int) -> None:
    _check(load().mg_autotune_save(path.encode(), device.encode(), sm_count))


def mg_autotune_lookup(tunable: int, kind: int, npts: int, nb: int, ncols: int) -> int:
    return load().mg_autotune_lookup(tunable, kind, npts, nb, ncols)


def mg_autotune_set(tunable: int, kind: int, npts: int, nb: int, ncols: int, value: int) -> None:
    load().mg_autotune_set(tunable, kind, npts, nb, ncols, value)


def mg_autotune_clear() -> None:
    load().mg_autotune_clear()


def mg_learned_forward_acts(h: int, rhat_dev, y_dev, acts_dev, nimg: int = 1) -> None:
    """Forward pass that also fills acts_dev ([4][nimg][n][16] floats)."""
    _check(load().mg_learned_forward_acts(h, _ptr(rhat_dev), _ptr(y_dev), _ptr(acts_dev), nimg))


def mg_learned_grad(h: int, params: np.ndarray, rhat_dev, e_dev, nimg: int, acts_dev=None, y_dev=None):
    """One forward + backward pass of the training kernels; returns
    (gradient as float64 array, mean loss)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    grad = np.zeros(mg_learned_num_params_of(h))
    loss = C.c_double(0.0)
    _check(load().mg_learned_grad(h, p.ctypes.data, _ptr(rhat_dev), _ptr(e_dev), nimg, grad.ctypes.data,
                                  _ptr(acts_dev) if acts_dev is not None else None,
                                  _ptr(y_dev) if y_dev is not None else None, C.byref(loss)))
    return grad, loss.value


def mg_learned_train(handles, pair_prob, rhat_dev, e_dev, params: np.ndarray, epochs: int = 10, batch: int = 8,
                     lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, seed: int = 7):
    """Train in place: ``params`` (host float32 array) holds the initial and
    returns the trained weights; returns the per-epoch mean loss."""
    hs = (C.c_void_p * len(handles))(*handles)
    pp = np.ascontiguousarray(pair_prob, dtype=np.int32)
    o = mg_train_opts(epochs, batch, lr, beta1, beta2, eps, seed)
    loss = np.zeros(max(epochs, 1))
    assert params.dtype == np.float32 and params.flags["C_CONTIGUOUS"]
    _check(load().mg_learned_train(hs, len(handles), pp.ctypes.data, len(pp), _ptr(rhat_dev), _ptr(e_dev),
                                   C.byref(o), params.ctypes.data, loss.ctypes.data))
    return loss[:epochs]


def mg_hierarchy_destroy(h: int) -> None:
    if h:
        load().mg_hierarchy_destroy(h)


def mg_num_problems(h: int) -> int:
    return load().mg_num_problems(h)


class BatchedHierarchy:
    """Owning wrapper of a batched hierarchy: nprob problems on one grid."""

    def __init__(self, stencils, dim: int, nodes: int, levels: int, dofs_per_node: int = 1,
                 faces: int = MPCG_ALL_FACES, **options):
        self.options = mpcg_default_options(**options)
        self._keep = list(stencils)
        ops = (mg_operator * len(self._keep))(*[mg_operator(dim, nodes, MPCG_FORMAT_STENCIL, _ptr(s),
                                                            dofs_per_node, faces) for s in self._keep])
        h = C.c_void_p()
        _check(load().mg_hierarchy_setup_batched(ops, len(self._keep), levels, C.byref(self.options), C.byref(h)))
        self.h = h.value
        self.nprob = len(self._keep)
        self.n = mg_level_size(self.h, levels - 1)

    def solve(self, b, x, rtol=1e-8, maxit=500):
        """b, x: nprob x n (device tensors or host arrays); returns (status, iterations[nprob])."""
        it = np.zeros(self.nprob, dtype=np.int32)
        st = load().mpcg_solve(self.h, _ptr(b), _ptr(x), rtol, maxit, it.ctypes.data_as(C.POINTER(C.c_int)),
                               None, None)
        _check(st, allow=(MPCG_OK, MPCG_NOT_CONVERGED))
        return st, it

    def close(self):
        if self.h:
            mg_hierarchy_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mpcg_solve_batched(classes, bs, xs, rtol=1e-8, maxit=500, one_graph=None):
    """Solve every BatchedHierarchy in ``classes`` concurrently; returns
    (status, [iterations per class]).  one_graph=True calls
    mpcg_solve_batched_graph (one graph launch, mixed precision only);
    None lets the library choose."""
    n = len(classes)
    hs = (C.c_void_p * n)(*[c.h for c in classes])
    bp = (C.c_void_p * n)(*[_ptr(b) for b in bs])
    xp = (C.c_void_p * n)(*[_ptr(x) for x in xs])
    its = [np.zeros(c.nprob, dtype=np.int32) for c in classes]
    ip = (C.c_void_p * n)(*[i.ctypes.data for i in its])
    fn = load().mpcg_solve_batched_graph if one_graph else load().mpcg_solve_batched
    st = fn(hs, n, bp, xp, rtol, maxit, ip)
    _check(st, allow=(MPCG_OK, MPCG_NOT_CONVERGED))
    return st, its


def mg_amg_default_options(**overrides) -> mg_amg_options:
    o = mg_amg_options()
    _check(load().mg_amg_default_options(C.byref(o)))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def mg_hierarchy_setup_algebraic(indptr, indices, data, amg: mg_amg_options | None = None,
                                 options: mpcg_options | None = None) -> int:
    """Algebraic hierarchy of the host CSR matrix (indptr, indices, data)."""
    rp = np.ascontiguousarray(indptr, dtype=np.int32)
    ci = np.ascontiguousarray(indices, dtype=np.int32)
    va = np.ascontiguousarray(data, dtype=np.float64)
    A = mg_csr(len(rp) - 1, rp.ctypes.data, ci.ctypes.data, va.ctypes.data)
    h = C.c_void_p()
    a = amg if amg is not None else mg_amg_default_options()
    opt = options if options is not None else mpcg_default_options()
    _check(load().mg_hierarchy_setup_algebraic(C.byref(A), C.byref(a), C.byref(opt), C.byref(h)))
    return h.value


def mg_amg_aggregates(h: int, level: int) -> np.ndarray:
    out = np.empty(mg_level_size(h, level), dtype=np.int32)
    _check(load().mg_amg_aggregates(h, level, out.ctypes.data))
    return out


def mg_amg_nnz(h: int, level: int, which: int) -> int:
    return load().mg_amg_nnz(h, level, which)


def mg_amg_get(h: int, level: int, which: int):
    """(indptr, indices, data) of A_level or P_level as numpy arrays."""
    nnz = mg_amg_nnz(h, level, which)
    if nnz < 0:
        raise MpcgError(MPCG_ERR_ARG, "bad level or matrix")
    rp = np.empty(mg_level_size(h, level) + 1, dtype=np.int32)
    ci = np.empty(nnz, dtype=np.int32)
    va = np.empty(nnz, dtype=np.float64)
    _check(load().mg_amg_get(h, level, which, rp.ctypes.data, ci.ctypes.data, va.ctypes.data))
    return rp, ci, va


class AmgHost:
    """The smoothed-aggregation grids built on the host only (no device):
    levels, sizes, aggregates and the CSR matrices of every grid."""

    def __init__(self, A, theta=None, w=None, max_levels=None, coarse_size=None):
        amg = {k: v for k, v in dict(theta=theta, w=w, max_levels=max_levels, coarse_size=coarse_size).items()
               if v is not None}
        rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
        ci = np.ascontiguousarray(A.indices, dtype=np.int32)
        va = np.ascontiguousarray(A.data, dtype=np.float64)
        M = mg_csr(len(rp) - 1, rp.ctypes.data, ci.ctypes.data, va.ctypes.data)
        h = C.c_void_p()
        _check(load().mg_amg_setup_host(C.byref(M), C.byref(mg_amg_default_options(**amg)), C.byref(h)))
        self.h = h.value
        self.levels = load().mg_amg_host_levels(self.h)

    def size(self, level: int) -> int:
        return load().mg_amg_host_size(self.h, level)

    def aggregates(self, level: int) -> np.ndarray:
        out = np.empty(self.size(level), dtype=np.int32)
        _check(load().mg_amg_host_aggregates(self.h, level, out.ctypes.data))
        return out

    def get(self, level: int, which: int):
        """(indptr, indices, data) of A_level (MPCG_AMG_A) or P_level (MPCG_AMG_P)."""
        nnz = load().mg_amg_host_nnz(self.h, level, which)
        if nnz < 0:
            raise MpcgError(MPCG_ERR_ARG, "bad level or matrix")
        rp = np.empty(self.size(level) + 1, dtype=np.int32)
        ci = np.empty(nnz, dtype=np.int32)
        va = np.empty(nnz, dtype=np.float64)
        _check(load().mg_amg_host_get(self.h, level, which, rp.ctypes.data, ci.ctypes.data, va.ctypes.data))
        return rp, ci, va

    def ell(self, level: int, which: int):
        """(lg, sptr, col, val): the sliced-ELLPACK arrays the device reads for
        A_level, P_level or R_level (MPCG_AMG_R)."""
        ne = load().mg_amg_host_ell_entries(self.h, level, which)
        if ne < 0:
            raise MpcgError(MPCG_ERR_ARG, "bad level or matrix")
        rows = {MPCG_AMG_A: self.size(level), MPCG_AMG_P: self.size(level),
                MPCG_AMG_R: self.size(level - 1) if level >= 1 else 0}[which]
        lg, ns = C.c_int(), C.c_int()
        sptr = np.empty(rows + 2, dtype=np.int32)     # >= nslices + 1 for any lane count
        col = np.empty(ne, dtype=np.int32)
        val = np.empty(ne, dtype=np.float64)
        _check(load().mg_amg_host_ell(self.h, level, which, C.byref(lg), C.byref(ns), sptr.ctypes.data,
                                      col.ctypes.data, val.ctypes.data))
        return lg.value, sptr[:ns.value + 1].copy(), col, val

    def close(self):
        if self.h:
            load().mg_amg_host_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AlgebraicHierarchy:
    """Owning wrapper of an algebraic hierarchy handle built from a host CSR
    matrix (anything with indptr / indices / data, e.g. scipy.sparse.csr_matrix)."""

    def __init__(self, A, theta=None, w=None, max_levels=None, coarse_size=None, **options):
        amg = {k: v for k, v in dict(theta=theta, w=w, max_levels=max_levels, coarse_size=coarse_size).items()
               if v is not None}
        self.amg = mg_amg_default_options(**amg)
        self.options = mpcg_default_options(**options)
        self.h = mg_hierarchy_setup_algebraic(A.indptr, A.indices, A.data, self.amg, self.options)
        self.levels = mg_num_levels(self.h)

    def solve(self, b, x, rtol=1e-8, maxit=500, histories=True):
        return mpcg_solve(self.h, b, x, rtol, maxit, histories)

    def close(self):
        if self.h:
            mg_hierarchy_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hierarchy:
    """Owning wrapper of a hierarchy handle (torch tensors for device memory)."""

    def __init__(self, stencil_dev, dim: int, nodes: int, levels: int, dofs_per_node: int = 1,
                 faces: int = MPCG_ALL_FACES, **options):
        self.options = mpcg_default_options(**options)
        self.dim, self.nodes, self.levels = dim, nodes, levels
        self._keep = stencil_dev
        self.h = mg_hierarchy_setup(stencil_dev, dim, nodes, levels, self.options, dofs_per_node, faces)

    def solve(self, b, x, rtol=1e-8, maxit=500, histories=True):
        return mpcg_solve(self.h, b, x, rtol, maxit, histories)

    def close(self):
        if self.h:
            mg_hierarchy_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
