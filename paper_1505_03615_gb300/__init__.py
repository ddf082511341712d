"""Python binding of liblbmg, the GB300 library for the connectivity-aware
multi-level finite-element system of Chuang & Kazhdan (arXiv 1505.03615).

Every function here has the name of a C entry point in ``include/lbmg.h`` and
only marshals arguments: numpy arrays and torch tensors are passed as raw
pointers (host or device), torch streams as ``cudaStream_t``.  All arithmetic
runs in the library's CUDA kernels; there is no fallback: if the shared
library is missing or fails to load, importing the functions raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = [
    "LbmgError", "Options", "Stats", "load_library", "exported_symbols",
    "LBMG_OK", "LBMG_NOT_CONVERGED", "LBMG_DEVICE_TIMEOUT", "LBMG_FP64", "LBMG_MIXED", "LBMG_GS_COLOURED", "LBMG_JACOBI",
    "lbmg_build_hierarchy", "lbmg_destroy", "lbmg_levels", "lbmg_level_info", "lbmg_embedding",
    "lbmg_assemble", "lbmg_set_area_weights", "lbmg_project_rhs", "lbmg_solve", "lbmg_vcycles", "lbmg_residual", "lbmg_smooth",
    "lbmg_restrict", "lbmg_prolong_add", "lbmg_eval_vertices", "lbmg_get_dofs", "lbmg_get_matrix",
    "lbmg_get_prolongation", "lbmg_launch_counts", "lbmg_build_batch", "lbmg_instances", "lbmg_instance_info",
    "lbmg_instance_residuals", "lbmg_row_instances", "lbmg_learned_nparams", "lbmg_learned_params", "lbmg_learned_collect",
    "lbmg_learned_loss_grad", "lbmg_learned_train", "lbmg_learned_enable", "lbmg_learned_apply",
    "lbmg_learned_state", "lbmg_residual_split",
    "lbmg_residual_norms_noalloc", "lbmg_status_string", "lbmg_last_cuda_error", "lbmg_default_options",
    "lbmg_solve_pcg", "lbmg_cmcf_step", "lbmg_eigs", "lbmg_autotune", "lbmg_launch_shape", "lbmg_tuned_times", "lbmg_set_launch_shape", "lbmg_set_host_check", "lbmg_tune_cache_save", "lbmg_tune_cache_load",
    "lbmg_host_build", "lbmg_host_destroy", "lbmg_host_levels", "lbmg_host_level_info", "lbmg_host_get_dofs",
    "lbmg_host_get_pattern", "lbmg_host_get_prolongation", "lbmg_host_build_batch", "lbmg_host_instances",
    "lbmg_host_row_instances",
]

LBMG_OK = 0
LBMG_NOT_CONVERGED = 4
LBMG_DEVICE_TIMEOUT = 9
LBMG_FP64 = 0
LBMG_MIXED = 1
LBMG_GS_COLOURED = 0
LBMG_JACOBI = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


class LbmgError(RuntimeError):
    def __init__(self, code, where):
        msg = f"{where}: {_lib.lbmg_status_string(code).decode()} ({code})" if _lib else f"{where}: status {code}"
        if _lib is not None and (code == 7 or where.startswith(("lbmg_build", "lbmg_host_build"))):
            detail = _lib.lbmg_last_cuda_error().decode()
            if detail:
                msg += " -- " + detail
        super().__init__(msg)
        self.code = code


class Options(C.Structure):
    _fields_ = [("min_depth", C.c_int), ("coarse_max", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("smoother", C.c_int), ("jacobi_omega", C.c_double), ("split", C.c_int), ("threads", C.c_int),
                ("persistent", C.c_int), ("narrow_max", C.c_int), ("barrier_phantoms", C.c_int),
                ("use_graphs", C.c_int), ("pdl", C.c_int), ("copy_phantom_bytes", C.c_int),
                ("host_alloc_fail", C.c_int), ("host_check", C.c_int), ("cycle", C.c_int),
                ("coarse_smooth", C.c_int), ("gpu_clip", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("converged", C.c_int), ("rel_residual", C.c_double * 4),
                ("initial_residual", C.c_double * 4), ("ms_total", C.c_float), ("ms_fine_smooth", C.c_float),
                ("learned", C.c_int), ("learned_fallback", C.c_int), ("host_syncs", C.c_int)]


def load_library():
    """Load (building first if needed) paper_1505_03615_gb300/_build/liblbmg.so."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    path = _build.build()
    lib = C.CDLL(path)
    P, i, l, d = C.c_void_p, C.c_int, C.c_long, C.c_double
    sig = {
        "lbmg_status_string": (C.c_char_p, [i]),
        "lbmg_last_cuda_error": (C.c_char_p, []),
        "lbmg_default_options": (None, [P]),
        "lbmg_build_hierarchy": (i, [P, i, P, i, i, P, P]),
        "lbmg_destroy": (None, [P]),
        "lbmg_levels": (i, [P, P, P]),
        "lbmg_level_info": (i, [P, i, P, P, P]),
        "lbmg_embedding": (i, [P, P, P]),
        "lbmg_assemble": (i, [P, d, P]),
        "lbmg_set_area_weights": (i, [P, P, P]),
        "lbmg_project_rhs": (i, [P, P, i, P, P]),
        "lbmg_solve": (i, [P, P, P, i, d, i, i, P, P]),
        "lbmg_solve_pcg": (i, [P, P, P, i, d, i, i, P, P]),
        "lbmg_vcycles": (i, [P, P, P, i, i, i, P]),
        "lbmg_residual": (i, [P, i, P, P, P, i, P]),
        "lbmg_residual_split": (i, [P, i, P, P, P, i, P]),
        "lbmg_smooth": (i, [P, i, P, P, i, i, i, P]),
        "lbmg_restrict": (i, [P, i, P, P, i, P]),
        "lbmg_prolong_add": (i, [P, i, P, P, i, P]),
        "lbmg_eval_vertices": (i, [P, P, i, P, P]),
        "lbmg_get_dofs": (i, [P, i, P, P]),
        "lbmg_launch_counts": (i, [P, i, P, P, P, P]),
        "lbmg_autotune": (i, [P, i, i, i, P, P]),
        "lbmg_launch_shape": (i, [P, i, i, P]),
        "lbmg_tuned_times": (i, [P, i, i, P]),
        "lbmg_set_launch_shape": (i, [P, i, i, i, i, i]),
        "lbmg_set_host_check": (i, [P, i]),
        "lbmg_cmcf_step": (i, [P, P, d, P, d, i, i, i, P, P, P]),
        "lbmg_eigs": (i, [P, i, d, i, P, P, P, P, P, P]),
        "lbmg_tune_cache_save": (i, [C.c_char_p]),
        "lbmg_tune_cache_load": (i, [C.c_char_p]),
        "lbmg_get_matrix": (i, [P, i, P, P, P, P]),
        "lbmg_get_prolongation": (i, [P, i, P, P]),
        "lbmg_build_batch": (i, [P, P, P, P, P, i, P, P]),
        "lbmg_instances": (i, [P, P]),
        "lbmg_instance_info": (i, [P, i, P, P, P, P, P]),
        "lbmg_instance_residuals": (i, [P, i, P]),
        "lbmg_row_instances": (i, [P, i, P]),
        "lbmg_learned_nparams": (i, []),
        "lbmg_learned_params": (i, [P, P, P, P]),
        "lbmg_learned_collect": (i, [P, P, i, i, i, P]),
        "lbmg_learned_loss_grad": (i, [P, P, i, P, P, P]),
        "lbmg_learned_train": (i, [P, i, d, P, i, P, P]),
        "lbmg_learned_enable": (i, [P, i, P]),
        "lbmg_learned_apply": (i, [P, P, i, i, P, P, P]),
        "lbmg_learned_state": (i, [P, P, P, P]),
        "lbmg_residual_norms_noalloc": (i, [P, i, P, P, i, P, P]),
        "lbmg_host_build": (i, [P, i, P, i, i, P, P]),
        "lbmg_host_destroy": (None, [P]),
        "lbmg_host_levels": (i, [P, P, P]),
        "lbmg_host_level_info": (i, [P, i, P, P, P]),
        "lbmg_host_get_dofs": (i, [P, i, P, P]),
        "lbmg_host_get_pattern": (i, [P, i, P, P]),
        "lbmg_host_get_prolongation": (i, [P, i, P, P]),
        "lbmg_host_build_batch": (i, [P, P, P, P, P, i, P, P]),
        "lbmg_host_instances": (i, [P, P, P, P]),
        "lbmg_host_row_instances": (i, [P, i, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names declared in include/lbmg.h (parsed from the header)."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "lbmg.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"\b(lbmg_[a-z_0-9]+)\s*\(", text)))


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return C.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return C.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported argument type {type(a)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _nrhs(a):
    return 1 if len(a.shape) == 1 else int(a.shape[1])


def _check(code, where, allow=()):
    if code != LBMG_OK and code not in allow:
        raise LbmgError(code, where)
    return code


def lbmg_status_string(code):
    return load_library().lbmg_status_string(int(code)).decode()


def lbmg_last_cuda_error():
    return load_library().lbmg_last_cuda_error().decode()


def lbmg_default_options():
    o = Options()
    load_library().lbmg_default_options(C.byref(o))
    return o


def lbmg_build_hierarchy(V, F, depth, **opts):
    """Build the hierarchy; V float64 [nv,3], F int32 [nt,3] on the host.  Returns the handle."""
    lib = load_library()
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    o = lbmg_default_options()
    for k, v in opts.items():
        setattr(o, k, v)
    h = C.c_void_p()
    _check(lib.lbmg_build_hierarchy(_ptr(V), V.shape[0], _ptr(F), F.shape[0], int(depth), C.byref(o), C.byref(h)),
           "lbmg_build_hierarchy")
    return h


def lbmg_build_batch(meshes, **opts):
    """Build one hierarchy for a list of (V, F, depth) meshes solved together.  Returns the handle."""
    lib = load_library()
    Vs = [np.ascontiguousarray(V, dtype=np.float64) for V, _, _ in meshes]
    Fs = [np.ascontiguousarray(F, dtype=np.int32) for _, F, _ in meshes]
    n = len(meshes)
    Vp = (C.c_void_p * n)(*[V.ctypes.data for V in Vs])
    Fp = (C.c_void_p * n)(*[F.ctypes.data for F in Fs])
    nv = (C.c_int * n)(*[V.shape[0] for V in Vs])
    nt = (C.c_int * n)(*[F.shape[0] for F in Fs])
    dp = (C.c_int * n)(*[int(d) for _, _, d in meshes])
    o = lbmg_default_options()
    for k, v in opts.items():
        setattr(o, k, v)
    h = C.c_void_p()
    _check(lib.lbmg_build_batch(Vp, nv, Fp, nt, dp, n, C.byref(o), C.byref(h)), "lbmg_build_batch")
    return h


def lbmg_instances(h):
    n = C.c_int()
    _check(load_library().lbmg_instances(h, C.byref(n)), "lbmg_instances")
    return n.value


def lbmg_instance_info(h, inst):
    """(depth, min_depth, finest functions, row offset in finest vectors, vertex offset)."""
    d, d0 = C.c_int(), C.c_int()
    nf, ro, vo = C.c_long(), C.c_long(), C.c_long()
    _check(load_library().lbmg_instance_info(h, int(inst), C.byref(d), C.byref(d0), C.byref(nf), C.byref(ro),
                                             C.byref(vo)), "lbmg_instance_info")
    return d.value, d0.value, nf.value, ro.value, vo.value


def lbmg_instance_residuals(h, nrhs):
    n = lbmg_instances(h)
    out = np.zeros((n, nrhs))
    _check(load_library().lbmg_instance_residuals(h, int(nrhs), _ptr(out)), "lbmg_instance_residuals")
    return out


def lbmg_row_instances(h, d):
    """The mesh of every row of level d (device dof order)."""
    n, _, _ = lbmg_level_info(h, d)
    inst = np.zeros(n, np.int32)
    _check(load_library().lbmg_row_instances(h, int(d), _ptr(inst)), "lbmg_row_instances")
    return inst


def lbmg_learned_nparams():
    return load_library().lbmg_learned_nparams()


def lbmg_learned_params(h, set_params=None, stream=None):
    """Set (if given, flat float64; resets Adam) and return the flat parameters W1 [32][64], b1, w2, b2."""
    P = lbmg_learned_nparams()
    out = np.zeros(P)
    s = None if set_params is None else np.ascontiguousarray(set_params, dtype=np.float64)
    if s is not None and s.size != P:
        raise ValueError(f"expected {P} parameters")
    _check(load_library().lbmg_learned_params(h, _ptr(out), _ptr(s), _stream(stream)), "lbmg_learned_params")
    return out


def lbmg_learned_collect(h, rhs, skip, keep, stream=None):
    return _check(load_library().lbmg_learned_collect(h, _ptr(rhs), _nrhs(rhs), int(skip), int(keep), _stream(stream)),
                  "lbmg_learned_collect")


def lbmg_learned_loss_grad(h, r0, stream=None, grad=True):
    P = lbmg_learned_nparams()
    loss = C.c_double()
    g = np.zeros(P) if grad else None
    _check(load_library().lbmg_learned_loss_grad(h, _ptr(r0), _nrhs(r0), C.byref(loss), _ptr(g), _stream(stream)),
           "lbmg_learned_loss_grad")
    return loss.value, g


def lbmg_learned_train(h, order, lr, stream=None):
    order = np.ascontiguousarray(order, dtype=np.int32)
    steps, batch = order.shape
    hist = np.zeros(steps)
    _check(load_library().lbmg_learned_train(h, int(steps), float(lr), _ptr(order), int(batch), _ptr(hist),
                                             _stream(stream)), "lbmg_learned_train")
    return hist


def lbmg_learned_enable(h, on=True, stream=None):
    return _check(load_library().lbmg_learned_enable(h, int(bool(on)), _stream(stream)), "lbmg_learned_enable")


def lbmg_learned_state(h, set_state=None, stream=None):
    """Set (if given) and return the optimiser state: parameters, Adam moments, step count."""
    P = lbmg_learned_nparams()
    out = np.zeros(3 * P + 1)
    st = None if set_state is None else np.ascontiguousarray(set_state, dtype=np.float64)
    if st is not None and st.size != 3 * P + 1:
        raise ValueError(f"expected {3 * P + 1} values")
    _check(load_library().lbmg_learned_state(h, _ptr(out), _ptr(st), _stream(stream)), "lbmg_learned_state")
    return out


def lbmg_learned_apply(h, r, precision, omega, delta, stream=None):
    """The solve's correction of the residual r (device [n][ns]): omega [n] and delta [n][ns] (device)."""
    return _check(load_library().lbmg_learned_apply(h, _ptr(r), _nrhs(r), int(precision), _ptr(omega), _ptr(delta),
                                                    _stream(stream)), "lbmg_learned_apply")


def lbmg_destroy(h):
    load_library().lbmg_destroy(h)


def lbmg_levels(h):
    a, b = C.c_int(), C.c_int()
    _check(load_library().lbmg_levels(h, C.byref(a), C.byref(b)), "lbmg_levels")
    return a.value, b.value


def lbmg_level_info(h, d):
    n, z, f = C.c_long(), C.c_long(), C.c_long()
    _check(load_library().lbmg_level_info(h, int(d), C.byref(n), C.byref(z), C.byref(f)), "lbmg_level_info")
    return n.value, z.value, f.value


def lbmg_embedding(h):
    s = C.c_double()
    c = np.zeros(3)
    _check(load_library().lbmg_embedding(h, C.byref(s), _ptr(c)), "lbmg_embedding")
    return s.value, c


def lbmg_assemble(h, t, stream=None):
    return _check(load_library().lbmg_assemble(h, float(t), _stream(stream)), "lbmg_assemble")


def lbmg_set_area_weights(h, w_tri=None, stream=None):
    """Per-triangle area weights of the mass matrix and the right-hand side (host float64 [nt]);
    None restores the build-time metric."""
    w = None if w_tri is None else np.ascontiguousarray(w_tri, dtype=np.float64)
    return _check(load_library().lbmg_set_area_weights(h, _ptr(w), _stream(stream)), "lbmg_set_area_weights")


def lbmg_project_rhs(h, f_vertex, rhs, stream=None):
    return _check(load_library().lbmg_project_rhs(h, _ptr(f_vertex), _nrhs(f_vertex), _ptr(rhs), _stream(stream)),
                  "lbmg_project_rhs")


def lbmg_solve(h, rhs, x, tol, max_cycles, precision, stream=None, raise_not_converged=False):
    """Returns (status, Stats); status is LBMG_OK or LBMG_NOT_CONVERGED."""
    st = Stats()
    code = load_library().lbmg_solve(h, _ptr(rhs), _ptr(x), _nrhs(rhs), float(tol), int(max_cycles), int(precision),
                                     C.byref(st), _stream(stream))
    _check(code, "lbmg_solve", allow=() if raise_not_converged else (LBMG_NOT_CONVERGED, LBMG_DEVICE_TIMEOUT))
    return code, st


def lbmg_solve_pcg(h, rhs, x, tol, max_iters, precision, stream=None, raise_not_converged=False):
    """V-cycle-preconditioned conjugate gradients; returns (status, Stats) like lbmg_solve."""
    st = Stats()
    code = load_library().lbmg_solve_pcg(h, _ptr(rhs), _ptr(x), _nrhs(rhs), float(tol), int(max_iters),
                                         int(precision), C.byref(st), _stream(stream))
    _check(code, "lbmg_solve_pcg", allow=() if raise_not_converged else (LBMG_NOT_CONVERGED, LBMG_DEVICE_TIMEOUT))
    return code, st


def lbmg_cmcf_step(h, X, delta, x, tol, max_cycles, precision, X_next, solver=0, stream=None):
    """One conformalized mean-curvature-flow step (device tensors X [nv,3], x [n,3] in/out,
    X_next [nv,3]); returns (status, Stats) like lbmg_solve."""
    st = Stats()
    code = load_library().lbmg_cmcf_step(h, _ptr(X), float(delta), _ptr(x), float(tol), int(max_cycles),
                                         int(precision), int(solver), _ptr(X_next), C.byref(st), _stream(stream))
    _check(code, "lbmg_cmcf_step", allow=(LBMG_NOT_CONVERGED,))
    return code, st


def lbmg_eigs(h, X0, tol, max_iters, X=None, stream=None):
    """The k = X0.shape[1] smallest eigenpairs of L x = lambda M x (device tensors X0 [n,k] and X);
    returns (status, lambda [k], residuals [k], iterations)."""
    k = X0.shape[1]
    X = X0 if X is None else X
    lam = np.zeros(k)
    res = np.zeros(k)
    its = C.c_int(0)
    code = load_library().lbmg_eigs(h, int(k), float(tol), int(max_iters), _ptr(X0), _ptr(lam), _ptr(X), _ptr(res),
                                    C.byref(its), _stream(stream))
    _check(code, "lbmg_eigs", allow=(LBMG_NOT_CONVERGED,))
    return code, lam, res, its.value


def lbmg_vcycles(h, rhs, x, cycles, precision, stream=None):
    return _check(load_library().lbmg_vcycles(h, _ptr(rhs), _ptr(x), _nrhs(rhs), int(cycles), int(precision),
                                              _stream(stream)), "lbmg_vcycles")


def lbmg_residual(h, d, rhs, x, r, stream=None):
    return _check(load_library().lbmg_residual(h, int(d), _ptr(rhs), _ptr(x), _ptr(r), _nrhs(rhs), _stream(stream)),
                  "lbmg_residual")


def lbmg_residual_norms_noalloc(h, d, rhs, x, norms, stream=None):
    """Per-column ||rhs - A_d x||_2 into `norms` (all device tensors); the call allocates nothing."""
    return _check(load_library().lbmg_residual_norms_noalloc(h, int(d), _ptr(rhs), _ptr(x), _nrhs(rhs), _ptr(norms),
                                                             _stream(stream)), "lbmg_residual_norms_noalloc")


def lbmg_residual_split(h, d, rhs, x, r, stream=None):
    """The mixed solve's outer residual (FP64 values as FP32 pairs), same conventions as lbmg_residual."""
    return _check(load_library().lbmg_residual_split(h, int(d), _ptr(rhs), _ptr(x), _ptr(r), _nrhs(rhs),
                                                     _stream(stream)), "lbmg_residual_split")


def lbmg_smooth(h, d, rhs, x, sweeps, precision, stream=None):
    return _check(load_library().lbmg_smooth(h, int(d), _ptr(rhs), _ptr(x), _nrhs(rhs), int(sweeps), int(precision),
                                             _stream(stream)), "lbmg_smooth")


def lbmg_restrict(h, d, r_fine, r_coarse, stream=None):
    return _check(load_library().lbmg_restrict(h, int(d), _ptr(r_fine), _ptr(r_coarse), _nrhs(r_fine),
                                               _stream(stream)), "lbmg_restrict")


def lbmg_prolong_add(h, d, x_coarse, x_fine, stream=None):
    return _check(load_library().lbmg_prolong_add(h, int(d), _ptr(x_coarse), _ptr(x_fine), _nrhs(x_coarse),
                                                  _stream(stream)), "lbmg_prolong_add")


def lbmg_eval_vertices(h, x, u, stream=None):
    return _check(load_library().lbmg_eval_vertices(h, _ptr(x), _nrhs(x), _ptr(u), _stream(stream)),
                  "lbmg_eval_vertices")


def lbmg_launch_counts(h, precision):
    """(assemble, project_rhs, per_cycle, solve_fixed) kernel launch counts."""
    v = [C.c_int() for _ in range(4)]
    _check(load_library().lbmg_launch_counts(h, int(precision), *[C.byref(x) for x in v]), "lbmg_launch_counts")
    return tuple(x.value for x in v)


def lbmg_autotune(h, nrhs, precision, reps=4, stream=None):
    """Tune the launch shapes of every level; returns how many (level, kernel) pairs were timed."""
    n = C.c_int()
    _check(load_library().lbmg_autotune(h, int(nrhs), int(precision), int(reps), C.byref(n), _stream(stream)),
           "lbmg_autotune")
    return n.value


def lbmg_launch_shape(h, d, precision):
    """((sweep threads/row, sweep threads/block), (residual threads/row, residual threads/block)) of level d."""
    out = (C.c_int * 4)()
    _check(load_library().lbmg_launch_shape(h, int(d), int(precision), out), "lbmg_launch_shape")
    return (out[0], out[1]), (out[2], out[3])


def lbmg_tuned_times(h, d, precision):
    """(ms per Gauss-Seidel sweep, ms per residual) the last autotune measured for level d (0: not timed)."""
    out = (C.c_float * 2)()
    _check(load_library().lbmg_tuned_times(h, int(d), int(precision), out), "lbmg_tuned_times")
    return out[0], out[1]


def lbmg_set_launch_shape(h, d, precision, kind, tpr, tpb):
    return _check(load_library().lbmg_set_launch_shape(h, int(d), int(precision), int(kind), int(tpr), int(tpb)),
                  "lbmg_set_launch_shape")


def lbmg_set_host_check(h, on):
    return _check(load_library().lbmg_set_host_check(h, int(on)), "lbmg_set_host_check")


def lbmg_tune_cache_save(path):
    return _check(load_library().lbmg_tune_cache_save(os.fsencode(path)), "lbmg_tune_cache_save")


def lbmg_tune_cache_load(path):
    return _check(load_library().lbmg_tune_cache_load(os.fsencode(path)), "lbmg_tune_cache_load")


def lbmg_get_dofs(h, d):
    n, _, _ = lbmg_level_info(h, d)
    corner = np.zeros((n, 3), np.int32)
    mintri = np.zeros(n, np.int32)
    _check(load_library().lbmg_get_dofs(h, int(d), _ptr(corner), _ptr(mintri)), "lbmg_get_dofs")
    return corner, mintri


def lbmg_get_matrix(h, d):
    n, nnz, _ = lbmg_level_info(h, d)
    rp = np.zeros(n + 1, np.int32)
    ci = np.zeros(nnz, np.int32)
    M = np.zeros(nnz)
    L = np.zeros(nnz)
    _check(load_library().lbmg_get_matrix(h, int(d), _ptr(rp), _ptr(ci), _ptr(M), _ptr(L)), "lbmg_get_matrix")
    return rp, ci, M, L


def lbmg_get_prolongation(h, d):
    n, _, _ = lbmg_level_info(h, d)
    par = np.zeros((n, 8), np.int32)
    w = np.zeros((n, 8))
    _check(load_library().lbmg_get_prolongation(h, int(d), _ptr(par), _ptr(w)), "lbmg_get_prolongation")
    return par, w


def lbmg_host_build(V, F, depth, **opts):
    """Host-only hierarchy (no GPU needed); V float64 [nv,3], F int32 [nt,3].  Returns the host handle."""
    lib = load_library()
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    o = lbmg_default_options()
    for k, v in opts.items():
        setattr(o, k, v)
    h = C.c_void_p()
    _check(lib.lbmg_host_build(_ptr(V), V.shape[0], _ptr(F), F.shape[0], int(depth), C.byref(o), C.byref(h)),
           "lbmg_host_build")
    return h


def lbmg_host_build_batch(meshes, **opts):
    """Host-only batch hierarchy (no GPU needed) of a list of (V, F, depth).  Returns the host handle."""
    lib = load_library()
    Vs = [np.ascontiguousarray(V, dtype=np.float64) for V, _, _ in meshes]
    Fs = [np.ascontiguousarray(F, dtype=np.int32) for _, F, _ in meshes]
    n = len(meshes)
    Vp = (C.c_void_p * n)(*[V.ctypes.data for V in Vs])
    Fp = (C.c_void_p * n)(*[F.ctypes.data for F in Fs])
    nv = (C.c_int * n)(*[V.shape[0] for V in Vs])
    nt = (C.c_int * n)(*[F.shape[0] for F in Fs])
    dp = (C.c_int * n)(*[int(d) for _, _, d in meshes])
    o = lbmg_default_options()
    for k, v in opts.items():
        setattr(o, k, v)
    h = C.c_void_p()
    _check(lib.lbmg_host_build_batch(Vp, nv, Fp, nt, dp, n, C.byref(o), C.byref(h)), "lbmg_host_build_batch")
    return h


def lbmg_host_instances(h):
    """(number of meshes, finest depth per mesh, coarsest depth per mesh)."""
    n = C.c_int()
    _check(load_library().lbmg_host_instances(h, C.byref(n), None, None), "lbmg_host_instances")
    D = np.zeros(n.value, np.int32)
    d0 = np.zeros(n.value, np.int32)
    _check(load_library().lbmg_host_instances(h, C.byref(n), _ptr(D), _ptr(d0)), "lbmg_host_instances")
    return n.value, D, d0


def lbmg_host_row_instances(h, d):
    n, _, _ = lbmg_host_level_info(h, d)
    inst = np.zeros(n, np.int32)
    _check(load_library().lbmg_host_row_instances(h, int(d), _ptr(inst)), "lbmg_host_row_instances")
    return inst


def lbmg_host_destroy(h):
    load_library().lbmg_host_destroy(h)


def lbmg_host_levels(h):
    a, b = C.c_int(), C.c_int()
    _check(load_library().lbmg_host_levels(h, C.byref(a), C.byref(b)), "lbmg_host_levels")
    return a.value, b.value


def lbmg_host_level_info(h, d):
    n, z, f = C.c_long(), C.c_long(), C.c_long()
    _check(load_library().lbmg_host_level_info(h, int(d), C.byref(n), C.byref(z), C.byref(f)),
           "lbmg_host_level_info")
    return n.value, z.value, f.value


def lbmg_host_get_dofs(h, d):
    n, _, _ = lbmg_host_level_info(h, d)
    corner = np.zeros((n, 3), np.int32)
    mintri = np.zeros(n, np.int32)
    _check(load_library().lbmg_host_get_dofs(h, int(d), _ptr(corner), _ptr(mintri)), "lbmg_host_get_dofs")
    return corner, mintri


def lbmg_host_get_pattern(h, d):
    n, nnz, _ = lbmg_host_level_info(h, d)
    rp = np.zeros(n + 1, np.int32)
    ci = np.zeros(nnz, np.int32)
    _check(load_library().lbmg_host_get_pattern(h, int(d), _ptr(rp), _ptr(ci)), "lbmg_host_get_pattern")
    return rp, ci


def lbmg_host_get_prolongation(h, d):
    n, _, _ = lbmg_host_level_info(h, d)
    par = np.zeros((n, 8), np.int32)
    w = np.zeros((n, 8))
    _check(load_library().lbmg_host_get_prolongation(h, int(d), _ptr(par), _ptr(w)), "lbmg_host_get_prolongation")
    return par, w
