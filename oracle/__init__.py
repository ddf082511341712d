"""FP64 CPU oracle for the connectivity-aware multi-level FEM (arXiv 1505.03615).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the GPU library (``paper_1505_03615_gb300``) and never imports it.

The arithmetic lives in ``lbmg_oracle.c`` (plain C, FP64); this module only
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbmg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, FP64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P = C.c_void_p
    i, l, d = C.c_int, C.c_long, C.c_double
    sig = {
        "orc_build": (P, [P, i, P, i, i, i, i, i]),
        "orc_build_embedded": (P, [P, i, P, i, i, i, i, i, d, P]),
        "orc_free": (None, [P]),
        "orc_depth": (i, [P]),
        "orc_min_depth": (i, [P]),
        "orc_cube_side": (d, [P]),
        "orc_center": (None, [P, P]),
        "orc_ndof": (i, [P, i]),
        "orc_nfrag": (i, [P, i]),
        "orc_nnz": (l, [P, i]),
        "orc_prolong_nnz": (l, [P, i]),
        "orc_dofs": (None, [P, i, P, P]),
        "orc_ncorner_tri": (i, [P, i]),
        "orc_corner_tri": (None, [P, i, P, P, P]),
        "orc_fragments": (None, [P, i, P, P, P]),
        "orc_matrices": (None, [P, i, P, P, P, P]),
        "orc_mass_weighted": (None, [P, i, P, P]),
        "orc_prolongation": (None, [P, i, P, P, P]),
        "orc_check_nesting": (l, [P]),
        "orc_project_rhs": (None, [P, P, i, P]),
        "orc_project_rhs_weighted": (None, [P, P, i, P, P]),
        "orc_eval_vertices": (None, [P, P, i, P]),
        "orc_solve": (i, [P, d, P, P, i, d, i, i, i, P]),
        "orc_vcycles": (i, [P, d, P, P, i, i, i, i]),
        "orc_cycles": (i, [P, d, P, P, i, i, i, i, i, i, i]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def embedding_of(V):
    """The default embedding (reading A5): cube side 1.1 x the largest extent of the bounding
    box, centred on it; returns (S, centre) for Hierarchy(..., embedding=...)."""
    V = np.asarray(V, dtype=np.float64)
    mn, mx = V.min(axis=0), V.max(axis=0)
    return 1.1 * float((mx - mn).max()), 0.5 * (mn + mx)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Hierarchy:
    """Oracle hierarchy of the split B-spline space on a mesh (Sections 3-4).

    Levels run from ``min_depth`` (coarsest) to ``depth`` (finest).  With
    ``min_depth < 0`` the coarsest level is the first one, going down from the
    finest, with at most ``coarse_max`` functions.  ``split=False`` gives the
    connectivity-unaware space of Section 3.2 for comparison.  ``embedding =
    (S, center)`` fixes the grid cube (side S, centre) instead of fitting it to
    the bounding box, so that a piece of a mesh lies on the whole mesh's grid.
    """

    def __init__(self, V, F, depth, min_depth=-1, coarse_max=4096, split=True, embedding=None):
        lib = _load()
        self._V = np.ascontiguousarray(V, dtype=np.float64)
        self._F = np.ascontiguousarray(F, dtype=np.int32)
        if embedding is None:
            h = lib.orc_build(_ptr(self._V), self._V.shape[0], _ptr(self._F), self._F.shape[0],
                              int(depth), int(min_depth), int(coarse_max), int(bool(split)))
        else:
            S, c = embedding
            c = np.ascontiguousarray(c, dtype=np.float64)
            h = lib.orc_build_embedded(_ptr(self._V), self._V.shape[0], _ptr(self._F), self._F.shape[0],
                                       int(depth), int(min_depth), int(coarse_max), int(bool(split)),
                                       float(S), _ptr(c))
        if not h:
            raise ValueError("oracle: invalid mesh or depth")
        self._h = h
        self._lib = lib
        self.depth = lib.orc_depth(h)
        self.min_depth = lib.orc_min_depth(h)
        self.cube_side = lib.orc_cube_side(h)
        c = np.zeros(3)
        lib.orc_center(h, _ptr(c))
        self.center = c
        self.nv = self._V.shape[0]

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.orc_free(self._h)
            self._h = None

    def levels(self):
        return list(range(self.min_depth, self.depth + 1))

    def ndof(self, d):
        return self._lib.orc_ndof(self._h, d)

    def nfrag(self, d):
        return self._lib.orc_nfrag(self._h, d)

    def dofs(self, d):
        """(corner index triples [n,3], smallest triangle of each component [n])."""
        n = self.ndof(d)
        corner = np.zeros((n, 3), np.int32)
        mintri = np.zeros(n, np.int32)
        self._lib.orc_dofs(self._h, d, _ptr(corner), _ptr(mintri))
        return corner, mintri

    def corner_tri(self, d):
        """Membership table: (corner key, triangle, dof) for every triangle of every support."""
        m = self._lib.orc_ncorner_tri(self._h, d)
        key = np.zeros(m, np.int64)
        tri = np.zeros(m, np.int32)
        dof = np.zeros(m, np.int32)
        self._lib.orc_corner_tri(self._h, d, _ptr(key), _ptr(tri), _ptr(dof))
        return key, tri, dof

    def fragments(self, d):
        """(triangle [nf], voxel [nf,3], physical area [nf]) of each triangle/voxel piece."""
        nf = self.nfrag(d)
        tri = np.zeros(nf, np.int32)
        vox = np.zeros((nf, 3), np.int32)
        area = np.zeros(nf)
        self._lib.orc_fragments(self._h, d, _ptr(tri), _ptr(vox), _ptr(area))
        return tri, vox, area

    def matrices(self, d):
        """Mass and stiffness matrices of level d as scipy CSR (M, L)."""
        import scipy.sparse as sp
        n = self.ndof(d)
        nnz = self._lib.orc_nnz(self._h, d)
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(nnz, np.int32)
        M = np.zeros(nnz)
        L = np.zeros(nnz)
        self._lib.orc_matrices(self._h, d, _ptr(rp), _ptr(ci), _ptr(M), _ptr(L))
        return sp.csr_matrix((M, ci, rp), shape=(n, n)), sp.csr_matrix((L, ci, rp), shape=(n, n))

    def mass_weighted(self, d, w_tri):
        """M_ij = sum_T w_T int_T b_i b_j at level d (one weight per triangle; Section 5.3 M_t),
        scipy CSR in the pattern of matrices(d)."""
        import scipy.sparse as sp
        n = self.ndof(d)
        nnz = self._lib.orc_nnz(self._h, d)
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(nnz, np.int32)
        self._lib.orc_matrices(self._h, d, _ptr(rp), _ptr(ci), None, None)
        w = np.ascontiguousarray(w_tri, dtype=np.float64)
        if w.shape != (self._F.shape[0],):
            raise ValueError("one weight per triangle expected")
        M = np.zeros(nnz)
        self._lib.orc_mass_weighted(self._h, d, _ptr(w), _ptr(M))
        return sp.csr_matrix((M, ci, rp), shape=(n, n))

    def prolongation(self, d):
        """P from level d-1 to level d as scipy CSR of shape (n_d, n_{d-1})."""
        import scipy.sparse as sp
        n = self.ndof(d)
        nc = self.ndof(d - 1)
        nnz = self._lib.orc_prolong_nnz(self._h, d)
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(nnz, np.int32)
        v = np.zeros(nnz)
        self._lib.orc_prolongation(self._h, d, _ptr(rp), _ptr(ci), _ptr(v))
        return sp.csr_matrix((v, ci, rp), shape=(n, nc))

    def check_nesting(self):
        """Number of violations of the Observation of Section 4.1 (0 expected)."""
        return self._lib.orc_check_nesting(self._h)

    def project_rhs(self, f_vertex):
        """int f b_i over the finest level, f linear per triangle; returns [n_D, nrhs]."""
        f = np.ascontiguousarray(f_vertex, dtype=np.float64)
        if f.ndim == 1:
            f = f[:, None]
        out = np.zeros((self.ndof(self.depth), f.shape[1]))
        self._lib.orc_project_rhs(self._h, _ptr(f), f.shape[1], _ptr(out))
        return out

    def project_rhs_weighted(self, f_vertex, w_tri):
        """int f b_i with triangle T's area element scaled by w_T (the M_t u_t of Section 5.3)."""
        f = np.ascontiguousarray(f_vertex, dtype=np.float64)
        if f.ndim == 1:
            f = f[:, None]
        w = np.ascontiguousarray(w_tri, dtype=np.float64)
        if w.shape != (self._F.shape[0],):
            raise ValueError("one weight per triangle expected")
        out = np.zeros((self.ndof(self.depth), f.shape[1]))
        self._lib.orc_project_rhs_weighted(self._h, _ptr(f), f.shape[1], _ptr(w), _ptr(out))
        return out

    def cmcf_step(self, X, delta):
        """One step of conformalized mean-curvature flow (Section 5.3) on the build-time space:
        solve (M_t + delta L_0) x = M_t u_t, where u_t are the current vertex positions X
        (linear per triangle), M_t weighs each triangle by its current over its build-time
        area and L_0 is the build-time stiffness; returns the new vertex positions.  The
        linear system is solved directly (FP64 sparse LU)."""
        import scipy.sparse.linalg as spla
        X = np.ascontiguousarray(X, dtype=np.float64)

        def areas(P):
            e1 = P[self._F[:, 1]] - P[self._F[:, 0]]
            e2 = P[self._F[:, 2]] - P[self._F[:, 0]]
            return 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1)

        w = areas(X) / areas(self._V)
        D = self.depth
        _, L0 = self.matrices(D)
        A = (self.mass_weighted(D, w) + delta * L0).tocsc()
        x = spla.splu(A).solve(self.project_rhs_weighted(X, w))
        return self.eval_vertices(x)

    def eval_vertices(self, x):
        """u(v) = sum_i x_i b_i(v) at every mesh vertex; x is [n_D, nrhs]."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        if x.ndim == 1:
            x = x[:, None]
        out = np.zeros((self.nv, x.shape[1]))
        self._lib.orc_eval_vertices(self._h, _ptr(x), x.shape[1], _ptr(out))
        return out

    def solve(self, t, rhs, x0=None, tol=1e-10, max_cycles=100, nu1=2, nu2=2):
        """V-cycles on (M + t L) x = rhs to relative residual tol; returns (x, cycles, history)."""
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        if rhs.ndim == 1:
            rhs = rhs[:, None]
        x = np.zeros_like(rhs) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).copy()
        hist = np.zeros((max_cycles + 1, rhs.shape[1]))
        c = self._lib.orc_solve(self._h, float(t), _ptr(rhs), _ptr(x), rhs.shape[1], float(tol),
                                int(max_cycles), int(nu1), int(nu2), _ptr(hist))
        if c < 0:
            raise RuntimeError("oracle: coarse Cholesky failed")
        return x, c, hist[: c + 1]

    def vcycles(self, t, rhs, x0=None, cycles=1, nu1=2, nu2=2):
        """Exactly `cycles` V-cycles per right-hand side (used for timing)."""
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        if rhs.ndim == 1:
            rhs = rhs[:, None]
        x = np.zeros_like(rhs) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).copy()
        rc = self._lib.orc_vcycles(self._h, float(t), _ptr(rhs), _ptr(x), rhs.shape[1], int(cycles),
                                   int(nu1), int(nu2))
        if rc != 0:
            raise RuntimeError("oracle: coarse Cholesky failed")
        return x

    def cycles(self, t, rhs, x0=None, cycles=1, nu1=2, nu2=2, gamma=1, coloured=False, coarse_smooth=False):
        """Exactly `cycles` multigrid cycles (Section 4.3) per right-hand side on (M + t L) x = rhs:
        gamma 1 = V-cycle, 2 = W-cycle; coloured Gauss-Seidel (colours 0..7 down, 7..0 up, the
        order of the GPU cycle) or lexicographic; the coarsest level solved directly or, with
        coarse_smooth, relaxed by nu1 + nu2 sweeps (the min-depth experiment of Section 5.2)."""
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        if rhs.ndim == 1:
            rhs = rhs[:, None]
        x = np.zeros_like(rhs) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).copy()
        if x.ndim == 1:
            x = x[:, None]
        rc = self._lib.orc_cycles(self._h, float(t), _ptr(rhs), _ptr(x), rhs.shape[1], int(cycles), int(nu1),
                                  int(nu2), int(gamma), int(bool(coloured)), int(bool(coarse_smooth)))
        if rc != 0:
            raise RuntimeError("oracle: bad cycle options or coarse Cholesky failed")
        return x
