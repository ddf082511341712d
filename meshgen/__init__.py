"""Seeded synthetic triangle meshes and right-hand sides.

This module is the one place shared by the FP64 oracle's tests and the GPU
library's tests and benchmark.  It only generates inputs (vertex positions,
triangle indices, per-vertex values); it holds none of the finite-element
method's arithmetic (no embedding, clipping, basis functions or quadrature).

Every generator is deterministic given its ``seed`` (numpy PCG64).  The shapes
stand in for the paper's models (Section 5), which are not available: a jittered
icosphere, torus-knot tubes whose distant segments share coarse voxels, two
parallel displaced sheets half a finest voxel apart, tori and ellipsoids.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "icosphere",
    "ellipsoid",
    "bumpy_sphere",
    "torus",
    "torus_knot_tube",
    "double_sheet",
    "cube_grid",
    "batch_mix",
    "random_start",
    "sphere_harmonic_rhs",
    "uniform_rhs",
    "coordinate_rhs",
    "config_mesh",
    "CONFIGS",
]


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _jitter(V, amount, rng):
    if amount > 0:
        V = V + rng.uniform(-amount, amount, size=V.shape)
    return V


def icosphere(level=3, radius=1.0, jitter=1e-3, seed=1):
    """Icosahedron subdivided ``level`` times, projected to the sphere.

    level 3 gives 642 vertices and 1280 triangles.  Each coordinate is then
    perturbed by U(-jitter, jitter).
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in V]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}
        newF = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]

        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            newF += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = newF
    V = np.array(V) * radius
    V = _jitter(V, jitter, _rng(seed))
    return np.ascontiguousarray(V, dtype=np.float64), np.ascontiguousarray(F, dtype=np.int32)


def bumpy_sphere(level=4, amplitude=0.25, seed=12):
    """A seeded genus-0 surface with bumps of several sizes: the icosphere of the given level
    with radius 1 + amplitude * (sum of three products of sines of the coordinates with seeded
    frequencies 1..4 and phases), normalised to a largest bump of `amplitude`."""
    V, F = icosphere(level=level, radius=1.0, jitter=0.0, seed=seed)
    rng = _rng(seed)
    bump = np.zeros(V.shape[0])
    for _ in range(3):
        k = rng.integers(1, 5, size=3)
        ph = rng.uniform(0, 2 * np.pi, size=3)
        bump += np.prod(np.sin(k[None, :] * np.pi * V + ph[None, :]), axis=1)
    bump *= amplitude / np.abs(bump).max()
    V = V * (1.0 + bump)[:, None]
    return np.ascontiguousarray(V), F


def ellipsoid(axes=(1.0, 0.7, 0.5), level=5, jitter=1e-6, seed=3):
    """Icosphere of the given subdivision level scaled by ``axes``."""
    V, F = icosphere(level=level, radius=1.0, jitter=0.0, seed=seed)
    V = V * np.asarray(axes, dtype=np.float64)[None, :]
    V = _jitter(V, jitter, _rng(seed))
    return np.ascontiguousarray(V), F


def _grid_tris(nu, nv, wrap_u, wrap_v):
    """Two triangles per quad of an nu x nv vertex grid, optionally wrapped."""
    F = []
    iu_max = nu if wrap_u else nu - 1
    iv_max = nv if wrap_v else nv - 1
    for i in range(iu_max):
        i1 = (i + 1) % nu
        for j in range(iv_max):
            j1 = (j + 1) % nv
            a, b, c, d = i * nv + j, i1 * nv + j, i1 * nv + j1, i * nv + j1
            F.append((a, b, c))
            F.append((a, c, d))
    return np.asarray(F, dtype=np.int32)


def torus(R=1.0, r=0.3, n_major=200, n_minor=60, jitter=1e-6, seed=5):
    """Torus of major radius R and tube radius r; 2*n_major*n_minor triangles."""
    u = 2 * np.pi * np.arange(n_major) / n_major
    v = 2 * np.pi * np.arange(n_minor) / n_minor
    U, W = np.meshgrid(u, v, indexing="ij")
    X = (R + r * np.cos(W)) * np.cos(U)
    Y = (R + r * np.cos(W)) * np.sin(U)
    Z = r * np.sin(W)
    V = np.stack([X, Y, Z], axis=-1).reshape(-1, 3)
    F = _grid_tris(n_major, n_minor, True, True)
    V = _jitter(V, jitter, _rng(seed))
    return np.ascontiguousarray(V), F


def torus_knot_tube(p=2, q=3, knot_radius=1.0, tube_radius=0.04, n_seg=1000,
                    n_ring=100, jitter=1e-6, seed=2):
    """Circular tube around the (p, q) torus knot.

    Centre curve: ((R + R/2 cos q phi) cos p phi, (R + R/2 cos q phi) sin p phi,
    R/2 sin q phi) with R = knot_radius.  The ring frame is parallel-transported
    along the closed curve and the closing twist is spread evenly.  The tube has
    n_seg * n_ring * 2 triangles (1000 x 100 x 2 = 200k by default).
    """
    R = knot_radius
    phi = 2 * np.pi * np.arange(n_seg) / n_seg
    rr = R + 0.5 * R * np.cos(q * phi)
    C = np.stack([rr * np.cos(p * phi), rr * np.sin(p * phi), 0.5 * R * np.sin(q * phi)], -1)
    T = np.roll(C, -1, 0) - np.roll(C, 1, 0)
    T /= np.linalg.norm(T, axis=1, keepdims=True)
    N = np.zeros_like(C)
    a = np.array([0.0, 0.0, 1.0])
    if abs(T[0] @ a) > 0.9:
        a = np.array([1.0, 0.0, 0.0])
    n0 = a - (a @ T[0]) * T[0]
    N[0] = n0 / np.linalg.norm(n0)
    for i in range(1, n_seg):
        n = N[i - 1] - (N[i - 1] @ T[i]) * T[i]
        N[i] = n / np.linalg.norm(n)
    # closing twist: angle between transported N[n-1]->T[0] and N[0]
    n_end = N[-1] - (N[-1] @ T[0]) * T[0]
    n_end /= np.linalg.norm(n_end)
    B0 = np.cross(T[0], N[0])
    theta = math.atan2(n_end @ B0, n_end @ N[0])
    B = np.cross(T, N)
    ang = -theta * np.arange(n_seg) / n_seg
    N2 = np.cos(ang)[:, None] * N + np.sin(ang)[:, None] * B
    B2 = np.cross(T, N2)
    alpha = 2 * np.pi * np.arange(n_ring) / n_ring
    V = (C[:, None, :]
         + tube_radius * (np.cos(alpha)[None, :, None] * N2[:, None, :]
                          + np.sin(alpha)[None, :, None] * B2[:, None, :]))
    V = V.reshape(-1, 3)
    F = _grid_tris(n_seg, n_ring, True, True)
    V = _jitter(V, jitter, _rng(seed))
    return np.ascontiguousarray(V), F


def double_sheet(n=500, amplitude=0.05, depth=9, offset_voxels=0.5, jitter=1e-6, seed=4):
    """Two copies of a sinusoidally displaced unit square, stacked along z.

    Each sheet is an (n+1) x (n+1) vertex grid over [0,1]^2 (2 n^2 triangles)
    with height amplitude * sin(2 pi (2x) + a) * sin(2 pi (3y) + b) + offset,
    with seeded phases a, b.  The second sheet is the first shifted by
    ``offset_voxels`` finest voxels of a depth-``depth`` grid whose cube side is
    1.1 times the largest extent (1.1 / 2^depth per voxel), so the two sheets
    share every voxel's support at the finest levels but are never connected.
    """
    rng = _rng(seed)
    a, b = rng.uniform(0, 2 * np.pi, size=2)
    x = np.arange(n + 1) / n
    X, Y = np.meshgrid(x, x, indexing="ij")
    Z = amplitude * np.sin(2 * np.pi * 2 * X + a) * np.sin(2 * np.pi * 3 * Y + b)
    V1 = np.stack([X, Y, Z], -1).reshape(-1, 3)
    delta = offset_voxels * 1.1 / (2 ** depth)
    V2 = V1 + np.array([0.0, 0.0, delta])
    F1 = _grid_tris(n + 1, n + 1, False, False)
    V = np.concatenate([V1, V2])
    F = np.concatenate([F1, F1 + V1.shape[0]]).astype(np.int32)
    V = _jitter(V, jitter, rng)
    return np.ascontiguousarray(V), np.ascontiguousarray(F)


def cube_grid(n=6, size=1.0, gap=1.0, subdiv=4, jitter=1e-6, seed=8):
    """n x n x n axis-aligned cubes of side `size`, `gap` apart along every axis (the model of
    equidistantly spaced unit cubes of the convergence experiment, Section 5.2).

    Each cube is a closed surface whose faces are subdiv x subdiv grids of quads, two
    triangles per quad, oriented outwards (12 subdiv^2 triangles per cube).  Every vertex
    is then perturbed by U(-jitter, jitter).
    """
    s = int(subdiv)
    idx = {}
    Vc = []
    for i in range(s + 1):
        for j in range(s + 1):
            for k in range(s + 1):
                if min(i, j, k) == 0 or max(i, j, k) == s:
                    idx[(i, j, k)] = len(Vc)
                    Vc.append((i, j, k))
    Vc = np.asarray(Vc, dtype=np.float64) * (size / s)
    Fc = []
    for axis in range(3):
        a1, a2 = [a for a in range(3) if a != axis]
        for side in (0, s):
            normal = np.zeros(3)
            normal[axis] = 1.0 if side == s else -1.0
            for u in range(s):
                for v in range(s):
                    def key(du, dv):
                        c = [0, 0, 0]
                        c[axis], c[a1], c[a2] = side, u + du, v + dv
                        return idx[tuple(c)]
                    q = (key(0, 0), key(1, 0), key(1, 1), key(0, 1))
                    for tri in ((q[0], q[1], q[2]), (q[0], q[2], q[3])):
                        A, B, C = Vc[list(tri)]
                        if np.cross(B - A, C - A) @ normal < 0:
                            tri = (tri[0], tri[2], tri[1])
                        Fc.append(tri)
    Fc = np.asarray(Fc, dtype=np.int64)
    Vs, Fs = [], []
    pitch = size + gap
    for i in range(n):
        for j in range(n):
            for k in range(n):
                Fs.append(Fc + len(Vs) * Vc.shape[0])
                Vs.append(Vc + pitch * np.array([i, j, k], dtype=np.float64))
    V = _jitter(np.concatenate(Vs), jitter, _rng(seed))
    return np.ascontiguousarray(V), np.ascontiguousarray(np.concatenate(Fs), dtype=np.int32)


def random_start(n, ncols=1, seed=9):
    """Initial coefficients drawn from U[0, 1] (the random initial guess of Section 5.2)."""
    return np.ascontiguousarray(_rng(seed).uniform(0.0, 1.0, size=(n, ncols)))


def batch_mix(count=64, min_tris=10_000, max_tris=300_000, seed=7):
    """Seeded list of (V, F, depth) of uneven size: tori, ellipsoids, torus knots.

    Triangle counts are drawn log-uniformly in [min_tris, max_tris]; depth is
    7 below 100k triangles, 8 below 250k and 9 above, which keeps the 64-mesh
    batch at about 170M stored entries on its finest level (one deeper level per
    mesh would quadruple that).
    """
    rng = _rng(seed)
    out = []
    for i in range(count):
        nt = int(math.exp(rng.uniform(math.log(min_tris), math.log(max_tris))))
        kind = ("torus", "ellipsoid", "knot")[i % 3]
        if kind == "torus":
            nm = max(8, int(math.sqrt(nt / 2 / 0.3)))
            V, F = torus(R=1.0, r=rng.uniform(0.2, 0.45), n_major=nm,
                         n_minor=max(6, int(nt / 2 / nm)), seed=int(rng.integers(1 << 30)))
        elif kind == "ellipsoid":
            level = max(2, int(round(math.log(nt / 20) / math.log(4))))
            V, F = ellipsoid(axes=tuple(rng.uniform(0.4, 1.0, 3)), level=level,
                             seed=int(rng.integers(1 << 30)))
        else:
            pq = [(2, 3), (2, 5), (3, 4), (3, 5)][int(rng.integers(4))]
            ring = 24
            V, F = torus_knot_tube(p=pq[0], q=pq[1], tube_radius=rng.uniform(0.04, 0.08),
                                   n_seg=max(40, nt // (2 * ring)), n_ring=ring,
                                   seed=int(rng.integers(1 << 30)))
        ntr = F.shape[0]
        depth = 7 if ntr < 100_000 else (8 if ntr < 250_000 else 9)
        out.append((V, F, depth))
    return out


def sphere_harmonic_rhs(V, noise=0.01, seed=11):
    """Per-vertex P_3(z/|v|) = z(5z^2-3)/2 (the m=0, l=3 harmonic) plus N(0, noise^2)."""
    z = V[:, 2] / np.linalg.norm(V, axis=1)
    f = 0.5 * z * (5 * z * z - 3)
    f = f + _rng(seed).normal(0.0, noise, size=f.shape)
    return np.ascontiguousarray(f[:, None], dtype=np.float64)


def uniform_rhs(nv, seed=13):
    """Per-vertex values drawn from U[-1, 1], shape (nv, 1)."""
    return np.ascontiguousarray(_rng(seed).uniform(-1, 1, size=(nv, 1)))


def coordinate_rhs(V):
    """Per-vertex x, y, z coordinates as three right-hand sides, shape (nv, 3)."""
    return np.ascontiguousarray(V, dtype=np.float64)


# Named workloads: (mesh builder, depth, screening t, rhs builder, tolerance, precision)
CONFIGS = {
    "icosphere_l3_d5": dict(mesh=lambda: icosphere(3, 1.0, 1e-3, 1), depth=5, t=1e-3,
                            rhs=lambda V: sphere_harmonic_rhs(V), tol=1e-10, precision="fp64"),
    "knot23_200k_d8": dict(mesh=lambda: torus_knot_tube(2, 3, 1.0, 0.04, 1000, 100, 1e-6, 2),
                           depth=8, t=1e-4, rhs=coordinate_rhs, tol=1e-6, precision="mixed"),
    "double_sheet_1m_d9": dict(mesh=lambda: double_sheet(500, 0.05, 9, 0.5, 1e-6, 4), depth=9,
                               t=1e-3, rhs=lambda V: uniform_rhs(V.shape[0]), tol=1e-6,
                               precision="mixed"),
    "knot35_4m_d10": dict(mesh=lambda: torus_knot_tube(3, 5, 1.0, 0.02, 10000, 200, 1e-7, 6),
                          depth=10, t=1e-4, rhs=coordinate_rhs, tol=1e-6, precision="mixed"),
    # the same knot surface on the same depth-10 grid with a quarter of the triangles: its
    # finest level has the same functions and stencils, with a quarter of the voxel pieces
    # (a case small enough for whole-kernel profiling)
    "knot35_1m_d10": dict(mesh=lambda: torus_knot_tube(3, 5, 1.0, 0.02, 5000, 100, 1e-7, 6),
                          depth=10, t=1e-4, rhs=coordinate_rhs, tol=1e-6, precision="mixed"),
}


def config_mesh(name):
    """Return (V, F, depth, t, f_vertex, tol, precision) for a named workload."""
    c = CONFIGS[name]
    V, F = c["mesh"]()
    return V, F, c["depth"], c["t"], c["rhs"](V), c["tol"], c["precision"]
