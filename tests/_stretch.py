"""Oracle parity at full size through a stretch of the mesh (test helper).

The oracle is too slow to build the multi-million-triangle workloads, but a function's rows of M
and L and its right-hand side involve only the triangles that meet its support.  So the oracle is
built on a stretch of consecutive triangles, on the full mesh's grid (the same embedding, reading
A5), and compared only on functions whose support, and whose neighbours' supports, no triangle
outside the stretch can meet: there a function of the stretch (grid corner, component, smallest
triangle) is the full mesh's function, with the same entries and right-hand side.  A corner counts
as free of outside triangles when no outside triangle's bounding box meets its open support cube,
a conservative test."""
import numpy as np

from tests._match import dof_keys

OFFSETS = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], np.int64)


def stretch(V, F, t0, ntri):
    """Triangles [t0, t0 + ntri) of F with their vertices, renumbered (triangle order kept)."""
    Fp = F[t0:t0 + ntri]
    used = np.unique(Fp)
    remap = np.full(V.shape[0], -1, dtype=np.int64)
    remap[used] = np.arange(used.size)
    return np.ascontiguousarray(V[used]), np.ascontiguousarray(remap[Fp], dtype=np.int32)


def free_corners(V, F, t0, ntri, S, centre, depth, corners):
    """True for each corner (int [k, 3], depth `depth`) whose open support cube no triangle outside
    [t0, t0 + ntri) can meet (by bounding boxes, in finest-grid units)."""
    G = (np.asarray(V, np.float64) - (np.asarray(centre) - S / 2)) / (S / 2 ** depth)
    outside = np.ones(F.shape[0], bool)
    outside[t0:t0 + ntri] = False
    Fo = F[outside]
    lo = np.minimum(np.minimum(G[Fo[:, 0]], G[Fo[:, 1]]), G[Fo[:, 2]])
    hi = np.maximum(np.maximum(G[Fo[:, 0]], G[Fo[:, 1]]), G[Fo[:, 2]])
    cmin, cmax = corners.min(axis=0) - 1, corners.max(axis=0) + 1
    near = np.all((hi > cmin) & (lo < cmax), axis=1)
    lo, hi = lo[near], hi[near]
    free = np.ones(len(corners), bool)
    for k, cc in enumerate(corners):
        free[k] = not np.any(np.all((hi > cc - 1) & (lo < cc + 1), axis=1))
    return free


def complete_sample(V, F, t0, ntri, S, centre, depth, orc_corner, orc_mintri, count, seed=0):
    """Up to `count` oracle functions of the stretch (indices into its dofs) whose corner and 26
    neighbouring corners are free of outside triangles, and their keys with global triangles."""
    rng = np.random.default_rng(seed)
    cand = rng.permutation(len(orc_corner))[:max(8 * count, 64)]
    nb = (orc_corner[cand].astype(np.int64)[:, None, :] + OFFSETS[None]).reshape(-1, 3)
    uniq, inv = np.unique(nb, axis=0, return_inverse=True)
    free = free_corners(V, F, t0, ntri, S, centre, depth, uniq)
    ok = free[inv.reshape(len(cand), 27)].all(axis=1)
    pick = cand[ok][:count]
    return pick


def oracle_to_library(orc_corner, orc_mintri_global, lib_corner, lib_mintri, nt):
    """For every oracle function, the library function with the same corner and smallest triangle
    (-1 when absent)."""
    ko = dof_keys(orc_corner, orc_mintri_global, nt)
    kl = dof_keys(lib_corner, lib_mintri, nt)
    order = np.argsort(kl)
    pos = np.minimum(np.searchsorted(kl[order], ko), len(kl) - 1)
    idx = order[pos]
    idx[kl[idx] != ko] = -1
    return idx
