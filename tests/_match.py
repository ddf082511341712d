"""Matching the library's dof numbering with the oracle's (same functions, other order).

A function is identified by its grid corner and the smallest triangle index of its
component, which both numberings report."""
import numpy as np


def dof_keys(corner, mintri, nt):
    c = corner.astype(np.int64)
    return ((c[:, 0] * 8192 + c[:, 1]) * 8192 + c[:, 2]) * (nt + 1) + mintri.astype(np.int64)


def permutation(lib_corner, lib_mintri, orc_corner, orc_mintri, nt):
    """perm[i] = oracle index of library dof i (-1 if absent)."""
    kl = dof_keys(lib_corner, lib_mintri, nt)
    ko = dof_keys(orc_corner, orc_mintri, nt)
    order = np.argsort(ko)
    pos = np.searchsorted(ko[order], kl)
    pos = np.minimum(pos, len(ko) - 1)
    perm = order[pos]
    perm[ko[perm] != kl] = -1
    return perm


def csr_to_scipy(rp, ci, val, n):
    import scipy.sparse as sp
    return sp.csr_matrix((val, ci, rp), shape=(n, n))
