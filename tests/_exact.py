"""Exact integrals used to pin the oracle (independent of its quadrature).

Polynomials on a triangle are expanded in barycentric coordinates and
integrated with the closed form  int_T l0^a l1^b l2^c dA = 2|T| a! b! c! / (a+b+c+2)!.
"""
from __future__ import annotations

from math import factorial

import numpy as np


def _mul(p, q):
    out = {}
    for ka, va in p.items():
        for kb, vb in q.items():
            k = (ka[0] + kb[0], ka[1] + kb[1], ka[2] + kb[2])
            out[k] = out.get(k, 0.0) + va * vb
    return out


def _add(p, q, s=1.0):
    out = dict(p)
    for k, v in q.items():
        out[k] = out.get(k, 0.0) + s * v
    return out


def _scale(p, s):
    return {k: v * s for k, v in p.items()}


def linear_form(values):
    """Homogeneous linear polynomial sum_i values[i] * l_i."""
    return {(1, 0, 0): float(values[0]), (0, 1, 0): float(values[1]), (0, 0, 1): float(values[2])}


def integrate(p, area):
    s = 0.0
    for (a, b, c), v in p.items():
        s += v * 2.0 * area * factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 2)
    return s


def triangle_area_normal(P):
    cr = np.cross(P[1] - P[0], P[2] - P[0])
    a = 0.5 * np.linalg.norm(cr)
    return a, cr / (2 * a)


def monomial_integral(P, powers):
    """int_T x^i y^j z^k dA over triangle P (3x3 array) exactly."""
    area, _ = triangle_area_normal(P)
    poly = {(0, 0, 0): 1.0}
    # homogeneous degree bookkeeping: constant 1 = l0+l1+l2
    one = linear_form([1, 1, 1])
    deg = 0
    for ax, pw in enumerate(powers):
        for _ in range(pw):
            poly = _mul(poly, linear_form(P[:, ax]))
            deg += 1
    if deg == 0:
        poly = {(0, 0, 0): 1.0}
    return integrate(poly, area)


def hat_matrices_single_voxel(P, lo, s):
    """Exact 8x8 mass and tangential-stiffness matrices of the trilinear hats of
    the voxel [lo, lo+s]^3 over a triangle P lying inside it.

    Corner a has bits (a&1, a>>1&1, a>>2&1) = upper side per axis.
    """
    area, n = triangle_area_normal(P)
    u = (P - lo[None, :]) / s          # local coordinates of the vertices
    phi = {}
    for ax in range(3):
        phi[(ax, 0)] = linear_form(1.0 - u[:, ax])
        phi[(ax, 1)] = linear_form(u[:, ax])
    b, g = [], []
    for a in range(8):
        bits = (a & 1, (a >> 1) & 1, (a >> 2) & 1)
        b.append(_mul(_mul(phi[(0, bits[0])], phi[(1, bits[1])]), phi[(2, bits[2])]))
        grad = []
        for ax in range(3):
            sign = (1.0 if bits[ax] else -1.0) / s
            others = [phi[(o, bits[o])] for o in range(3) if o != ax]
            grad.append(_scale(_mul(others[0], others[1]), sign))
        # tangential projection (I - n n^T) grad
        tg = []
        for ax in range(3):
            comp = dict(grad[ax])
            for bx in range(3):
                comp = _add(comp, grad[bx], -n[ax] * n[bx])
            tg.append(comp)
        g.append(tg)
    M = np.zeros((8, 8))
    L = np.zeros((8, 8))
    for a in range(8):
        for c in range(8):
            M[a, c] = integrate(_mul(b[a], b[c]), area)
            acc = {}
            for ax in range(3):
                acc = _add(acc, _mul(g[a][ax], g[c][ax]))
            L[a, c] = integrate(acc, area)
    return M, L
