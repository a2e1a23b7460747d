"""Exact oracle of the mesh volume of Eq. 2 (test infrastructure only).

Sec. 3.2.1 applies the divergence theorem with the field F = p / 3 to a
polyhedron whose faces A_i = (u_i, v_i, w_i) are counter-clockwise seen
from outside: V = (1/6) sum_i u_i . n_i with n_i = (v_i - u_i) x (w_i - u_i)
(Eq. 2).  This module evaluates that sum exactly: every float coordinate is a
dyadic rational m 2^e, so after scaling all coordinates of the mesh by a
common power of two they are integers, and the sum of the per-face triple
products is an exact integer (Python ints), divided by 6 and by the scale
cubed as a Fraction at the end.  No rounding anywhere.

The value is the signed volume for a closed, consistently oriented mesh
(negative when the faces are clockwise); for an open mesh it is the
formula's value, which depends on the origin.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def _to_ints(V: np.ndarray):
    """Integer coordinates X and exponent k with V = X * 2^k exactly."""
    V = np.asarray(V, dtype=np.float64)
    m, e = np.frexp(V)  # V = m 2^e, 0.5 <= |m| < 1 (m = 0 for 0)
    nz = V != 0
    if not nz.any():
        return np.zeros(V.shape, dtype=object), 0
    k = int(e[nz].min()) - 53
    # each m is an exact 53-bit fraction: m * 2^53 is an integer
    X = np.empty(V.shape, dtype=object)
    flat_m, flat_e, flat_x = m.ravel(), e.ravel(), X.ravel()
    for j in range(flat_m.size):
        if flat_m[j] == 0.0:
            flat_x[j] = 0
        else:
            mi = int(flat_m[j] * (1 << 53))  # exact
            flat_x[j] = mi << (int(flat_e[j]) - 53 - k)
    return X, k


def volume_exact(V, I) -> Fraction:
    """(1/6) sum over faces of u . ((v - u) x (w - u)), exactly (Eq. 2)."""
    I = np.asarray(I, dtype=np.int64).reshape(-1, 3)
    X, k = _to_ints(V)
    total = 0
    for a, b, c in I:
        u, v, w = X[a], X[b], X[c]
        e0 = (v[0] - u[0], v[1] - u[1], v[2] - u[2])
        e1 = (w[0] - u[0], w[1] - u[1], w[2] - u[2])
        n = (e0[1] * e1[2] - e0[2] * e1[1], e0[2] * e1[0] - e0[0] * e1[2], e0[0] * e1[1] - e0[1] * e1[0])
        total += u[0] * n[0] + u[1] * n[1] + u[2] * n[2]
    return Fraction(total, 6) * (Fraction(2) ** (3 * k))


def volume(V, I) -> float:
    """The exact value of Eq. 2 rounded once to the nearest double."""
    return float(volume_exact(V, I))


def rounding_scale(V, I) -> float:
    """sum_i |u_i| |v_i - u_i| |w_i - u_i| / 6 (2-norms, in double): the
    magnitude an FP64 evaluation of Eq. 2 rounds relative to -- each term's
    triple product is bounded by it, and so is the error of computing it."""
    V = np.asarray(V, dtype=np.float64)
    I = np.asarray(I, dtype=np.int64).reshape(-1, 3)
    u, v, w = V[I[:, 0]], V[I[:, 1]], V[I[:, 2]]
    s = np.linalg.norm(u, axis=1) * np.linalg.norm(v - u, axis=1) * np.linalg.norm(w - u, axis=1)
    return float(math.fsum(s)) / 6.0
