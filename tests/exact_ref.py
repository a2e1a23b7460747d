"""Independent checks used to pin the oracle (tests only).

- `minkowski_intersects`: closed triangles T1, T2 share a point iff the origin
  lies in the convex hull of the nine differences a_i - b_j (the Minkowski
  difference T1 - T2).  By Caratheodory's theorem it then lies in the hull of
  at most four affinely independent differences, so every such subset is
  tried with exact rational Gaussian elimination.  This formulation has no
  orientation predicate, plane cut or 2D projection in common with the
  oracle's edge-by-edge test.
- `qp_distance`: the squared distance between two parametric triangles
  T1(u,v) = A0 + u(A1-A0) + v(A2-A0), T2(s,t) likewise (Eq. 3 extended to two
  triangles) is a convex quadratic over a polytope; it is minimised by SLSQP,
  whose local minimum is then global.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import combinations

import numpy as np


def _solve_exact(M, rhs):
    """Exact solution of M x = rhs (rows >= cols); None if the columns are
    dependent or the system is inconsistent."""
    rows, cols = len(M), len(M[0])
    A = [list(M[r]) + [rhs[r]] for r in range(rows)]
    piv_rows = []
    r = 0
    for c in range(cols):
        p = next((i for i in range(r, rows) if A[i][c] != 0), None)
        if p is None:
            return None  # dependent columns: a smaller subset covers it
        A[r], A[p] = A[p], A[r]
        inv = 1 / A[r][c]
        A[r] = [x * inv for x in A[r]]
        for i in range(rows):
            if i != r and A[i][c] != 0:
                f = A[i][c]
                A[i] = [x - f * y for x, y in zip(A[i], A[r])]
        piv_rows.append(r)
        r += 1
    for i in range(r, rows):
        if A[i][cols] != 0:
            return None
    return [A[i][cols] for i in range(cols)]


def minkowski_intersects(T1, T2) -> bool:
    T1 = np.asarray(T1, np.float64).reshape(3, 3)
    T2 = np.asarray(T2, np.float64).reshape(3, 3)
    P = [tuple(Fraction(float(T1[i, k])) - Fraction(float(T2[j, k])) for k in range(3))
         for i in range(3) for j in range(3)]
    if any(all(x == 0 for x in p) for p in P):
        return True
    for m in (2, 3, 4):
        for sub in combinations(range(9), m):
            M = [[P[j][k] for j in sub] for k in range(3)] + [[Fraction(1)] * m]
            rhs = [Fraction(0)] * 3 + [Fraction(1)]
            x = _solve_exact(M, rhs)
            if x is not None and all(v >= 0 for v in x):
                return True
    return False


def qp_distance(T1, T2) -> float:
    from scipy.optimize import minimize
    A = np.asarray(T1, np.float64).reshape(3, 3)
    B = np.asarray(T2, np.float64).reshape(3, 3)
    o = A[0].copy()
    A = A - o
    B = B - o
    ea0, ea1 = A[1] - A[0], A[2] - A[0]
    eb0, eb1 = B[1] - B[0], B[2] - B[0]
    M = np.stack([ea0, ea1, -eb0, -eb1], axis=1)
    c = A[0] - B[0]

    def f(x):
        r = M @ x + c
        return float(r @ r)

    def g(x):
        return 2 * M.T @ (M @ x + c)

    cons = [{"type": "ineq", "fun": lambda x: 1 - x[0] - x[1], "jac": lambda x: np.array([-1., -1, 0, 0])},
            {"type": "ineq", "fun": lambda x: 1 - x[2] - x[3], "jac": lambda x: np.array([0., 0, -1, -1])}]
    best = np.inf
    for x0 in ([1 / 3] * 4, [0, 0, 0, 0], [1, 0, 1, 0], [0, 1, 0, 1], [0.5, 0, 0, 0.5]):
        r = minimize(f, np.array(x0, float), jac=g, bounds=[(0, 1)] * 4, constraints=cons,
                     method="SLSQP", options={"ftol": 1e-16, "maxiter": 500})
        x = np.clip(r.x, 0, 1)
        for (i, j) in ((0, 1), (2, 3)):
            s = x[i] + x[j]
            if s > 1:
                x[i] /= s
                x[j] /= s
        best = min(best, f(x))
    return float(np.sqrt(max(best, 0.0)))


def frac_orient3d(a, b, c, d) -> int:
    F = [[Fraction(float(p[k])) - Fraction(float(d[k])) for k in range(3)] for p in (a, b, c)]
    det = (F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1])
           - F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0])
           + F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]))
    return (det > 0) - (det < 0)
