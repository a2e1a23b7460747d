"""Pins of the oracle's intersects test on near-coplanar face pairs whose
answer only exact arithmetic decides (vertices 2^-32 off, or exactly on, a
plane with a normal about 2^38 long, at coordinates about 2^20).

The generator's construction fixes the answer for most kinds (touching,
strictly one side, crossing inside); where it does not, the independent
Minkowski-difference test in exact rationals decides.  Both are checked
against the oracle, which the GPU exact stage is then compared with.
Definitions: Sec. 3.2.3 (Eq. 4 in sign form, closed faces)."""
from fractions import Fraction

import numpy as np
import pytest

from exact_ref import frac_orient3d, minkowski_intersects
from paper_1808_09571_gb300 import synth

CASES = synth.near_coplanar_face_pairs(40)


def test_construction_is_exact():
    """Every vertex is the intended dyadic rational: a vertex built on the
    plane has an exactly zero orientation, one moved by 2^-32 a nonzero one
    of the intended sign, and the two far vertices are strictly positive."""
    for T1, T2, exp, kind in CASES:
        P, Q, R = T1
        s0 = frac_orient3d(P, Q, R, T2[0])
        if kind == "coplanar":
            assert all(frac_orient3d(P, Q, R, v) == 0 for v in T2)
            continue
        s1, s2 = frac_orient3d(P, Q, R, T2[1]), frac_orient3d(P, Q, R, T2[2])
        assert s1 == s2 != 0
        if kind == "interior" and exp is False:
            assert s0 == s1
        elif kind == "interior" and exp is True:
            assert s0 in (0, -s1)
        # the orientation of a vertex off the plane is tiny: |N . (X - P)|
        # below 2^7 while |N| is about 2^38
        N = np.cross(Q - P, R - P)
        h = sum(Fraction(float(N[k])) * (Fraction(float(T2[0][k])) - Fraction(float(P[k]))) for k in range(3))
        assert abs(h) < 2 ** 7


@pytest.mark.parametrize("k", range(len(CASES)))
def test_oracle_on_near_coplanar_pairs(orc, k):
    T1, T2, exp, kind = CASES[k]
    got = orc.tri_intersects(T1, T2)
    assert got == orc.tri_intersects(T2, T1)
    if exp is not None:
        assert got == exp, kind
    assert got == minkowski_intersects(T1, T2), kind
    assert (orc.tri_distance(T1, T2) == 0.0) == got


def test_kinds_cover_both_answers(orc):
    ans = {}
    for T1, T2, exp, kind in CASES:
        ans.setdefault(kind, set()).add(orc.tri_intersects(T1, T2))
    assert ans["interior"] == {True, False}
    assert ans["coplanar"] == {True, False}
