"""Pins of the exact volume oracle (Eq. 2) against closed forms and
invariants that do not go through the oracle's own arithmetic (CPU)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import volume as VO
from paper_1808_09571_gb300 import synth


def box(a, b, c, origin=(0.0, 0.0, 0.0)):
    return synth.box_mesh(a, b, c, origin)


def test_box_closed_form():
    assert VO.volume_exact(*box(2.0, 3.0, 5.0)) == 30
    assert VO.volume_exact(*box(0.5, 0.25, 0.125)) == Fraction(1, 64)
    # dyadic sides far from the origin: still exact
    assert VO.volume_exact(*box(3.0, 7.0, 1.5, origin=(1024.0, -2048.0, 4096.0))) == Fraction(63, 2)


def test_tetrahedron_closed_form():
    """Unit-corner tetrahedron: 1/6; a scaled one: a b c / 6."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float64)
    I = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.uint32)
    assert VO.volume_exact(V, I) == Fraction(1, 6)
    V2 = V * np.array([2.0, 3.0, 0.5])
    assert VO.volume_exact(V2, I) == Fraction(1, 2)


def test_orientation_and_translation():
    """Reversing every face negates the volume; translating a closed mesh
    leaves it unchanged (the field's flux through a closed surface)."""
    m = synth.small_ore_body()
    V = m.V.astype(np.float64)
    v0 = VO.volume_exact(V, m.I)
    assert VO.volume_exact(V, m.I[:, ::-1]) == -v0
    assert VO.volume_exact(V + np.array([0.5, -0.25, 8.0]), m.I) == v0


def test_ellipsoid_converges_to_closed_form():
    """A fine UV ellipsoid approaches 4/3 pi a b c from below (inscribed)."""
    V, I = synth.uv_ellipsoid((4.0, 2.5, 1.5), 128, 128, jitter=0.0, seed=0)
    v = VO.volume(V, I)
    ref = 4.0 / 3.0 * np.pi * 4.0 * 2.5 * 1.5
    assert 0 < ref - v < 2e-3 * ref, (v, ref)


def test_double_rounding():
    """volume() is the exact value rounded once."""
    V = np.array([[0.1, 0.2, 0.3], [1.1, 0.2, 0.3], [0.1, 1.3, 0.3], [0.1, 0.2, 1.7]], np.float64)
    I = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.uint32)
    ex = VO.volume_exact(V, I)
    assert VO.volume(V, I) == float(ex)
    closed = Fraction(V[1, 0]) - Fraction(V[0, 0]), Fraction(V[2, 1]) - Fraction(V[0, 1]), \
        Fraction(V[3, 2]) - Fraction(V[0, 2])
    assert ex == closed[0] * closed[1] * closed[2] / 6


def test_open_surface_uses_the_origin():
    """For one face the formula is det(u, v, w) / 6 with the origin as the
    apex (an open surface is not translation invariant)."""
    V = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    I = np.array([[0, 1, 2]], np.uint32)
    assert VO.volume_exact(V, I) == Fraction(1, 6)
    assert VO.volume_exact(V + 1.0, I) == Fraction(4, 6)  # det[[2,1,1],[1,2,1],[1,1,2]] = 4
