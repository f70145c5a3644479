"""Pin of the oracle's far sets (Sec. 3.1: I_n of eq. Fmin, E_n of eq. Emin, C_n of eq. Cmin,
and the 3D list I_n, F_n, E_n, C_n).  Every stencil test builds its far set through
``class_far_set``, so an off-by-one in the printed strict inequalities (-n < j < -b) would
pass them all.  Here the sets are enumerated by hand from those inequalities for tiny grids
and written out literally.

Class convention of the oracle: +1 = the point lies on the high face of that axis (its far
points lie at negative offsets, as for the paper's right edge / top-right corner), -1 = the
low face (the mirror image), 0 = no face on that axis.
"""

import numpy as np

import oracle as O


def as_set(a):
    return {tuple(int(v) for v in row) for row in np.asarray(a)}


def test_2d_right_edge_n5():
    # E_5 with b = 1: -5 < j1 < -1, -5 < j2 < 5
    want_b1 = {(j1, j2) for j1 in (-4, -3, -2) for j2 in (-4, -3, -2, -1, 0, 1, 2, 3, 4)}
    assert as_set(O.class_far_set(5, 1, (1, 0))) == want_b1
    # b = 2: -5 < j1 < -2
    want_b2 = {(-4, -4), (-4, -3), (-4, -2), (-4, -1), (-4, 0), (-4, 1), (-4, 2), (-4, 3), (-4, 4),
               (-3, -4), (-3, -3), (-3, -2), (-3, -1), (-3, 0), (-3, 1), (-3, 2), (-3, 3), (-3, 4)}
    got = O.class_far_set(5, 2, (1, 0))
    assert len(got) == 18 and as_set(got) == want_b2


def test_2d_edges_on_the_other_faces_are_mirror_images_n5_b2():
    # left edge: 2 < j1 < 5; top edge (axis 1 high): -5 < j2 < -2; bottom: 2 < j2 < 5
    assert as_set(O.class_far_set(5, 2, (-1, 0))) == {(j1, j2) for j1 in (3, 4) for j2 in range(-4, 5)}
    assert as_set(O.class_far_set(5, 2, (0, 1))) == {(j1, j2) for j1 in range(-4, 5) for j2 in (-4, -3)}
    assert as_set(O.class_far_set(5, 2, (0, -1))) == {(j1, j2) for j1 in range(-4, 5) for j2 in (3, 4)}


def test_2d_corner_n5():
    # C_5 with b = 1: -5 < j1, j2 < -1
    assert as_set(O.class_far_set(5, 1, (1, 1))) == {
        (-4, -4), (-4, -3), (-4, -2), (-3, -4), (-3, -3), (-3, -2), (-2, -4), (-2, -3), (-2, -2)}
    # b = 2: -5 < j1, j2 < -2
    assert as_set(O.class_far_set(5, 2, (1, 1))) == {(-4, -4), (-4, -3), (-3, -4), (-3, -3)}
    # the other corners by mirror images, b = 2
    assert as_set(O.class_far_set(5, 2, (-1, 1))) == {(4, -4), (4, -3), (3, -4), (3, -3)}
    assert as_set(O.class_far_set(5, 2, (-1, -1))) == {(4, 4), (4, 3), (3, 4), (3, 3)}


def test_2d_interior_n3():
    # I_3: -3 < j1, j2 < 3 without mu(0) = {-1, 0, 1}^2: the 16 points of the outer ring
    want = {(-2, -2), (-2, -1), (-2, 0), (-2, 1), (-2, 2), (2, -2), (2, -1), (2, 0), (2, 1), (2, 2),
            (-1, -2), (0, -2), (1, -2), (-1, 2), (0, 2), (1, 2)}
    got = O.class_far_set(3, 1, (0, 0))
    assert len(got) == 16 and as_set(got) == want
    # the interior set does not depend on b (the buffer only enters boundary sets)
    assert as_set(O.class_far_set(3, 2, (0, 0))) == want


def test_3d_sets_n4():
    # face on the high side of axis 0, b = 2 (F_4: -4 < j1 < -2, -4 < j2, j3 < 4): j1 = -3 only
    face = O.class_far_set(4, 2, (1, 0, 0))
    assert len(face) == 49 and as_set(face) == {(-3, a, c) for a in range(-3, 4) for c in range(-3, 4)}
    # edge (E_4, b = 1: -4 < j1, j2 < -1, -4 < j3 < 4)
    assert as_set(O.class_far_set(4, 1, (1, 1, 0))) == {
        (-3, -3, -3), (-3, -3, -2), (-3, -3, -1), (-3, -3, 0), (-3, -3, 1), (-3, -3, 2), (-3, -3, 3),
        (-3, -2, -3), (-3, -2, -2), (-3, -2, -1), (-3, -2, 0), (-3, -2, 1), (-3, -2, 2), (-3, -2, 3),
        (-2, -3, -3), (-2, -3, -2), (-2, -3, -1), (-2, -3, 0), (-2, -3, 1), (-2, -3, 2), (-2, -3, 3),
        (-2, -2, -3), (-2, -2, -2), (-2, -2, -1), (-2, -2, 0), (-2, -2, 1), (-2, -2, 2), (-2, -2, 3)}
    # corner (C_4, b = 1: -4 < j1, j2, j3 < -1); the corner is read on x_1 = 1 like the others
    assert as_set(O.class_far_set(4, 1, (1, 1, 1))) == {
        (-3, -3, -3), (-3, -3, -2), (-3, -2, -3), (-3, -2, -2),
        (-2, -3, -3), (-2, -3, -2), (-2, -2, -3), (-2, -2, -2)}
    # b = 2: a single far point per axis
    assert as_set(O.class_far_set(4, 2, (1, 1, 1))) == {(-3, -3, -3)}
    assert as_set(O.class_far_set(4, 2, (-1, 1, -1))) == {(3, -3, 3)}


def test_3d_interior_n3():
    # I_3: -3 < j_k < 3 without {-1, 0, 1}^3: 125 - 27 = 98 points
    got = as_set(O.class_far_set(3, 1, (0, 0, 0)))
    assert len(got) == 98
    assert {(2, 0, 0), (-2, -2, -2), (0, 1, -2), (2, 2, 2)} <= got
    assert not ({(1, 1, 1), (0, 0, 0), (-1, 0, 1), (3, 0, 0)} & got)
