"""Pins of the oracle's dG(r) time matrices (Sec. 3.2, eqs. At, Bt, Ct) against
hand-derived closed forms, textbook Radau IIA data and identities that hold
for any r (integration by parts, reproduction of constants)."""
from math import sqrt

import numpy as np

from oracle import time_dg


def test_dg1_closed_forms():
    # right Radau nodes {1/3, 1}: v_0 = 3(1-t)/2, v_1 = (3t-1)/2 (hand derivation)
    assert np.allclose(time_dg.radau_right_nodes(1), [1 / 3, 1.0], atol=1e-15)
    for tau in (1.0, 0.1, 1 / 64):
        A, B, C = time_dg.time_matrices(1, tau)
        assert np.allclose(A, [[9 / 8, 3 / 8], [-9 / 8, 5 / 8]], atol=1e-15)
        assert np.allclose(B, tau * np.diag([3 / 4, 1 / 4]), atol=1e-15 * tau + 1e-17)
        assert np.allclose(C, [[0.0, 3 / 2], [0.0, -1 / 2]], atol=1e-15)


def test_dg0_is_backward_euler():
    A, B, C = time_dg.time_matrices(0, 0.25)
    assert np.allclose(A, [[1.0]]) and np.allclose(B, [[0.25]]) and np.allclose(C, [[1.0]])


def test_radau_iia_nodes_and_weights():
    # textbook Radau IIA (s = 3): c = (4 -+ sqrt 6)/10, 1; b = (16 -+ sqrt 6)/36, 1/9
    n = time_dg.radau_right_nodes(2)
    assert np.allclose(n, [(4 - sqrt(6)) / 10, (4 + sqrt(6)) / 10, 1.0], atol=1e-14)
    _, B, _ = time_dg.time_matrices(2, 1.0)
    assert np.allclose(np.diag(B), [(16 - sqrt(6)) / 36, (16 + sqrt(6)) / 36, 1 / 9], atol=1e-14)


def test_identities_any_degree():
    for r in range(0, 6):
        A, B, C = time_dg.time_matrices(r, 1.0)
        nodes = time_dg.radau_right_nodes(r)
        l0 = time_dg.lagrange_values(nodes, [0.0])[:, 0]
        er = np.zeros(r + 1)
        er[r] = 1.0
        # integration by parts: A + A^T = e_r e_r^T + l(0) l(0)^T
        assert np.allclose(A + A.T, np.outer(er, er) + np.outer(l0, l0), atol=1e-12)
        # the dG step reproduces constants: A 1 = l(0), and C 1 = l(0)
        assert np.allclose(A.sum(axis=1), l0, atol=1e-12)
        assert np.allclose(C.sum(axis=1), l0, atol=1e-12)
        # (r+1)-point right Radau is exact to degree 2r: B is diagonal,
        # with the Radau weights (end weight 1/(r+1)^2, sum 1) on it
        assert np.abs(B - np.diag(np.diag(B))).max() < 1e-14
        assert abs(B[r, r] - 1.0 / (r + 1) ** 2) < 1e-14
        assert abs(np.trace(B) - 1.0) < 1e-14
    nodes3 = time_dg.radau_right_nodes(3)
    assert np.allclose(nodes3, [0.088587959512704, 0.409466864440735, 0.787659461760847, 1.0], atol=1e-12)
