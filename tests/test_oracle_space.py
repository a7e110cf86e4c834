"""Pins of the oracle's Q_k spatial matrices (Sec. 3.1 and "Spatial matrices"
in Sec. 3.5): textbook 1D element matrices, exact rational integrals with a
linear coefficient, Kronecker identities of the tensor-product mesh, and the
invariants 1^T M 1 = |D|, K 1 = 0."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import coeff, space_fe


def one_piece(dim, amp=1.0, factors=None):
    return [dict(mu=(0,), amp=amp, factors=factors or [("one", 0)] * dim)]


def mats(dim, cells, lo, hi, k, pieces):
    mesh = space_fe.Mesh(dim, cells, lo, hi, k)
    Mx, Ks = space_fe.assemble(mesh, coeff.at_cell_points(pieces))
    return mesh, Mx, Ks


@pytest.mark.parametrize("h", [1.0, 0.25, 0.1])
def test_textbook_1d_element_matrices(h):
    _, M1, K1 = mats(1, (1,), (0.0,), (h,), 1, one_piece(1))
    assert np.allclose(K1[0].toarray(), np.array([[1, -1], [-1, 1]]) / h, atol=1e-13)
    assert np.allclose(M1.toarray(), h / 6 * np.array([[2, 1], [1, 2]]), atol=1e-15)
    _, M2, K2 = mats(1, (1,), (0.0,), (h,), 2, one_piece(1))
    assert np.allclose(K2[0].toarray(), np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / (3 * h), atol=1e-12)
    assert np.allclose(M2.toarray(), h / 30 * np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]), atol=1e-15)


def test_linear_coefficient_exact_rational_integrals():
    sympy = pytest.importorskip("sympy")
    x = sympy.symbols("x")
    h = sympy.Rational(1, 2)
    nodes = [0, h / 2, h]
    basis = []
    for i in range(3):
        b = 1
        for j in range(3):
            if j != i:
                b *= (x - nodes[j]) / (nodes[i] - nodes[j])
        basis.append(sympy.expand(b))
    want = np.array([[float(sympy.integrate(x * sympy.diff(basis[i], x) * sympy.diff(basis[j], x), (x, 0, h)))
                      for j in range(3)] for i in range(3)])
    _, _, K = mats(1, (1,), (0.0,), (0.5,), 2, one_piece(1, factors=[("pow", 1)]))
    assert np.allclose(K[0].toarray(), want, atol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_tensor_product_identities_2d(k):
    cx, cy, Lx, Ly = 3, 2, 1.0, 0.7
    _, Mx1, Kx1 = mats(1, (cx,), (0.0,), (Lx,), k, one_piece(1))
    _, My1, Ky1 = mats(1, (cy,), (0.0,), (Ly,), k, one_piece(1))
    mesh, M, K = mats(2, (cx, cy), (0.0, 0.0), (Lx, Ly), k, one_piece(2))
    # x fastest: kron(y-factor, x-factor)
    assert abs(M - sp.kron(My1, Mx1)).max() < 1e-14
    assert abs(K[0] - (sp.kron(My1, Kx1[0]) + sp.kron(Ky1[0], Mx1))).max() < 1e-11
    one = np.ones(mesh.n_nodes)
    assert abs(one @ (M @ one) - Lx * Ly) < 1e-13
    assert np.abs(K[0] @ one).max() < 1e-11


def test_tensor_product_identities_3d():
    k = 2
    c, L = (2, 2, 3), (1.0, 0.5, 0.9)
    m1 = [mats(1, (c[d],), (0.0,), (L[d],), k, one_piece(1)) for d in range(3)]
    M1 = [m[1] for m in m1]
    K1 = [m[2][0] for m in m1]
    mesh, M, K = mats(3, c, (0, 0, 0), L, k, one_piece(3))
    want_K = (sp.kron(M1[2], sp.kron(M1[1], K1[0])) + sp.kron(M1[2], sp.kron(K1[1], M1[0]))
              + sp.kron(K1[2], sp.kron(M1[1], M1[0])))
    assert abs(M - sp.kron(M1[2], sp.kron(M1[1], M1[0]))).max() < 1e-14
    assert abs(K[0] - want_K).max() < 1e-11
    one = np.ones(mesh.n_nodes)
    assert abs(one @ (M @ one) - np.prod(L)) < 1e-13


def test_separable_coefficient_is_kronecker_of_weighted_1d():
    # a(x, y) = sin(pi x) * y^1: Gauss tensor quadrature of a separable integrand
    # factorises into the 1D rules, so K = kron(M1[y], K1[sin]) + kron(K1[y], M1[sin])
    k = 2
    fx, fy = ("sin", 1), ("pow", 1)
    mx = space_fe.Mesh(1, (4,), (0.0,), (1.0,), k)
    my = space_fe.Mesh(1, (3,), (0.0,), (1.0,), k)
    def weighted(mesh1, f):
        pieces = [dict(mu=(0,), amp=1.0, factors=[f])]
        # mass with weight f: assemble K with coefficient and separately the
        # f-weighted mass by brute force over the 1D Gauss points
        fe = space_fe.FE1D(k)
        wJ, phi, grad = space_fe.reference_shape(mesh1, fe)
        cells = np.arange(mesh1.n_cells)
        xq = space_fe.cell_points(mesh1, fe, cells)
        a = coeff.evaluate(pieces, xq)[0]
        conn = mesh1.cell_dofs(cells)
        n = mesh1.n_nodes
        Mw, Kw = np.zeros((n, n)), np.zeros((n, n))
        for c in cells:
            for i in range(k + 1):
                for j in range(k + 1):
                    Mw[conn[c, i], conn[c, j]] += np.sum(wJ * a[c] * phi[i] * phi[j])
                    Kw[conn[c, i], conn[c, j]] += np.sum(wJ * a[c] * grad[i, :, 0] * grad[j, :, 0])
        return Mw, Kw
    Mwx, Kwx = weighted(mx, fx)
    Mwy, Kwy = weighted(my, fy)
    mesh = space_fe.Mesh(2, (4, 3), (0, 0), (1, 1), k)
    _, K = space_fe.assemble(mesh, coeff.at_cell_points([dict(mu=(0,), amp=1.0, factors=[fx, fy])]))
    assert np.abs(K[0].toarray() - (np.kron(Mwy, Kwx) + np.kron(Kwy, Mwx))).max() < 1e-12


def test_node_rows_match_assembly():
    pieces = [dict(mu=(0, 0), amp=1.0, factors=[("one", 0)] * 3),
              dict(mu=(1, 0), amp=0.1, factors=[("sin", 1), ("sin", 2), ("one", 0)])]
    mesh = space_fe.Mesh(3, (3, 2, 2), (0, 0, 0), (1, 1, 1), 2)
    f = coeff.at_cell_points(pieces)
    M, K = space_fe.assemble(mesh, f)
    for node in [0, 7, 31, 62, mesh.n_nodes - 1]:
        cols, mr, kr = space_fe.node_rows(mesh, f, node)
        assert np.allclose(M[node].toarray()[0, cols], mr, atol=1e-15)
        assert np.allclose(np.delete(M[node].toarray()[0], cols), 0.0)
        for t in range(2):
            assert np.allclose(K[t][node].toarray()[0, cols], kr[t], atol=1e-13)
