"""Plants plausible mistakes in the oracle (on the CPU, through monkeypatching)
and checks that the weak-form pin of the slab operator rejects each of them:
a transposed A_t, a dropped dG jump term, a sign error in the Hermite
linearisation, swapped mesh directions, and a mass term scaled by tau."""
import numpy as np
import pytest

from oracle import hermite, operator, time_dg

from test_oracle_operator import brute_bilinear, linear_pieces


def _pin_gap(spec):
    p = operator.SGProblem(spec)
    rng = np.random.default_rng(11)
    U = rng.uniform(-1, 1, p.shape)
    V = rng.uniform(-1, 1, p.shape)
    U[:, :, p.bmask] = 0.0
    V[:, :, p.bmask] = 0.0
    return abs(float(np.sum(V * p.apply(U))) - brute_bilinear(p, U, V))


SPEC = dict(dim=2, cells=(3, 2), lo=(0.0, 0.0), hi=(1.0, 0.6), k=2, r=1, n_slabs=4, T=1.2,
            M=2, P=2, coef=linear_pieces())


def test_unmutated_passes():
    assert _pin_gap(SPEC) < 1e-12


def _time_transposed(r, tau):
    A, B, C = ORIG_TIME(r, tau)
    return A.T, B, C


def _time_no_jump(r, tau):
    A, B, C = ORIG_TIME(r, tau)
    nodes = time_dg.radau_right_nodes(r)
    l0 = time_dg.lagrange_values(nodes, [0.0])[:, 0]
    return A - np.outer(l0, l0), B, C


def _time_mass_tau(r, tau):
    A, B, C = ORIG_TIME(r, tau)
    return A * tau, B, C


def _triple_sign(a, b, c):
    v = ORIG_TRIPLE(a, b, c)
    return -v if (a + b + c) % 4 == 2 and a > 0 else v


ORIG_TIME = time_dg.time_matrices
ORIG_TRIPLE = hermite.triple_1d


@pytest.mark.parametrize("target,name,fake", [
    (operator.time_dg, "time_matrices", _time_transposed),
    (operator.time_dg, "time_matrices", _time_no_jump),
    (operator.time_dg, "time_matrices", _time_mass_tau),
    (hermite, "triple_1d", _triple_sign),
])
def test_planted_mistake_is_caught(monkeypatch, target, name, fake):
    monkeypatch.setattr(target, name, fake)
    assert _pin_gap(SPEC) > 1e-6


def test_swapped_directions_caught(monkeypatch):
    orig = operator.space_fe.Mesh.__init__

    def swapped(self, dim, cells, lo, hi, k):
        orig(self, dim, cells, lo, hi, k)
        self.h = self.h[::-1].copy()
    monkeypatch.setattr(operator.space_fe.Mesh, "__init__", swapped)
    p = operator.SGProblem(SPEC)
    monkeypatch.setattr(operator.space_fe.Mesh, "__init__", orig)
    # the brute force uses the true geometry
    q = operator.SGProblem(SPEC)
    rng = np.random.default_rng(11)
    U = rng.uniform(-1, 1, q.shape)
    V = rng.uniform(-1, 1, q.shape)
    U[:, :, q.bmask] = 0.0
    V[:, :, q.bmask] = 0.0
    assert abs(float(np.sum(V * p.apply(U))) - brute_bilinear(q, U, V)) > 1e-6
