"""Pins of the oracle's manufactured-solution machinery: the load vector
(eq. load_vector, with the forcing modes f_beta = E[f Psi_beta] of eq.
manufactured_rhs_benchmark), the initial vector (eq. initial_vector), slab
marching (eq. local_tensor_system) and the error norms (Definition "error
norms and quantities").

* A solution that lies in the discrete space is reproduced exactly.
* The paper's benchmark at p = 0: the variance error equals Table 1's
  printed value, and the full error's truncation part equals the closed form
  of eq. finite-truncation-error-L2.
* The even coefficient leaves the mean unchanged under odd enrichment
  (p = 0 -> 1), as Table 1 prints.
* Q_k / dG(r) converge at order k+1 in L2 (Table 4 reports 4 for Q3/dG(3))."""
import os
from math import comb, sqrt

import numpy as np
import pytest

from oracle import hermite, manufactured, operator
from paper_2605_21046_gb300 import inputs as I
from paper_2605_21046_gb300.inputs import paper_coefficient

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_discrete_space_solution_is_reproduced():
    one, px = ("one", 0), ("pow", 1)
    coef = [dict(mu=(0, 0), amp=1.0, factors=[one, one]), dict(mu=(0, 0), amp=0.3, factors=[px, one]),
            dict(mu=(1, 0), amp=0.2, factors=[px, px]), dict(mu=(0, 1), amp=-0.1, factors=[one, px]),
            dict(mu=(1, 1), amp=0.05, factors=[one, one])]
    spec = dict(dim=2, cells=(4, 3), lo=(0.0, 0.0), hi=(1.0, 0.8), k=2, r=1, n_slabs=3, T=0.6, M=2, P=2, coef=coef)
    p = operator.SGProblem(spec)
    bx, by = ("poly", [0.0, 1.0, -1.0]), ("poly", [0.0, 1.25, -1.5625])     # s(1-s), s(1 - s/0.8)
    ex = {"q": 2, "c": [1.0, 0.5, -0.3, 0.2, 0.1, -0.4], "phi": [[bx, by]] * 6, "T": [0.5, 2.0]}
    man = manufactured.Manufactured(p, ex)
    err = man.errors(man.march(3))
    assert max(err.values()) < 1e-12, err


def _paper_row(p_xi):
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_table1.txt"))
    return rows[rows[:, 0] == p_xi][0]


def paper_problem(P, cells=(8, 8), slabs=8):
    spec = dict(dim=2, cells=cells, lo=(-1.0, -1.0), hi=(1.0, 1.0), k=3, r=3, n_slabs=slabs, T=1.0, M=4, P=P,
                coef=paper_coefficient())
    return operator.SGProblem(spec)


def test_paper_variance_error_and_truncation_at_p0():
    p = paper_problem(0)
    man = manufactured.Manufactured(p, manufactured.paper_exact())
    err = man.errors(man.march(8))
    row = _paper_row(0)
    assert abs(err["var"] - row[4]) <= 1e-5 * row[4]
    # E_full^2 = E_mean^2 + (truncated modes)^2 at p = 0 (modal identity, eq.
    # modal-sum-L2); truncation = ||t^4 Phi|| * sqrt(sum_{0<|a|<=6} eta^{2|a|})
    eta = 0.35
    trunc = (1 / 3) * sqrt(sum(comb(k + 3, 3) * eta ** (2 * k) for k in range(1, 7)))
    assert abs(sqrt(err["full"] ** 2 - err["mean"] ** 2) - trunc) <= 1e-5 * trunc
    # the paper's printed full error has the same truncation part
    assert sqrt(row[2] ** 2 - row[3] ** 2) == pytest.approx(trunc, rel=1e-4)


def test_mean_unchanged_under_odd_enrichment():
    e0 = manufactured.Manufactured(paper_problem(0, (4, 4), 4), manufactured.paper_exact())
    e1 = manufactured.Manufactured(paper_problem(1, (4, 4), 4), manufactured.paper_exact())
    m0 = e0.errors(e0.march(4))["mean"]
    m1 = e1.errors(e1.march(4))["mean"]
    assert abs(m0 - m1) <= 1e-10 * m0


def test_convergence_rate_k_plus_one():
    errs = []
    for n in (4, 8):
        spec = dict(dim=2, cells=(n, n), lo=(0.0, 0.0), hi=(1.0, 1.0), k=2, r=2, n_slabs=n, T=1.0, M=1, P=1,
                    coef=I.linear_sine_coef(1, 2, 0.1, [(1, 1)]))
        p = operator.SGProblem(spec)
        ex = {"q": 1, "c": [1.0, 0.3], "phi": [[("sin", 1), ("sin", 1)], [("sin", 2), ("sin", 1)]], "T": [0, 1, 0, 1]}
        man = manufactured.Manufactured(p, ex)
        errs.append(man.errors(man.march(n))["full"])
    rate = np.log2(errs[0] / errs[1])
    assert 2.6 < rate < 3.5, (errs, rate)      # k + 1 = 3 for Q2 / dG(2)
