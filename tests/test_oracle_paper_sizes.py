"""The paper's benchmark discretisation (Sec. 4.3-4.4 and its solver-performance
table) as the oracle discretises it: the unknowns per slab equal the N_SG the
paper prints for p = 0..6 (tests/golden/paper_table2_sizes.txt), which pins the
node count of Q3 on 128^2 cells, the four dG(3) time nodes and the chaos
dimension together."""
import os

import numpy as np

from oracle import operator
from paper_2605_21046_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_paper_discretisation_sizes_match_the_paper():
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_table2_sizes.txt"), dtype=np.int64)
    for p_xi, n_sg in rows:
        spec = I.config_paper_q3(P=int(p_xi))
        op = operator.SGProblem(spec, assemble_space=False)
        assert op.n_xi * op.n_t * op.n_x == n_sg, (p_xi, op.shape)
        assert op.n_t == 4 and op.n_x == (3 * 128 + 1) ** 2
