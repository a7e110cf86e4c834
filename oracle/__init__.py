"""Oracle: a plain, slow, obviously correct FP64 CPU implementation of the
stochastic-Galerkin (SG) space-time slab operator and its building blocks.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_2605_21046_gb300``) never imports, links or executes
anything here, and nothing here imports the product package: the two share no
code.  Every function cites the passage of the paper it follows.

Modules
-------
hermite    Hermite chaos: psi_n (eq. Hermit_def), total-degree index set
           Lambda_p (Sec. 3.3), triple products G_mu (eq. triple_stoch and the
           factorisation remark that follows it).
time_dg    dG(r) time discretisation with the right Gauss-Radau nodal basis
           (Sec. 3.2) and the temporal matrices A_t, B_t, C_t (eqs. At, Bt, Ct).
space_fe   Conforming Q_k elements on uniform Cartesian meshes (Sec. 3.1),
           assembled mass M_x and coefficient-mode stiffness K_mu (Sec. 3.5,
           "Spatial matrices").
coeff      Evaluation of the coefficient expansion a = sum_mu a_mu(x) Psi_mu
           (eq. coeff_expansion) from a plain data description.
operator   The slab operator A^(n) = M_xi (x) A_t (x) M_x
           + sum_mu G_mu (x) B_t (x) K_mu (eq. local_rhs_tensor) applied as a
           Kronecker sum of assembled factors, and assembled outright for
           small cases.
"""
