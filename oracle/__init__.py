"""Plain FP64 CPU oracle for the exponential Rosenbrock shallow-water path.

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  The product path (the CUDA library under ``paper_1805_02144_gb300``) never
imports, links or calls anything here, and nothing here imports the product.

Modules
-------
mesh     icosahedral geodesic Voronoi grid and the sparse finite-volume
         operators G, D, V, L (Sec. 2, eq. (2.6)-(2.9))
swe      F(u) of eq. (2.6) with the dissipation of eq. (2.8), and the Jacobian
         J = J_v + J_r + J_m of eqs. (2.12)-(2.15)
phi      phi-functions (eqs. (3.6)-(3.7)), the augmented-matrix exponential of
         Algorithm 1 step 2(ii), and a dense reference for sum_l phi_l(A) v_l
phipm    phipm_simul_iom2 (Algorithm 1) with IOM2 and the substep controller
schemes  EPI2 (eq. 3.5), exprb42 (eq. 3.11), pexprb43 (eq. 3.12),
         exprb53 (eq. 3.13) and epi3 (eq. 3.19), driven as in Sec. 4.4
adjoint  gradient of EPI2 / exprb42 steps with the substep decisions frozen,
         by torch.autograd of a torch float64 re-evaluation of the same map,
         and the observation misfit of a forecast

Everything else is float64 numpy / scipy.sparse; library primitives used as
steps are sparse matrix-vector products, ``scipy.linalg.expm``,
``torch.linalg.matrix_exp`` and torch's reverse-mode differentiation.
"""
