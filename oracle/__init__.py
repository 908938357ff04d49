"""Oracle: a plain, slow FP64 CPU restatement of the staggered DG operators
and solves of Tavelli & Boscheri (Sec. 2.1-2.4, eqs. D, ad5.2, Mi, Mj, u,
ad5, pressure_final), of the semi-Lagrangian walk and transport (Sec. 2.5,
sl.py), of the IMEX tableaux, stage trajectories and SL-IMEX steps of
App. A and Sec. 3 (imex.py), and of the first-order Navier-Stokes step
(ns.py).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library,
its Python binding, the bench's timed legs) may import or call this package;
only the tests, the smoke check and the bench's CPU-baseline leg do.  It
shares no code with the CUDA path: the only common module is the seeded
input generator ``paper_2401_17806_gb300.synth``.

Readings of the paper that the oracle fixes (each one is listed in the design
notes): equispaced nodal basis, dual basis permutations by node coincidence,
deterministic left/right assignment, RCM + greedy colouring order, the SPSD
sign of the Schur operator, coefficient-space mean-zero pressure, CG with
x0 = 0 and relative-residual stopping.

Parity status: every function is pinned by the ``-m "not gpu"`` tests
(closed forms, exact rational integrals, adjointness, the reference-operator
decomposition, polynomial reproduction, nullspace, brute-force solves,
manufactured convergence).
"""
