"""Plain, slow FP64 CPU oracle of the aTTN ground-state search.

TEST INFRASTRUCTURE ONLY. Nothing in the product package imports this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may call it. It shares no code with the CUDA path: it has its
own lattice, tree, disentangler placement, Hamiltonian mapping, effective
operators, Lanczos, sweep and disentangler update, written from the paper in
its order and notation with numpy/scipy library primitives (matmul, einsum,
QR, SVD, symmetric eigensolvers) as single steps.

Citations name the paper's sections, equations, figures and algorithm
("Sec. 4.1.1", "Eq. (contracted)", "Fig. eff-op", "Algorithm 1").

Parity status per module (what pins it is listed in each module header):
  lattice       pinned (Hilbert-curve properties, ED energies, free-fermion chain)
  tree          pinned (link-dimension rule, region partition)
  disentangle   pinned (placement restrictions, dense D^T H D check)
  ttn           pinned (isometry, dense-state brute-force H_eff, energy identity)
  lanczos       pinned (dense eigensolver of the same operator)
  sweep         pinned (exact case m >= 2^(N/2) reaches ED; variational bound)
  de_update     pinned (dense-state RDMs, optimality Tr(u Gamma) = -sum sigma)
  mlp           pinned (finite differences; expm orthogonality, series check;
                Adam steps against hand-derived values)
  observables   pinned (dense 16-site aTTN state; correlation-matrix symmetry)
"""
