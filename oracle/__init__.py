"""CPU FP64 oracle for the batched coupled MLMC sample solve.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow, obviously-correct restatement of what the method
computes (Badia, Hampton, Principe, "A massively parallel implementation of
multilevel Monte Carlo for finite element models", arXiv 2111.11788), in
float64, with no blocking, fusion or reordering:

* ``philox``  - counter-based normals xi_k(l, i) (the paper is silent on the
  generator; Philox4x32-10 of Salmon et al., SC'11, with a Box-Muller
  transform built from IEEE-exact operations only).
* ``kle``     - the Karhunen-Loeve expansion of the lognormal diffusion
  coefficient (Sec. 5.2 uses an exponential-covariance KLE with per-dimension
  eigenfunctions; the 1D eigenpairs follow Ghanem & Spanos, ref. [ghanem1991]).
* ``fem``     - Q1 finite elements for -div(kappa grad u) = f with
  homogeneous Dirichlet data on the unit square / cube (Eq. (model), Sec. 2.1),
  the load vector, the QoI weights, and the linear solve (the plain definition
  u = A^{-1} b through a sparse direct factorisation, plus a Jacobi-PCG).
* ``mlmc``    - coupled samples Y_l = Q_l - Q_{l-1} (Eq. (mlmc_average)),
  Welford / Chan level statistics with the 1/N variance of Eq.
  (sample_variance), the estimator, and the optimal allocation of Eq.
  (mlmc_num_samples) inside the adaptive loop of Sec. 2.3 / Algorithm 2.

Every function cites the passage it follows. Parity pins live in
``tests/test_oracle_*.py``.
"""
