"""Plain FP64 CPU oracle of the many-chain surrogate mMALA step.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this package.  It shares no code with
the CUDA library and never imports it; the two meet only through the seeded
generators in `workloads/`.

Everything is written from the paper (Cao, O'Leary-Roseberry, Ghattas,
"Derivative-informed neural operator acceleration of geometric MCMC for
infinite-dimensional Bayesian inverse problems"): each function cites the
section and equation label it follows.  Arithmetic is float64 throughout;
numpy's matmul / Cholesky / solve serve as library primitives, with no
blocking, fusion or reordering beyond the definitions.

Modules
    philox   counter-based RNG (Philox4x32-10) and Box-Muller normals
    prior    grid, prior operator, KLE and DIS reduced bases, prior draws
    mlp      reduced MLP forward and its Jacobian (reverse and forward mode)
    mmala    misfit, gradient, Gauss-Newton Hessian, proposal, log-acceptance
    chains   the multi-chain driver (one transition of every chain per step)

Every function is pinned by a `-m "not gpu"` test against closed forms,
invariants, brute force or published known-answer vectors; none is "parity
unpinned".
"""
