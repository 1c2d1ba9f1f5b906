"""FP64 CPU oracle for multigrid with nonstandard (red-black) coarsening.

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import this package.
The CUDA library never calls it and shares no code with it.

`oracle.mg` is a plain level-by-level multigrid code over explicit sparse
matrices (Dirichlet rows and columns removed); Galerkin coarse operators are
formed by an explicit sparse product R A P. `oracle.lfa` holds the local Fourier
analysis symbols the paper derives, used to pin the oracle's convergence factors.
`oracle.spectral` solves the fine-level problem exactly by Fourier diagonalisation
(the operator's symbol, Sec. 2.4), the FP64 reference solution at sizes the sparse
oracle cannot reach; it is pinned to the oracle's sparse direct solve.
"""
