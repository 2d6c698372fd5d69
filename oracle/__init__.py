"""Plain CPU oracle of the space-time multigrid method for the eddy-current equation.

TEST INFRASTRUCTURE ONLY: a slow, obviously correct NumPy/SciPy restatement of the
paper's method (arXiv 1911.09548), used to check the CUDA library.  Only the test
suite, the smoke check and the benchmark's CPU-baseline leg may import it; the
library never does, and it shares no code with the library.

Modules: mesh (Kuhn meshes), fem (Nedelec/P1 matrices, G, K_n), transfer (P_x, P_n),
timeblocks (DG(0)/DG(1) blocks, time transfers), spacetime (L, S, A, transfers),
multigrid (hierarchy, V-cycle, solve, power-iteration rate), load (right-hand side).

Parity of individual V-cycle iterates is pinned only against the CUDA path: the
paper prints no worked example of an iterate ("parity unpinned" for exact iterate
values); every component underneath is pinned by tests against closed forms,
invariants and brute force.
"""
