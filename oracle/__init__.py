"""CPU FP64 oracle for the tensor jump method (TJM) hot path.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct
reference that the CUDA path is checked against.  It shares no code with the
CUDA library: only the tests, the smoke check and the benchmark's CPU-baseline
leg may import it, and the product path never routes through it.

Modules
-------
philox     Philox4x32-10 (SC'11 definition) and the (key, counter) layout.
mps_tjm    O1: the MPS tensor jump method in FP64 (dissipative contraction,
           stochastic jump, dynamic 1-/2-site TDVP with Lanczos exponentials,
           sampling MPS), step by step in the paper's order.
dense      O2: the same Strang-ordered jump schedule on a dense state vector,
           and O3: the dense Lindblad master equation for small chains.

Pins (tests/test_oracle_pins.py, tests/test_oracle_ensemble.py) fix every part
against closed forms, library routines on special cases, dense computations or
exactly solvable limits, with one exception: the TDVP sweep when a two-site
block's rank exceeds chi_max and is truncated (mps_tjm.Sweeper) is parity
unpinned -- no closed form exists; it is checked by its exactness at full bond
dimension, by exact update counts and exact norm and energy conservation of the
dynamic switch where nothing is truncated, and by its monotone convergence to
the dense evolution as chi_max grows.
"""
