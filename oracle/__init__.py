"""FP64 CPU oracle for one UDM(m)-PCG(n) ADMM iteration (Sec. 3 of the paper).

TEST INFRASTRUCTURE ONLY: the plain, slow, readable reference that the CUDA
library is checked against. Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the library never does, and the
two share no code. Every function cites the passage it follows.

Pins (what fixes this oracle other than itself) live in tests/test_oracle_*.py.
Parity unpinned: none of the functions here (each has at least one pin).
"""
