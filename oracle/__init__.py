"""CPU oracle for the Lindblad steady-state / low-spectrum method -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
import anything from this package.  The library itself never calls it, and it
shares no code with the CUDA path: it is plain NumPy / SciPy in float64 /
complex128, written from the paper's definitions.

Two tiers:
  * ``oracle.dense``  -- the plain definitions, forming the n^2 x n^2
    superoperators explicitly (column-major vectorisation,
    vec(A X B) = (B^T kron A) vec(X)).  Feasible up to n ~ 100.
  * ``oracle.krylov`` -- the paper's own algorithms (Bartels-Stewart resolvent,
    Alg. 2 preconditioner, Alg. 4 Phi-Arnoldi, Alg. 3 GMRES, Alg. 5 shift-invert
    Arnoldi) in plain, unblocked matrix-free form for sizes where the dense
    tier cannot run.

Pins (tests/test_oracle_pins.py, -m "not gpu") tie every function to closed
forms, printed values and invariants.  Functions without such a pin say
"parity unpinned" in their docstring.
"""
