"""CPU FP64 oracle for the indefinite least squares (ILS) solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference leg may import anything from this
package.  The CUDA library never calls it and shares no code with it: the two
sides meet only in the seeded input generators of ``workloads``.

Every function here is a plain, slow restatement of the paper's definitions
(Zhang & Li, "Splitting-based randomized iterative methods for solving
indefinite least squares problem"), in float64, with numpy/scipy routines
(matmul, QR, Cholesky, triangular solve) used only as single steps.

Parity status (what pins each function, see ``tests/test_oracle_*.py``):
  * qr_cholesky_solve / normal_equation_solve: exact rational solve for n <= 4,
    numpy ``lstsq`` for q = 0, and each other.
  * sp_solve: Theorem 2.1 contraction in the energy norm against rho from a
    generalized eigenvalue solve; convergence to the direct solution; q = 0
    converges in one step; the paper's Tables 2-3 iteration count.
  * sp_rk_rgs_solve: Theorem 3.2 fixed point (tight inner tolerance reproduces
    SP's outer iterates); the Pythagorean identity of Theorem 3.3 for the RGS
    half-step; j1 = j2 reduces to coordinate descent (Sec. 4).
  * sp_scd_solve: Theorem 4.1's exact energy decrease per step; alpha = n is the
    greedy (Motzkin) rule; the rank sampler has the same law as the literal
    alpha/subset sampler (exact enumeration for small n).
  * theta_at (the inner-stop schedule): its closed form; gamma = 1 reproduces the
    constant stop; each outer step within ||Abar1^{-1}|| theta_k ||r_k|| of the SP step.
  * philox4x32_10: the published known-answer vectors.
  * mlp_*: central finite differences.
  * sparse.*: hand-computed products of a literal 4 x 3 CSR matrix; the dense
    oracle on the densified matrix; the generator's pattern statistics.
"""
from .ils_oracle import *  # noqa: F401,F403
from .philox import philox4x32_10, step_uniforms, words_to_uniform  # noqa: F401
from . import sparse  # noqa: F401
