"""Plain, slow, CPU reference ("oracle") of the M2M training step.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
the CPU-baseline leg of the benchmark may import this package; the library
never does, and nothing here imports the library.

It restates, step by step and in float64 numpy, what the paper defines in
Section 2:

* the merit function F = -1/2 chi^2 + mu S (Eq. 1) with the pseudo-entropy
  S = -sum_i w_i ln(w_i / w_hat_i) (Eq. 2);
* weights adapted while the particles are evolved in the potential (the
  prescription after Eq. 2): dw_i/dt = eps w_i dF/dw_i with dF/dw_i =
  mu dS/dw_i - sum_j K_ij Delta~_j / sigma_j, integrated over one step with
  the gradient held fixed (w <- w exp(eps dt G));
* exponentially time-smoothed residuals Delta~ of Delta_j = (y_j-Y_j)/sigma_j;
* flat priors w_hat = 1/N and the paper's moving priors (Section 2.1):
  w_hat_i = mean weight of the particles in i's cell of integral-of-motion
  space.

Particle orbits follow a kick-drift-kick leapfrog.  Positions and velocities
are kept in the *state precision* (float64, or float32 for the
FP32-compensated form) so that every integer decision (bin and cell
membership) is taken in the same precision as the kernel's; weights, sums,
residuals and the update are float64.

Modules: :mod:`oracle.potentials` (accelerations, potentials), :mod:`oracle.gh`
(Gauss-Hermite kernels), :mod:`oracle.m2m` (push, observe, residual, update,
priors, step loop).  Every function is pinned by a `-m "not gpu"` test in
`tests/test_oracle_*.py`.
"""
from . import potentials, gh, m2m  # noqa: F401
