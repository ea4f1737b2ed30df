"""FP64 CPU oracle for the joint p0 / speed-of-sound reconstruction (test infrastructure).

This package is the plain, slow, obviously correct statement of what the GPU
library computes.  It is TEST INFRASTRUCTURE: only ``tests/``, the smoke check
in ``__graft_entry__.py`` and the CPU-baseline leg of ``bench.py`` may import
it.  The product path (the CUDA library and its Python binding) never imports,
links or calls anything here, and nothing here imports the product path.  The
only code both sides share is the seeded input generator ``pat_synth``, which
holds no arithmetic of the method.

Contents (paper sections in brackets):

* ``grid``      wavenumbers, k-space correction, staggering shifts, PML, time
                step (Sec. 2.1 forward model; Table 1 discretisations)
* ``sensors``   bilinear point-sensor sampling matrix S (Sec. 4: point sensors)
* ``forward``   k-space pseudospectral forward solve f^i(p0^i, c) and the
                discrete acoustic energy (Eq. WaveEquation, Eq. ObservationModel)
* ``adjoint``   objective and exact discrete adjoint gradient (Eq.
                Minimised_functional, Eq. AdjointEquation, Eqs. gradient_p0 /
                gradient_sos)
* ``lbfgs``     projected L-BFGS with backtracking (Eq. BFGS_iterations,
                Algorithm 1, Eq. bound_constraints)
* ``multigrid`` coarse-to-fine schedule, prolongation, data time interpolation
                (Sec. 3.1, Sec. 4.1.2)
* ``metrics``   relative errors (Eq. RelativeError)
* ``prior``     Ornstein-Uhlenbeck prior terms with a dense Cholesky factor (Eq.
                Minimised_functional, Sec. 4.1.2)
* ``unet``      plain-PyTorch CPU reference of the warm-start network (no paper
                counterpart; imported on its own, it needs torch)

Every function is pinned by a ``-m "not gpu"`` test against closed forms,
invariants, finite differences or library routines; none is "parity
unpinned".
"""
from . import grid, sensors, forward, adjoint, lbfgs, multigrid, metrics, prior  # noqa: F401
