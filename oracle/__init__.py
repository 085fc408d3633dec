"""Plain FP64 CPU oracle for the RBM-Chebyshev method.

Hendry, Chen, Weinberg, Feiguin, "Chebyshev expansion of spectral functions
using restricted Boltzmann machines" (arXiv:2103.08804).

THIS PACKAGE IS TEST INFRASTRUCTURE. It exists only so that the tests, the
smoke check and the CPU-baseline leg of the benchmark can check the CUDA path
against a slow, obviously correct restatement of the paper. The product path
(the C-ABI library and its Python binding) never imports, links or executes
anything in here, and nothing in here imports the product package.

Every function works in float64 / complex128 and follows the paper's
equations in the paper's order; library primitives (matrix products,
``numpy.linalg.eigh``, Cholesky) serve as single steps.  Module map:

  lattice   -- sites, periodic nearest-neighbour bonds, the probe S^z_q
               (Sec. V Heisenberg model; Appendix B momentum operator).
  philox    -- Philox4x32-10 counter-based generator (Salmon et al. 2011),
               the random stream both sides draw from.
  rbm       -- the complex RBM amplitude and its log-derivatives (Sec. I).
  sampler   -- Metropolis sampling of |psi_s|^2 with spin-exchange moves
               (Sec. III).
  target    -- the local ratio R(s) = phi_s / psi_s of the projected
               Chebyshev targets (Sec. III, last paragraph).
  sr        -- VMC estimators, Fubini-Study angle, natural-gradient system
               and its shifted solve (Sec. III).
  exact     -- exact diagonalisation and exact Chebyshev vectors on small
               lattices, used to pin everything else.
  chebyshev -- the Chebyshev recursion driver and the moments (Secs. II-III).
  krylov    -- moment correction and the Krylov (generalised
               eigenproblem) projection (Secs. IV-V).
  spectrum  -- the spectral function on a frequency grid: Chebyshev sum
               with Jackson damping (Secs. II, V) and the continued
               fraction of the Krylov projection (Sec. IV).
  groundstate -- ground-state preparation by natural-gradient energy
               descent (Sec. I) with the metric S of Sec. III.
  symmetry  -- translation and rotation projection of the local sequence
               onto every momentum of the square lattice (Appendix A).
  extrapolate -- higher moments from the known ones by linear prediction
               (Sec. VI; the method of the cited Chebyshev-MPS work).
"""

from . import (lattice, philox, rbm, sampler, target, sr, exact, chebyshev, krylov,  # noqa: F401
               spectrum, groundstate, symmetry, extrapolate)
