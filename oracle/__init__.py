"""FP64 CPU oracle of the thermocapillary central-moment phase-field LBM.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path (``paper_2401_03041_gb300``) and never imports it;
the only common dependency is the seeded input generator ``workloads``.

The oracle is plain, slow and literal: whole-lattice numpy arrays in float64,
one array operation per term of the paper's equations, the central-moment
transform taken from its definition, finite-difference stencils written as
explicit neighbour sums, boundary conditions as explicit branches.  Each
function names the passage of Holzer et al., "Development of a central-moment
phase-field lattice Boltzmann model for thermocapillary flows" (arXiv
2401.03041) that it follows.  Where the paper is silent or garbled, the
reading taken is stated next to the code.
"""
from .stencils import Stencil, stencil  # noqa: F401
from .model import OracleLBM  # noqa: F401
